// The whole Gauss-Newton loop of Sec. 2.3.1 in one persistent, cooperatively launched kernel.
//
// A problem is worked on by a group of co-resident blocks (the whole grid for one pair, or a
// block range of a wave of pairs).  Per GN iteration:
//   evaluation at b        J, grad J, d, e, 1/diag (Eq. 1-5)                       | barrier + sums
//   Jacobi PCG             H q = -grad J (pcg_run: init + up to max_it iterations) | its barriers
//                                                                                  | barrier
//   gamma = 1 trial        J, grad J, d, e, 1/diag at b + q, grad^T q              | barrier + sums
//   halvings (if needed)   J(b + 2^-t q), kGnLsT trials per pass                   | barrier + sums
//   update                 gamma = 1: none (the trial wrote b + q into the second field buffer,
//                          which becomes the iterate); 0 < gamma < 1: b += gamma q | barrier
// Every barrier is also the reduction of its phase's sums (grid_allreduce: a fixed order, in
// double-float), so every block of the group holds the same totals and takes the same scalar
// decisions (Armijo acceptance, the halving that wins, the stop on a non-finite J) without
// another round trip; block 0 of the group mirrors them into the device state and writes the
// statistics rows.  When the gamma = 1 trial is accepted its coefficients are those of the next
// iterate and the next evaluation is skipped, as in the separate-kernel solve.
//
// The arithmetic per node is that of the separate kernels (eval_item, ls_items, pcg_run); only
// the per-block partial sums group 768 threads instead of 256, so sums (and J) agree with the
// separate-kernel solve to rounding.  Arrays written inside the launch (b, q, grad, d, e, 1/diag
// and the PCG vectors) are read with ordinary loads, never through the read-only path.
//
// Ordering: the evaluation's and the trial's barriers publish d, e, 1/diag and grad before the
// PCG reads them at other blocks' nodes; the barrier after the PCG publishes q (read by the trial
// at neighbouring nodes) and keeps the trial's writes of d, e, 1/diag after every block's last
// stencil read.  The next PCG's first barrier publishes the trial's b + q before the next trial
// reads it at neighbouring nodes; an explicit update (gamma < 1) ends with a barrier, since the
// next PCG's init zeroes q at other threads' nodes.
//
// Register budget: a 768-thread block per SM leaves 80 registers per thread, about what the
// evaluation and the PCG each need alone.  So little of one phase lives in registers across
// another: the problem's geometry and arguments are read from the launch parameters where used,
// and the loop's scalars (J and its terms, the stashed trial terms, g^T q) sit in shared memory,
// written by thread 0 and read after a later barrier.  Some spilling remains: measured at 3T, the
// PCG step takes ~194 us here against ~176 us as its own kernel and the trial ~58 against ~38 us,
// so a single solve is faster as separate kernels (pcg_path 0); this form serves the batched
// waves and the one-launch solve.
#include "eval_march.cuh"
#include "pcg_run.cuh"

namespace hysco {

constexpr int kGnLsT = 2;   // Armijo halvings per pass (3 sums each fit one barrier's slots)
constexpr int kGnUTrial = 2;   // nodes per load group of the trial inside the loop (registers)

// this thread's share of an evaluation at b (TRIAL: at b + q, writing b + q to fout): the column
// march's work items rank * warps + warp, stepping by the group's warps
template <typename TI, bool TRIAL>
__device__ __forceinline__ EvalAcc gn_eval(const Geo& g, const GnArgs& ga, const float* b,
                                           float* fout, int rank, int size) {
  const TI* Ip = static_cast<const TI*>(ga.Ip);
  const TI* Im = static_cast<const TI*>(ga.Im);
  const float* q = ga.pcg.x;
  float* grad_p = ga.grad_p;
  float* dco = const_cast<float*>(ga.pcg.dco);
  float* eco = const_cast<float*>(ga.pcg.eco);
  float* invd = const_cast<float*>(ga.pcg.invd);
  const int warps = blockDim.x >> 5, items = g.ntile * g.nseg;
  EvalAcc acc;
  for (int w = rank * warps + (threadIdx.x >> 5); w < items; w += size * warps) {
    if (TRIAL)
      eval_item<TI, true, false, kGnUTrial, 6, false>(g, Ip, Im, b, q, nullptr, nullptr,
                                                         grad_p, dco, eco, invd, 0.f, w,
                                                         threadIdx.x & 31, acc, fout);
    else
      eval_item<TI, false, false, kEvalU, 2, false>(g, Ip, Im, b, nullptr, nullptr, nullptr,
                                                     grad_p, dco, eco, invd, 0.f, w,
                                                     threadIdx.x & 31, acc);
  }
  return acc;
}

// the PCG of the GN step (pcg_run on the group), false when a barrier timed out
template <int P>
__device__ __forceinline__ bool gn_pcg(const Geo& g, const GnArgs& ga, int rank, int size,
                                       unsigned* gen) {
  __shared__ float shf[32 * 2];
  __shared__ df32 shd[32 * 2];
  extern __shared__ float4 slots[];
  const PcgArgs& a = ga.pcg;
  unsigned gn = *gen;
  const bool ok = pcg_run<P, false>(g, a, BarrierGroup{rank, size}, shf, shd, slots, gn);
  *gen = gn;
  return ok;
}

// this thread's share of kGnLsT halvings' sums (D, S, P per trial, t = t0 ..): the kBlock-wide
// virtual blocks rank * (blockDim / kBlock) + .., stepping by the group's virtual blocks
template <typename TI>
__device__ __forceinline__ void gn_ls(const Geo& g, const GnArgs& ga, const float* b, int t0,
                                      int rank, int size, float* v) {
  const int vper = blockDim.x / kBlock;
  float aD[kGnLsT], aS[kGnLsT], aP[kGnLsT], aR[kGnLsT], agq = 0.f;
#pragma unroll
  for (int t = 0; t < kGnLsT; ++t) { aD[t] = 0.f; aS[t] = 0.f; aP[t] = 0.f; aR[t] = 0.f; }
  ls_items<TI, kSeg, kGnLsT, false, false>(
      g, static_cast<const TI*>(ga.Ip), static_cast<const TI*>(ga.Im), b, ga.pcg.x,
      nullptr, nullptr, t0, rank * vper + threadIdx.x / kBlock, size * vper,
      threadIdx.x % kBlock, aD, aS, aP, aR, agq);
#pragma unroll
  for (int t = 0; t < kGnLsT; ++t) { v[3 * t] = aD[t]; v[3 * t + 1] = aS[t]; v[3 * t + 2] = aP[t]; }
}

// the loop's scalars, in shared memory (thread 0 writes them, every thread reads them after a
// later barrier)
struct GnScalars {
  double J, D, S, P, gnorm;       // at the iterate
  double Jn, Dn, Sn, Pn, gnn;     // at b + q, from the accepted gamma = 1 trial
  double gq;                      // grad^T q
};

template <typename TI, int P>
__device__ __forceinline__ void gn_run(const Geo& g, const GnArgs& a, GnScalars& sc,
                                       BarrierGroup grp, float* shf, df32* shd) {
  DevState* const st = a.pcg.st;
  const bool lead = grp.rank == 0 && threadIdx.x == 0;
  unsigned gen = 0;
  auto fail = [&]() {   // a barrier timed out: record it and leave (every block then times out)
    if (threadIdx.x == 0) { st->status = -6; st->stop = 1; }
  };
  auto barrier = [&]() {
    float v[1] = {0.f};
    return grid_allreduce<1>(v, a.pcg.sync, ++gen, shf, shd, 0, -1, kBarrierSpinCycles, grp);
  };
  if (st->stop) return;
  // the iterate lives in buffer cur (0: the caller's b, 1: bscr); an accepted gamma = 1 trial,
  // which wrote b + q to the other buffer, flips cur.  On exit the caller's buffer holds it.
  auto buf = [&](int k) { return k == 0 ? a.b : a.bscr; };
  int cur = 0;
  auto copy_back = [&]() {
    if (cur == 0) return;
    const float* src = a.bscr;
    float* dst = a.b;
    const int nf = g.nf;
    for (int i = grp.rank * blockDim.x + threadIdx.x; i < nf; i += grp.size * blockDim.x)
      dst[i] = src[i];
  };
  bool fresh = false;   // the coefficients at the iterate are in place (accepted gamma = 1 trial)
  for (int it = 0; it < a.gn_iters; ++it) {
    // ---- evaluation at b --------------------------------------------------------------------
    if (!fresh) {
      const EvalAcc acc = gn_eval<TI, false>(g, a, buf(cur), nullptr, grp.rank, grp.size);
      float v[4] = {acc.D, acc.S, acc.P, acc.G};
      double tot[4];
      if (!group_sum_d<4>(v, tot, a.pcg.sync, gen, shf, shd, grp)) { fail(); return; }
      const double hv = 0.5 * (double)g.vol;
      const double D = hv * tot[0], S = hv * tot[1], Pv = hv * tot[2];
      const double J = D + g.alpha_d * S + g.beta_d * Pv;
      if (threadIdx.x == 0) {
        sc.J = J; sc.D = D; sc.S = S; sc.P = Pv; sc.gnorm = sqrt(tot[3]);
      }
      if (lead) st->status = isnan(J) ? -4 : (isinf(J) ? 1 : 0);
      if (!isfinite(J)) {   // the run stops: this row keeps J, later rows are NaN
        if (lead) {
          st->J = J; st->D = D; st->S = S; st->P = Pv; st->gnorm = sqrt(tot[3]);
          st->stop = 1;
          st->stop_iter = it;
          if (a.stats) {
            const double nan = __longlong_as_double(0x7ff8000000000000LL);
            for (int r = it; r < a.gn_iters; ++r) {
              double* row = a.stats + r * 10;
              for (int k = 0; k < 10; ++k) row[k] = nan;
              if (r == it) { row[0] = J; row[1] = D; row[2] = S; row[3] = Pv; }
            }
          }
          st->gn_iter = a.gn_iters;
        }
        copy_back();
        return;
      }
    } else {
      if (threadIdx.x == 0) {
        sc.J = sc.Jn; sc.D = sc.Dn; sc.S = sc.Sn; sc.P = sc.Pn; sc.gnorm = sc.gnn;
      }
      if (lead) st->status = 0;
      fresh = false;
    }
    // ---- Jacobi PCG for H q = -grad J, then a barrier that publishes q ------------------------
    if (!gn_pcg<P>(g, a, grp.rank, grp.size, &gen)) return;
    if (!barrier()) { fail(); return; }
    // ---- the gamma = 1 trial: a full evaluation at b + q, b + q into the other buffer --------
    double gamma = 0.0;
    int trials = 0;
    bool done;
    {
      const EvalAcc acc = gn_eval<TI, true>(g, a, buf(cur), buf(cur ^ 1), grp.rank, grp.size);
      float v[5] = {acc.D, acc.S, acc.P, acc.G, acc.GQ};
      double tot[5];
      if (!group_sum_d<5>(v, tot, a.pcg.sync, gen, shf, shd, grp)) { fail(); return; }
      const double gq = tot[4], hv = 0.5 * (double)g.vol;
      const double Dt = hv * tot[0], St = hv * tot[1], Pt = hv * tot[2];
      const double Jt = Dt + g.alpha_d * St + g.beta_d * Pt;
      if (!(gq < 0.0)) {                     // not a descent direction: keep the iterate
        done = true;
      } else {
        trials = 1;
        if (Jt <= sc.J + a.c1 * gq) {     // Armijo with gamma = 1
          done = true;
          gamma = 1.0;
          fresh = true;
        } else {
          done = a.ls_max <= 1;
        }
      }
      __syncthreads();   // every thread has read sc.J before thread 0 may overwrite the stash
      if (threadIdx.x == 0) {
        sc.gq = gq;
        if (fresh) { sc.Jn = Jt; sc.Dn = Dt; sc.Sn = St; sc.Pn = Pt; sc.gnn = sqrt(tot[3]); }
      }
    }
    // ---- Armijo halvings gamma = 2^-t, t = 1 .. ls_max - 1 (J only) ---------------------------
    for (int t0 = 1; !done && t0 < a.ls_max; t0 += kGnLsT) {
      float v[3 * kGnLsT];
      double tot[3 * kGnLsT];
      gn_ls<TI>(g, a, buf(cur), t0, grp.rank, grp.size, v);
      if (!group_sum_d<3 * kGnLsT>(v, tot, a.pcg.sync, gen, shf, shd, grp)) { fail(); return; }
      const double hv = 0.5 * (double)g.vol;
      for (int t = 0; t < kGnLsT && t0 + t < a.ls_max; ++t) {
        const double gm = ldexp(1.0, -(t0 + t));
        const double Jt = hv * tot[3 * t] + g.alpha_d * hv * tot[3 * t + 1] +
                          g.beta_d * hv * tot[3 * t + 2];
        trials = t0 + t + 1;
        if (Jt <= sc.J + a.c1 * gm * sc.gq) { done = true; gamma = gm; break; }
      }
      if (!done && t0 + kGnLsT >= a.ls_max) { done = true; gamma = 0.0; }
    }
    // ---- statistics, then the new iterate ------------------------------------------------------
    if (lead) {
      st->J = sc.J; st->D = sc.D; st->S = sc.S; st->P = sc.P; st->gnorm = sc.gnorm;
      st->gq = sc.gq; st->gamma = gamma; st->ls_trials = trials; st->ls_done = 1;
      st->coef_fresh = fresh ? 1 : 0;
      if (fresh) {
        st->Jn = sc.Jn; st->Dn = sc.Dn; st->Sn = sc.Sn; st->Pn = sc.Pn; st->gnorm_n = sc.gnn;
        st->status_n = 0;
      }
      if (a.stats) {
        double* row = a.stats + it * 10;
        row[0] = sc.J; row[1] = sc.D; row[2] = sc.S; row[3] = sc.P;
        row[4] = sc.gnorm; row[5] = sc.gq; row[6] = gamma; row[7] = st->pcg_iter;
        row[8] = st->relres; row[9] = trials;
      }
      st->gn_iter = it + 1;
    }
    if (gamma == 1.0) {
      cur ^= 1;   // b + q, written by the trial
    } else if (gamma != 0.0) {
      update_nodes<false>(g, buf(cur), a.pcg.x, (float)gamma,
                          grp.rank * blockDim.x + threadIdx.x, grp.size * blockDim.x);
      if (!barrier()) { fail(); return; }   // the next evaluation reads b, the next PCG zeroes q
    }
  }
  copy_back();
}

// The problems of a wave: problem i on blocks blk0[i] .. blk0[i] + nblk[i] - 1, each group with
// its own sync words and barriers, so the problems' GN loops proceed independently.
template <typename TI>
__global__ void __launch_bounds__(kPcgBlock, 1)
k_gn_wave(const GnWave wv) {
  __shared__ float shf[32 * kSyncMaxK];
  __shared__ df32 shd[kSyncMaxK];
  __shared__ GnScalars sc;
  int i = 0;
  while (i + 1 < wv.n && (int)blockIdx.x >= wv.blk0[i + 1]) ++i;
  if ((int)blockIdx.x >= wv.blk0[i] + wv.nblk[i]) return;   // spare blocks of the launch
  const BarrierGroup grp{(int)blockIdx.x - wv.blk0[i], wv.nblk[i]};
  const Geo& g = wv.g[i];
  if (g.p == 0) gn_run<TI, 0>(g, wv.a[i], sc, grp, shf, shd);
  else if (g.p == 1) gn_run<TI, 1>(g, wv.a[i], sc, grp, shf, shd);
  else gn_run<TI, 2>(g, wv.a[i], sc, grp, shf, shd);
}

template <typename TI>
static int gn_setup_t(int device, int onchip) {
  int sms = 0, coop = 0, optin = 0, per_sm = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess ||
      cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, device) != cudaSuccess ||
      !coop ||
      cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, device) !=
          cudaSuccess)
    return 0;
  cudaFuncAttributes fa;
  if (cudaFuncGetAttributes(&fa, k_gn_wave<TI>) != cudaSuccess ||
      cudaFuncSetAttribute(k_gn_wave<TI>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           optin - (int)fa.sharedSizeBytes) != cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_gn_wave<TI>, kPcgBlock,
                                                    pcg_onchip_bytes(onchip)) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return per_sm;
}

int gn_setup(int device, int dtype, int onchip) {
  switch (dtype) {
    case 0: return gn_setup_t<float>(device, onchip);
    case 1: return gn_setup_t<__nv_bfloat16>(device, onchip);
    default: return gn_setup_t<__half>(device, onchip);
  }
}

cudaError_t launch_gn_wave(const GnWave& w, int dtype, int grid, int onchip_max, unsigned* sync,
                           size_t sync_words, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(sync, 0, sync_words * sizeof(unsigned), s);
  if (e != cudaSuccess) return e;
  GnWave copy = w;
  void* args[] = {&copy};
  const void* fn = dtype == 0 ? (const void*)k_gn_wave<float>
                              : (dtype == 1 ? (const void*)k_gn_wave<__nv_bfloat16>
                                            : (const void*)k_gn_wave<__half>);
  return cudaLaunchCooperativeKernel(fn, dim3(grid), dim3(kPcgBlock), args,
                                     pcg_onchip_bytes(onchip_max), s);
}

}  // namespace hysco
