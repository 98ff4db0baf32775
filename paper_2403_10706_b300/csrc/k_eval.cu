// Objective kernels: J(b) = D + alpha S + beta P with gradient and Gauss-Newton coefficients
// (Sec. 2.1 Eq. 1-5, Sec. 2.3.1), the Armijo line search, the GN update, the corrected images
// (Sec. 2.4) and the interpolation cell indices.
//
// Thread mapping ("column march"): thread = (PE column c, segment of nodes along PE).
// Consecutive threads own consecutive columns, so for pe_dim != 2 every PE step is a coalesced
// row access.  Absent neighbours are read at the node itself (zero Laplacian difference); an
// interpolation tap outside the image is a predicated-off load that reads 0.
// Per cell j (nodes j, j+1):
//   bc = (b_j + b_{j+1}) / 2, delta = b_{j+1} - b_j, t+- = j +- bc      (averaging / FD operators)
//   I(t) = I[i] + w (I[i+1] - I[i]), i = floor(t), w = t - i, I = 0 outside 0..m-1
//   T+ = I+(t+)(1 + delta), T- = I-(t-)(1 - delta), r = T+ - T-         (Eq. 1)
//   a = I+'(1 + delta) + I-'(1 - delta), c = I+(t+) + I-(t-);  dr/db_j = a/2 - c, dr/db_{j+1} = a/2 + c
// Per node k the Gauss-Newton Hessian restricted to the column is tridiagonal:
//   d_k = (dr_{k-1}/db_k)^2 + (dr_k/db_k)^2 + psi_{k-1} + psi_k,   e_k = dr_k/db_k * dr_k/db_{k+1} - psi_k
// with psi = beta/2 phi''(delta); H v = vol [e_{k-1} v_{k-1} + d_k v_k + e_k v_{k+1} + alpha (L v)_k],
// and the Jacobi preconditioner is 1 / (vol [d_k + alpha L_kk]).
#include <algorithm>

#include "eval_march.cuh"
#include "grid_sync.cuh"

namespace hysco {

// ------------------------------------------------------------------------------------------
// J, grad J, the tridiagonal GN coefficients (d, e) and the inverse Jacobi diagonal
// ------------------------------------------------------------------------------------------

constexpr int kEvalMinBlocks = 3;   // resident blocks per SM the registers must allow (80 regs)

// Whether an objective launch has nothing to do: a stopped run, a line search already decided,
// or (in a solve, when the previous gamma = 1 trial was accepted) coefficients already in place,
// whose stashed terms one thread promotes.  The same for every block, so no block enters the
// reduction and the ticket counter is untouched.
template <bool TRIAL, bool PROX>
__device__ __forceinline__ bool eval_skip(int it, DevState* st) {
  if (TRIAL) return st->stop || st->ls_done;
  if (it >= 0) {
    if (st->stop) return true;
    if (st->coef_fresh) {
      if (blockIdx.x == 0 && threadIdx.x == 0) promote_stash(st, PROX);
      return true;
    }
    return false;
  }
  return it < -1 && st->stop;   // it = -2: a fresh evaluation unless the run has stopped
}

// The finisher of an objective launch (the last block, after the grid sum of D, S, P, sum g^2,
// grad^T q and, with PROX, ||b - c||^2): J and its terms into the device state, and for the
// trial the Armijo decision for gamma = 1.
template <bool TRIAL, bool PROX, int NV>
__device__ __forceinline__ void eval_finish(const Geo& g, const double (&tot)[NV], float rho,
                                            int it, int ls_max, double c1, DevState* st,
                                            double* terms) {
  double hv = 0.5 * (double)g.vol;
  double D = hv * tot[0], S = hv * tot[1], P = hv * tot[2];
  double J = D + g.alpha_d * S + g.beta_d * P;
  if (PROX) {
    st->prox = hv * tot[NV - 1];
    J += (double)rho * st->prox;
  }
  if (!TRIAL) {
    st->J = J; st->D = D; st->S = S; st->P = P;
    if (PROX) st->Jacc = J;
    st->gnorm = sqrt(tot[3]);
    st->status = isnan(J) ? -4 : (isinf(J) ? 1 : 0);
    st->ls_done = 0; st->ls_trials = 0; st->gamma = 0.0; st->gq = 0.0;
    st->pcg_done = 0; st->pcg_iter = 0; st->relres = 0.0;
    st->coef_fresh = 0;
    if (it >= 0 && !isfinite(J)) { st->stop = 1; st->stop_iter = it; }
    if (it == -1) st->stop = 0;   // a single evaluation starts no run
    if (terms) {                  // a single evaluation's J, D, S, P for the caller
      terms[0] = J; terms[1] = D; terms[2] = S; terms[3] = P;
    }
  } else {
    double gq = tot[4];
    st->gq = gq;
    st->coef_fresh = 0;
    if (!(gq < 0.0)) {             // not a descent direction: keep the iterate
      st->ls_done = 1; st->gamma = 0.0; st->ls_trials = 0;
    } else {
      st->ls_trials = 1;
      if (J <= st->J + c1 * gq) {  // Armijo with gamma = 1
        st->ls_done = 1; st->gamma = 1.0;
        if (PROX) st->Jacc = J;
        st->coef_fresh = 1;
        st->Jn = J; st->Dn = D; st->Sn = S; st->Pn = P;
        st->gnorm_n = sqrt(tot[3]);
        st->status_n = 0;
      } else if (ls_max <= 1) {
        st->ls_done = 1; st->gamma = 0.0;
      }
    }
  }
}

// TRIAL = false: evaluation at b (GN iteration `it`, or it = -1 for a single hysco_eval call, or
// it = -2 for a fresh evaluation that a stopped run skips).  In a solve, when the previous
// gamma = 1 trial was accepted the coefficients at this iterate are already in place: one thread
// promotes the stashed terms and every block returns at once (no block enters the reduction, so
// the ticket counter is untouched).
// TRIAL = true: the gamma = 1 Armijo trial, an evaluation at b + q.
// PROX (the ADMM b-subproblem of Sec. 2.3.2): J gains rho vol/2 ||b - c||^2 (c pitched, rho the
// device state's admm_rho), the gradient rho vol (b - c) and the GN coefficient d the constant rho;
// with the split geometry (in-plane Laplacian weights 0) S is the PE part S3 alone.
// One warp per work item of the column march (eval_item): the grid is ntile * nseg warps.
template <typename TI, bool TRIAL, bool PROX, int U, int OUT>
__global__ void __launch_bounds__(kBlock, kEvalMinBlocks)
k_eval(Geo g, const TI* __restrict__ Ip, const TI* __restrict__ Im, const float* __restrict__ b,
       const float* __restrict__ q, const float* __restrict__ cpx, float* __restrict__ grad,
       float* __restrict__ grad_p, float* __restrict__ dco, float* __restrict__ eco,
       float* __restrict__ invd, int it, int ls_max, double c1, float* partials,
       unsigned* counter, DevState* st, double* terms) {
  if (eval_skip<TRIAL, PROX>(it, st)) return;
  const float rho = PROX ? st->admm_rho : 0.f;
  EvalAcc acc;
  const int wid = blockIdx.x * (kBlock / 32) + (threadIdx.x >> 5);
  if (wid < g.ntile * g.nseg)
    eval_item<TI, TRIAL, PROX, U, OUT, true>(g, Ip, Im, b, q, cpx, grad, grad_p, dco, eco, invd,
                                             rho, wid, threadIdx.x & 31, acc);
  constexpr int NV = PROX ? 6 : 5;
  float v[NV];
  v[0] = acc.D; v[1] = acc.S; v[2] = acc.P; v[3] = acc.G; v[4] = acc.GQ;
  if (PROX) v[NV - 1] = acc.R;
  double tot[NV];
  if (grid_sum<NV>(v, partials, counter, tot)) eval_finish<TRIAL, PROX, NV>(g, tot, rho, it, ls_max, c1, st, terms);
}

// ------------------------------------------------------------------------------------------
// Armijo line search: J(b + gamma_t q) for gamma_t = 2^-t, t = t0 .. t0+T-1, in one pass; the
// first accepted trial in order wins, exactly as sequential halving would pick it.  The first
// gamma = 1 trial is a full evaluation (launch_eval_trial); this kernel tries the halvings.
// ------------------------------------------------------------------------------------------

template <typename TI, int SEG, int T, bool PROX>
__global__ void __launch_bounds__(kBlock)
k_linesearch(Geo g, const TI* __restrict__ Ip, const TI* __restrict__ Im,
             const float* __restrict__ b, const float* __restrict__ q,
             const float* __restrict__ cpx, const float* __restrict__ grad, int t0, int ls_max,
             double c1, float* partials, unsigned* counter, DevState* st) {
  if (st->stop || st->ls_done) return;
  float aD[T], aS[T], aP[T], aR[T], agq = 0.f;
#pragma unroll
  for (int t = 0; t < T; ++t) { aD[t] = 0.f; aS[t] = 0.f; aP[t] = 0.f; aR[t] = 0.f; }
  // grid-stride over work items; accumulators carry across items
  ls_items<TI, SEG, T, PROX, true>(g, Ip, Im, b, q, cpx, grad, t0, blockIdx.x, gridDim.x,
                                   threadIdx.x, aD, aS, aP, aR, agq);
  constexpr int NV = (PROX ? 4 : 3) * T + 1;
  float v[NV];
  double tot[NV];
#pragma unroll
  for (int t = 0; t < T; ++t) {
    v[3 * t] = aD[t]; v[3 * t + 1] = aS[t]; v[3 * t + 2] = aP[t];
    if (PROX) v[3 * T + 1 + t] = aR[t];
  }
  v[3 * T] = agq;
  if (grid_sum<NV>(v, partials, counter, tot)) {
    if (t0 == 0) st->gq = tot[3 * T];
    double gq = st->gq, J = st->J, hv = 0.5 * (double)g.vol;
    if (!(gq < 0.0)) { st->ls_done = 1; st->gamma = 0.0; st->ls_trials = 0; return; }
    for (int t = 0; t < T && t0 + t < ls_max; ++t) {
      double gm = ldexp(1.0, -(t0 + t));
      double Jt = hv * tot[3 * t] + g.alpha_d * hv * tot[3 * t + 1] + g.beta_d * hv * tot[3 * t + 2];
      if (PROX) Jt += (double)st->admm_rho * hv * tot[3 * T + 1 + t];
      st->ls_trials = t0 + t + 1;
      if (Jt <= J + c1 * gm * gq) {
        st->ls_done = 1; st->gamma = gm;
        if (PROX) st->Jacc = Jt;
        return;
      }
    }
    if (t0 + T >= ls_max) { st->ls_done = 1; st->gamma = 0.0; }
  }
}

// the statistics row of GN iteration `it` (one thread): J, D, S, P, ||grad||, grad^T q, gamma,
// PCG iterations, relative residual, line-search trials; NaN past a stop
__device__ __forceinline__ void write_stats_row(const DevState* st, double* stats, int it) {
  if (!stats) return;
  const double nan = __longlong_as_double(0x7ff8000000000000LL);
  const bool stopped_before = st->stop && st->stop_iter < it;
  const bool stopped_now = st->stop && st->stop_iter == it;
  double* row = stats + it * 10;
  if (stopped_before) {
    for (int i = 0; i < 10; ++i) row[i] = nan;
  } else {
    row[0] = st->J; row[1] = st->D; row[2] = st->S; row[3] = st->P;
    if (stopped_now) {
      for (int i = 4; i < 10; ++i) row[i] = nan;
    } else {
      row[4] = st->gnorm; row[5] = st->gq; row[6] = st->gamma; row[7] = st->pcg_iter;
      row[8] = st->relres; row[9] = st->ls_trials;
    }
  }
}

// b += gamma q (b in the caller's layout, q pitched); block 0 records the iteration's statistics
__global__ void __launch_bounds__(kBlock)
k_update(Geo g, float* __restrict__ b, const float* __restrict__ q, int it, double* stats,
         DevState* st) {
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    write_stats_row(st, stats, it);
    st->gn_iter = it + 1;
  }
  if (st->stop) return;
  const float gam = (float)st->gamma;
  if (gam == 0.0f) return;
  update_nodes<true>(g, b, q, gam, blockIdx.x * blockDim.x + threadIdx.x, gridDim.x * blockDim.x);
}

// The Armijo halvings and the GN update of one step in one cooperative launch (kPcgBlock threads,
// one block per SM, all co-resident): when the gamma = 1 trial left the line search undecided,
// trials gamma_t = 2^-t, t = 1 .. ls_max - 1, kLsPass per pass, each pass's sums reduced by a
// device-wide barrier so that every block takes the same decision (the first accepted trial in
// order, exactly as sequential halving); then b += gamma q.  After an accepted gamma = 1 trial it
// is the update alone, with no barrier.  eval_next: then, unless an accepted gamma = 1 trial left
// the next iterate's coefficients in place (the next PCG launch then promotes the trial's stash),
// the next GN step's evaluation at the new b, by the same grid after a barrier (the evaluation's
// own launch is then not made).  sync: zeroed words (the step's PCG launch clears them).
constexpr int kLsPass = 2;   // halvings per pass (3 sums each fit one barrier's slots)

template <typename TI>
__global__ void __launch_bounds__(kPcgBlock)
k_ls_update(Geo g, const TI* __restrict__ Ip, const TI* __restrict__ Im, float* __restrict__ b,
            const float* __restrict__ q, int it, int ls_max, double c1, double* stats,
            unsigned* sync, DevState* st, int eval_next, float* grad_p, float* dco, float* eco,
            float* invd, unsigned* clear, int nclear) {
  __shared__ float shf[32 * kSyncMaxK];
  __shared__ df32 shd[kSyncMaxK];
  const bool lead = blockIdx.x == 0 && threadIdx.x == 0;
  const int T = gridDim.x * blockDim.x, gtid = blockIdx.x * blockDim.x + threadIdx.x;
  double gamma = st->gamma;
  unsigned gen = 0;
  // the next step's PCG launch's barrier words (not used by this launch)
  for (int i = gtid; i < nclear; i += T) clear[i] = 0u;
  if (!st->stop && !st->ls_done) {
    const double gq = st->gq, J = st->J, hv = 0.5 * (double)g.vol;
    const int vper = blockDim.x / kBlock;
    int trials = st->ls_trials;
    bool done = !(gq < 0.0);
    gamma = 0.0;
    for (int t0 = 1; !done && t0 < ls_max; t0 += kLsPass) {
      float aD[kLsPass], aS[kLsPass], aP[kLsPass], aR[kLsPass], agq = 0.f;
#pragma unroll
      for (int t = 0; t < kLsPass; ++t) { aD[t] = 0.f; aS[t] = 0.f; aP[t] = 0.f; aR[t] = 0.f; }
      ls_items<TI, kSeg, kLsPass, false, true>(g, Ip, Im, b, q, nullptr, nullptr, t0,
                                               blockIdx.x * vper + threadIdx.x / kBlock,
                                               gridDim.x * vper, threadIdx.x % kBlock, aD, aS,
                                               aP, aR, agq);
      float v[3 * kLsPass];
      double tot[3 * kLsPass];
#pragma unroll
      for (int t = 0; t < kLsPass; ++t) {
        v[3 * t] = aD[t]; v[3 * t + 1] = aS[t]; v[3 * t + 2] = aP[t];
      }
      if (!group_sum_d<3 * kLsPass>(v, tot, sync, gen, shf, shd)) {
        if (threadIdx.x == 0) { st->status = -6; st->stop = 1; }
        return;
      }
      for (int t = 0; t < kLsPass && t0 + t < ls_max; ++t) {
        const double gm = ldexp(1.0, -(t0 + t));
        const double Jt = hv * tot[3 * t] + g.alpha_d * hv * tot[3 * t + 1] +
                          g.beta_d * hv * tot[3 * t + 2];
        trials = t0 + t + 1;
        if (Jt <= J + c1 * gm * gq) { done = true; gamma = gm; break; }
      }
      if (!done && t0 + kLsPass >= ls_max) done = true;
    }
    if (lead) { st->ls_done = 1; st->gamma = gamma; st->ls_trials = trials; }
  }
  if (lead) {   // this thread wrote the line search's fields itself
    write_stats_row(st, stats, it);
    st->gn_iter = it + 1;
  }
  if (st->stop) return;
  if (gamma != 0.0) update_nodes<true, 8>(g, b, q, (float)gamma, gtid, T);   // 8 in flight
  if (!eval_next || st->coef_fresh) return;   // the same in every block
  // the next step's evaluation at the new b (read at other blocks' nodes: after a barrier)
  {
    float v[1] = {0.f};
    double t1[1];
    if (!group_sum_d<1>(v, t1, sync, gen, shf, shd)) {
      if (threadIdx.x == 0) { st->status = -6; st->stop = 1; }
      return;
    }
  }
  EvalAcc acc;
  const int warps = blockDim.x >> 5, items = g.ntile * g.nseg;
  for (int w = blockIdx.x * warps + (threadIdx.x >> 5); w < items; w += gridDim.x * warps)
    eval_item<TI, false, false, kEvalU, 2, false>(g, Ip, Im, b, nullptr, nullptr, nullptr,
                                                   grad_p, dco, eco, invd, 0.f, w,
                                                   threadIdx.x & 31, acc);
  float v[4] = {acc.D, acc.S, acc.P, acc.G};
  double tot[4];
  if (!group_sum_d<4>(v, tot, sync, gen, shf, shd)) {
    if (threadIdx.x == 0) { st->status = -6; st->stop = 1; }
    return;
  }
  if (lead) {   // as the evaluation's own finisher for GN iteration it + 1
    const double hv = 0.5 * (double)g.vol;
    const double D = hv * tot[0], S = hv * tot[1], P = hv * tot[2];
    const double J = D + g.alpha_d * S + g.beta_d * P;
    st->J = J; st->D = D; st->S = S; st->P = P;
    st->gnorm = sqrt(tot[3]);
    st->status = isnan(J) ? -4 : (isinf(J) ? 1 : 0);
    st->ls_done = 0; st->ls_trials = 0; st->gamma = 0.0; st->gq = 0.0;
    st->pcg_done = 0; st->pcg_iter = 0; st->relres = 0.0;
    st->coef_fresh = 0;
    if (!isfinite(J)) { st->stop = 1; st->stop_iter = it + 1; }
  }
}

// corrected images T+ = I+(t+)(1 + delta), T- = I-(t-)(1 - delta); MEAN: their average
// 1/2 (T+ + T-) into Tp
template <typename TI, bool MEAN>
__global__ void __launch_bounds__(kBlock)
k_correct(Geo g, const TI* __restrict__ Ip, const TI* __restrict__ Im, const float* __restrict__ b,
          float* __restrict__ Tp, float* __restrict__ Tm) {
  const int seg = kSeg;
  int c = blockIdx.x * blockDim.x + threadIdx.x;
  int j0 = blockIdx.y * seg, j1 = min(j0 + seg, g.m);
  if (c >= g.ncols) return;
  const int inner = g.inner, m = g.m;
  int ib = col_base(c, inner, g.img_ostride), fb = col_base(c, inner, g.fld_ostride);
  float bj = j0 < j1 ? __ldg(b + fb + j0 * inner) : 0.f;
  for (int j = j0; j < j1; ++j) {
    float bn = __ldg(b + fb + (j + 1) * inner);
    float tp, tm, wp, wm, vp, sp, vm, sm;
    cell_positions(bj, bn, j, tp, tm);
    int ip = cell_index(tp, m, wp), im = cell_index(tm, m, wm);
    interp(Ip + ib, inner, m, ip, wp, vp, sp);
    interp(Im + ib, inner, m, im, wm, vm, sm);
    float delta = bn - bj;
    const float tpv = vp * (1.0f + delta), tmv = vm * (1.0f - delta);
    if (MEAN) {
      Tp[ib + j * inner] = 0.5f * (tpv + tmv);
    } else {
      Tp[ib + j * inner] = tpv;
      Tm[ib + j * inner] = tmv;
    }
    bj = bn;
  }
}

__global__ void __launch_bounds__(kBlock)
k_cells(Geo g, const float* __restrict__ b, int* __restrict__ cp, int* __restrict__ cm) {
  const int seg = kSeg;
  int c = blockIdx.x * blockDim.x + threadIdx.x;
  int j0 = blockIdx.y * seg, j1 = min(j0 + seg, g.m);
  if (c >= g.ncols) return;
  int ib = col_base(c, g.inner, g.img_ostride), fb = col_base(c, g.inner, g.fld_ostride);
  for (int j = j0; j < j1; ++j) {
    float tp, tm, wp, wm;
    cell_positions(__ldg(b + fb + j * g.inner), __ldg(b + fb + (j + 1) * g.inner),
                   j, tp, tm);
    cp[ib + j * g.inner] = cell_index(tp, g.m, wp);
    cm[ib + j * g.inner] = cell_index(tm, g.m, wm);
  }
}


// ------------------------------------------------------------------------------------------

static dim3 march_grid(const Geo& g, int nodes) {
  return dim3(ceil_div(g.ncols, kBlock), ceil_div(nodes, kSeg));
}

// grid of the grid-stride march kernels (eval, trial, halvings): per_sm blocks per SM (their
// occupancy: 4 for the evaluations at 64 registers, 2 for the 9-trial halving pass at 128), at
// most one per work item.  An early-returning launch then costs one short wave.
static dim3 resident_grid(const Geo& g, int per_sm = 4) {
  static int sms = 0;
  if (sms == 0) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
      sms = 148;
  }
  const int items = ceil_div(g.ncols, kBlock) * ceil_div(g.E, kSeg);
  return dim3(std::min(items, sms * per_sm));
}

#define HYSCO_DISPATCH(dtype, T, ...)                                                  \
  switch (dtype) {                                                                     \
    case 0: { using T = float; __VA_ARGS__; break; }                                   \
    case 1: { using T = __nv_bfloat16; __VA_ARGS__; break; }                           \
    default: { using T = __half; __VA_ARGS__; break; }                                 \
  }

void set_march(Geo& g, int device) {
  int sms = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess ||
      sms <= 0)
    sms = 148;
  g.divIn = make_fastdiv((unsigned)g.inner);
  g.divA = make_fastdiv((unsigned)g.nA);
  g.ntile = ceil_div(g.ncols, 32);
  // resident warps: the fewest blocks per SM of any objective kernel, 8 warps each
  int per_sm = 64;
  auto occ = [&](const void* f) {
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, f, kBlock, 0) == cudaSuccess && n > 0)
      per_sm = std::min(per_sm, n);
  };
  occ((const void*)k_eval<float, false, false, kEvalU, 2>);
  occ((const void*)k_eval<float, true, false, kEvalUTrial, 2>);
  occ((const void*)k_eval<__nv_bfloat16, false, false, kEvalU, 2>);
  occ((const void*)k_eval<__nv_bfloat16, true, false, kEvalUTrial, 2>);
  occ((const void*)k_eval<__half, false, false, kEvalU, 2>);
  occ((const void*)k_eval<__half, true, false, kEvalUTrial, 2>);
  if (per_sm == 64) per_sm = kEvalMinBlocks;
  set_march_warps(g, sms * per_sm * (kBlock / 32));
}

void set_march_warps(Geo& g, int warps) {
  g.divIn = make_fastdiv((unsigned)g.inner);
  g.divA = make_fastdiv((unsigned)g.nA);
  g.ntile = ceil_div(g.ncols, 32);
  const int most = ceil_div(g.E, kMinMarch);     // segments of at least kMinMarch nodes
  int nseg = std::max(1, std::min(warps / g.ntile, most));
  g.mseg = ceil_div(g.E, nseg);
  g.nseg = ceil_div(g.E, g.mseg);
}

int eval_blocks(const Geo& g) { return ceil_div(g.ntile * g.nseg, kBlock / 32); }

#define HYSCO_EVAL_LAUNCH(TRIAL, PROX, U, OUT)                                                  \
  HYSCO_DISPATCH(dtype, T,                                                                      \
    (k_eval<T, TRIAL, PROX, U, OUT><<<eval_blocks(g), kBlock, 0, s>>>(                          \
        g, (const T*)Ip, (const T*)Im, b, q, cpx, grad, grad_p, dco, eco, invd, it, ls_max, c1,  \
        w.partials, w.counter, w.st, terms)))

cudaError_t launch_eval(const Geo& g, int dtype, const void* Ip, const void* Im, const float* b,
                        float* grad, float* grad_p, float* dco, float* eco, float* invd, int it,
                        const Work& w, cudaStream_t s, const float* cpx, double* terms) {
  const float* q = nullptr;
  const int ls_max = 0;
  const double c1 = 0.0;
  if (cpx) {
    HYSCO_EVAL_LAUNCH(false, true, kEvalUProx, 2)
  } else if (grad && !grad_p) {
    HYSCO_EVAL_LAUNCH(false, false, kEvalU, 1)
  } else if (!grad && grad_p) {
    HYSCO_EVAL_LAUNCH(false, false, kEvalU, 2)
  } else if (!grad && !grad_p) {
    HYSCO_EVAL_LAUNCH(false, false, kEvalU, 0)
  } else {
    HYSCO_EVAL_LAUNCH(false, false, kEvalU, 3)
  }
  return cudaGetLastError();
}

cudaError_t launch_eval_trial(const Geo& g, int dtype, const void* Ip, const void* Im,
                              const float* b, const float* q, float* grad_p, float* dco,
                              float* eco, float* invd, int ls_max, double c1, const Work& w,
                              cudaStream_t s, const float* cpx) {
  float* grad = nullptr;
  double* terms = nullptr;
  const int it = 0;
  if (cpx) {
    HYSCO_EVAL_LAUNCH(true, true, kEvalUProx, 2)
  } else {
    HYSCO_EVAL_LAUNCH(true, false, kEvalUTrial, 2)
  }
  return cudaGetLastError();
}

template <bool PROX>
static void linesearch_impl(const Geo& g, int dtype, const void* Ip, const void* Im,
                            const float* b, const float* q, const float* cpx, const float* grad,
                            int t0, int ls_max, double c1, const Work& w, cudaStream_t s) {
  if (t0 == 0) {
    HYSCO_DISPATCH(dtype, T,
      (k_linesearch<T, kSeg, 1, PROX><<<resident_grid(g), kBlock, 0, s>>>(
          g, (const T*)Ip, (const T*)Im, b, q, cpx, grad, t0, ls_max, c1, w.partials,
          w.counter, w.st)))
  } else {
    HYSCO_DISPATCH(dtype, T,
      (k_linesearch<T, kSeg, kLsBatch, PROX><<<resident_grid(g, 2), kBlock, 0, s>>>(
          g, (const T*)Ip, (const T*)Im, b, q, cpx, grad, t0, ls_max, c1, w.partials,
          w.counter, w.st)))
  }
}

cudaError_t launch_linesearch(const Geo& g, int dtype, const void* Ip, const void* Im,
                              const float* b, const float* q, const float* grad, int t0,
                              int ls_max, double c1, const Work& w, cudaStream_t s,
                              const float* cpx) {
  if (cpx) linesearch_impl<true>(g, dtype, Ip, Im, b, q, cpx, grad, t0, ls_max, c1, w, s);
  else linesearch_impl<false>(g, dtype, Ip, Im, b, q, nullptr, grad, t0, ls_max, c1, w, s);
  return cudaGetLastError();
}

cudaError_t launch_update(const Geo& g, float* b, const float* q, int it, double* stats,
                          const Work& w, cudaStream_t s) {
  int blocks = ceil_div(g.nf, 4 * kBlock);
  if (blocks > 148 * 8) blocks = 148 * 8;
  k_update<<<blocks, kBlock, 0, s>>>(g, b, q, it, stats, w.st);
  return cudaGetLastError();
}

int ls_update_grid(int device, int dtype) {
  int sms = 0, coop = 0, per_sm = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess ||
      cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, device) != cudaSuccess || !coop)
    return 0;
  const void* fn = dtype == 0 ? (const void*)k_ls_update<float>
                              : (dtype == 1 ? (const void*)k_ls_update<__nv_bfloat16>
                                            : (const void*)k_ls_update<__half>);
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kPcgBlock, 0) != cudaSuccess ||
      per_sm < 1) {
    cudaGetLastError();
    return 0;
  }
  return sms;   // one block per SM
}

cudaError_t launch_ls_update(const Geo& g, int dtype, int grid, const void* Ip, const void* Im,
                             float* b, const float* q, int it, int ls_max, double c1,
                             double* stats, unsigned* sync, DevState* st, cudaStream_t s,
                             int eval_next, float* grad_p, float* dco, float* eco,
                             float* invd, unsigned* clear, int nclear) {
  Geo gg = g;
  float* bb = b;
  const float* qq = q;
  void* args[] = {&gg,        (void*)&Ip, (void*)&Im, &bb,  &qq,  &it,  &ls_max, &c1,
                  &stats,     &sync,      &st,        &eval_next, &grad_p, &dco, &eco, &invd,
                  &clear,     &nclear};
  const void* fn = dtype == 0 ? (const void*)k_ls_update<float>
                              : (dtype == 1 ? (const void*)k_ls_update<__nv_bfloat16>
                                            : (const void*)k_ls_update<__half>);
  return cudaLaunchCooperativeKernel(fn, dim3(grid), dim3(kPcgBlock), args, 0, s);
}

cudaError_t launch_correct(const Geo& g, int dtype, const void* Ip, const void* Im,
                           const float* b, float* Tp, float* Tm, cudaStream_t s) {
  if (Tm) {
    HYSCO_DISPATCH(dtype, T,
      (k_correct<T, false><<<march_grid(g, g.m), kBlock, 0, s>>>(g, (const T*)Ip, (const T*)Im, b,
                                                                  Tp, Tm)))
  } else {
    HYSCO_DISPATCH(dtype, T,
      (k_correct<T, true><<<march_grid(g, g.m), kBlock, 0, s>>>(g, (const T*)Ip, (const T*)Im, b,
                                                                 Tp, nullptr)))
  }
  return cudaGetLastError();
}

cudaError_t launch_cells(const Geo& g, const float* b, int* cp, int* cm, cudaStream_t s) {
  k_cells<<<march_grid(g, g.m), kBlock, 0, s>>>(g, b, cp, cm);
  return cudaGetLastError();
}


}  // namespace hysco
