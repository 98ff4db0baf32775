// The whole Jacobi-preconditioned CG of one Gauss-Newton step (Sec. 2.3.1) in one persistent,
// cooperatively launched kernel.
//
// At 3T size every PCG kernel is short (tens of microseconds) and a kernel boundary costs about
// as much as a third of the work, so PCG init and all iterations run in one launch whose phases
// are separated by device-wide barriers:
//   init   r = rhs (-grad in a GN step), x = 0, z = r / diag  partials r.r, r.z | barrier
//   iter   A: w = H z, p = z + beta p, Hp = w + beta Hp (p = z, Hp = w at i = 0), partial p.Hp
//                                                                                     | barrier
//          B: x += alpha p, r -= alpha Hp, z = r / diag  partials r.r, r.z  | barrier
// Each barrier is also the reduction of that phase's dot products: a block publishes its partial
// sums as 64-bit words that carry the barrier's generation next to the value, and every block
// waits until it has seen every block's words of that generation and adds them itself, in the
// same fixed order and in double-float (compensated single precision), so every block takes the
// same scalar decisions (alpha, beta, the relative-residual stop, p.Hp <= 0) without another
// round trip.  H p is kept by the recurrence H p = H z + beta H p_old (H is linear), so the
// stencil reads one array (z) and p, Hp are updated in place.  The arithmetic per node is that
// of the separate kernels in k_pcg.cu.
//
// On-chip state: a thread's groups are the same in every phase (t = gtid + s T, slot s), and x, r,
// p and Hp are only ever touched at the thread's own groups (the stencil reads z alone).  So r, p
// and Hp of the first `onchip` slots live in dynamic shared memory for the whole launch (the
// thread's own words, no block synchronisation) and only z, x and the read-only coefficients
// travel through L2/HBM; slots beyond `onchip` (volumes too large for shared memory) keep r, p,
// Hp in global memory.  At 3T size every slot is on chip: 7 instead of 15 field streams per
// iteration.
//
// Memory: arrays written inside the launch (x, r, z, p, Hp) are read with ordinary (coherent)
// loads after a barrier, never through the read-only path; d, e, 1/diag and grad are read-only.
// A block releases its phase's writes with a fence before it publishes its words; a reader
// fences after it has seen them.  Barriers spin with a bounded clock budget: on expiry a block
// records an error in the device state and returns; every other block then also times out at
// its next barrier, so the launch always ends.

#include <algorithm>

#include "pcg_run.cuh"

namespace hysco {


template <int P>
__global__ void __launch_bounds__(kPcgBlock)
k_pcg_persistent(Geo g, PcgArgs a) {
  __shared__ float shf[32 * 2];
  __shared__ df32 shd[32 * 2];
  extern __shared__ float4 slots[];   // [r | p | Hp][onchip][kPcgBlock]
  // the step's evaluation launch was not made (an accepted gamma = 1 trial left its coefficients
  // in place): the trial's stash becomes the current state (only the device state's scalars, which
  // no block of this launch reads but stop)
  if (a.promote && blockIdx.x == 0 && threadIdx.x == 0 && a.st->coef_fresh && !a.st->stop)
    promote_stash(a.st, false);
  if (a.promote) {   // the tail launch's words, for its use after this launch
    const int W = (int)pcg_sync_words(gridDim.x);
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < W; i += gridDim.x * blockDim.x)
      a.sync[W + i] = 0u;
  }
  unsigned gen = 0;
  pcg_run<P>(g, a, whole_grid(), shf, shd, slots, gen);
}

// Several problems' PCGs in one cooperative launch (a wave of a batch): problem i is worked on by
// blocks w.blk0[i] .. w.blk0[i] + w.nblk[i] - 1 with its own arguments (its on-chip slots, its
// sync words) and barriers among those blocks only, so the problems proceed independently.
__global__ void __launch_bounds__(kPcgBlock)
k_pcg_wave(const PcgWave wv) {
  __shared__ float shf[32 * 2];
  __shared__ df32 shd[32 * 2];
  extern __shared__ float4 slots[];
  int i = 0;
  while (i + 1 < wv.n && (int)blockIdx.x >= wv.blk0[i + 1]) ++i;
  if ((int)blockIdx.x >= wv.blk0[i] + wv.nblk[i]) return;   // spare blocks of the launch
  const BarrierGroup grp{(int)blockIdx.x - wv.blk0[i], wv.nblk[i]};
  const Geo& g = wv.g[i];
  unsigned gen = 0;
  if (g.p == 0) pcg_run<0>(g, wv.a[i], grp, shf, shd, slots, gen);
  else if (g.p == 1) pcg_run<1>(g, wv.a[i], grp, shf, shd, slots, gen);
  else pcg_run<2>(g, wv.a[i], grp, shf, shd, slots, gen);
}

// ==========================================================================================
// One-barrier-per-iteration form of the same Jacobi PCG (same iterates in exact arithmetic).
//
// With w = H z and the direction product q = H p kept by q = w + beta q_old, iteration k's
// updates of p, q, x, r, z need only alpha_{k-1} and beta_{k-2}, and the next H z_k needs z_k at
// the stencil neighbours, which every thread recomputes from r_{k-1}, w_{k-1}, q_{k-2} and 1/diag
// there with the owner's own operations (bit-identical values).  So one phase per iteration does
//   p_{k-1} = z_{k-1} + beta_{k-2} p_{k-2}      q_{k-1} = w_{k-1} + beta_{k-2} q_{k-2}
//   x_k = x_{k-1} + alpha_{k-1} p_{k-1}         r_k = r_{k-1} - alpha_{k-1} q_{k-1}
//   z_k = r_k / diag                            w_k = H z_k
// and one fused barrier + reduction yields r.z, r.r and the pieces of the next denominator,
//   p_k.q_k = z_k.w_k + beta_{k-1} (z_k.q_{k-1} + p_{k-1}.w_k) + beta_{k-1}^2 p_{k-1}.q_{k-1},
// the bilinear expansion of p_k.H p_k.  Vectors read at neighbours while their owners write the
// next iterate (r, w, q) alternate between two buffers; p and x are updated in place.  Phase 0
// forms r_0 = rhs, z_0, w_0 = H z_0; the last phase (k = max_it) skips the stencil.
// ==========================================================================================

struct FusedArgs {
  const float* grad;   // right-hand side is rhs_sign * grad
  float rhs_sign;
  float* x;
  float* p;
  float* rb[2];
  float* wb[2];
  float* qb[2];
  const float* dco;
  const float* eco;
  const float* invd;
  unsigned* sync;
  DevState* st;
  int max_it;
  double rtol;
};

// w = H z at the four nodes of group t from z at the group, its axis-0/axis-1 neighbour groups and
// the innermost-axis neighbours zl (node 4t - 1) and zr (node 4t + 4); padding nodes give 0.
template <int P>
__device__ __forceinline__ void hz_group(const Geo& g, const GroupPos& q, int t, float4 zc,
                                         float4 z1m, float4 z1p, float4 z0m, float4 z0p, float zl,
                                         float zr, const float* __restrict__ dco,
                                         const float* __restrict__ eco, float (&w)[4]) {
  const int n = 4 * t, fe2 = g.fe[2];
  const int s1 = g.G4, s0 = g.fe[1] * g.G4;
  const float4 d4 = __ldg(reinterpret_cast<const float4*>(dco) + t);
  const float4 e4 = __ldg(reinterpret_cast<const float4*>(eco) + t);
  float4 em4 = make_float4(0.f, 0.f, 0.f, 0.f);
  float el = 0.f;
  if (P == 0 && q.i0 > 0) em4 = __ldg(reinterpret_cast<const float4*>(eco) + t - s0);
  if (P == 1 && q.i1 > 0) em4 = __ldg(reinterpret_cast<const float4*>(eco) + t - s1);
  if (P == 2 && q.x0 > 0) el = __ldg(eco + n - 1);
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const int x = q.x0 + u;
    const float zk = f4get(zc, u);
    const float a2m = x > 0 ? (u == 0 ? zl : f4get(zc, u - 1)) : zk;
    const float a2p = x < fe2 - 1 ? (u == 3 ? zr : f4get(zc, u + 1)) : zk;
    const float a1m = f4get(z1m, u), a1p = f4get(z1p, u);
    const float a0m = f4get(z0m, u), a0p = f4get(z0p, u);
    const float lap = g.w[0] * ((zk - a0m) + (zk - a0p)) + g.w[1] * ((zk - a1m) + (zk - a1p)) +
                      g.w[2] * ((zk - a2m) + (zk - a2p));
    float elo = P == 2 ? (u == 0 ? el : f4get(e4, u - 1)) : f4get(em4, u);
    if (P == 2 && x == 0) elo = 0.f;
    const float zlo = P == 0 ? a0m : (P == 1 ? a1m : a2m);
    const float zhi = P == 0 ? a0p : (P == 1 ? a1p : a2p);
    const float v = g.vol * (elo * zlo + f4get(d4, u) * zk + f4get(e4, u) * zhi + g.alpha * lap);
    w[u] = x < fe2 ? v : 0.f;
  }
}

// z_k at one node from the previous iterate (the owner's arithmetic, in this order)
__device__ __forceinline__ float z_next(float r, float w, float q, float id, float al, float be) {
  return id * fmaf(-al, fmaf(be, q, w), r);
}
__device__ __forceinline__ float4 z_next4(const float* r, const float* w, const float* q,
                                          const float* __restrict__ invd, int s, float al,
                                          float be, bool has_q) {
  const float4 rv = reinterpret_cast<const float4*>(r)[s];
  const float4 wv = reinterpret_cast<const float4*>(w)[s];
  const float4 qv = has_q ? reinterpret_cast<const float4*>(q)[s] : make_float4(0.f, 0.f, 0.f, 0.f);
  const float4 iv = __ldg(reinterpret_cast<const float4*>(invd) + s);
  return make_float4(z_next(rv.x, wv.x, qv.x, iv.x, al, be), z_next(rv.y, wv.y, qv.y, iv.y, al, be),
                     z_next(rv.z, wv.z, qv.z, iv.z, al, be), z_next(rv.w, wv.w, qv.w, iv.w, al, be));
}
__device__ __forceinline__ float4 z_init4(const float* __restrict__ grad,
                                          const float* __restrict__ invd, int s, float sign) {
  const float4 gv = __ldg(reinterpret_cast<const float4*>(grad) + s);
  const float4 iv = __ldg(reinterpret_cast<const float4*>(invd) + s);
  return make_float4(iv.x * (sign * gv.x), iv.y * (sign * gv.y), iv.z * (sign * gv.z),
                     iv.w * (sign * gv.w));
}

template <int P>
__global__ void __launch_bounds__(kBlock)
k_pcg_fused(Geo g, FusedArgs a) {
  __shared__ float shf[32 * 6];
  __shared__ df32 shd[32 * 6];
  DevState* st = a.st;
  if (st->stop) return;
  const int T = gridDim.x * blockDim.x;
  const int lane = threadIdx.x & 31;
  const int wbase = blockIdx.x * blockDim.x + (threadIdx.x & ~31);   // first group of this warp
  const int n4 = g.nfp >> 2;
  const int s1 = g.G4, s0 = g.fe[1] * g.G4, fe2 = g.fe[2];
  const unsigned full = 0xffffffffu;
  unsigned gen = 0;
  auto timed_out = [&]() { if (threadIdx.x == 0) { st->status = -6; st->stop = 1; } };
  const float sign = a.rhs_sign;

  // ---- phase 0: r_0 = rhs, z_0 = r_0 / diag, w_0 = H z_0 ------------------------------------
  float t0[3] = {0.f, 0.f, 0.f};   // r.z, r.r, z.w
  for (int base = wbase; base < n4; base += T) {
    const int t = min(base + lane, n4 - 1);
    const bool own = base + lane < n4;
    const GroupPos q = group_pos(g, t);
    const int n = 4 * t;
    const float4 gc = __ldg(reinterpret_cast<const float4*>(a.grad) + t);
    const float4 ic = __ldg(reinterpret_cast<const float4*>(a.invd) + t);
    const float rc[4] = {sign * gc.x, sign * gc.y, sign * gc.z, sign * gc.w};
    const float4 zc = make_float4(ic.x * rc[0], ic.y * rc[1], ic.z * rc[2], ic.w * rc[3]);
    const float4 z1m = q.i1 > 0 ? z_init4(a.grad, a.invd, t - s1, sign) : zc;
    const float4 z1p = q.i1 < g.fe[1] - 1 ? z_init4(a.grad, a.invd, t + s1, sign) : zc;
    const float4 z0m = q.i0 > 0 ? z_init4(a.grad, a.invd, t - s0, sign) : zc;
    const float4 z0p = q.i0 < g.fe[0] - 1 ? z_init4(a.grad, a.invd, t + s0, sign) : zc;
    float zl = __shfl_up_sync(full, zc.w, 1), zr = __shfl_down_sync(full, zc.x, 1);
    if (lane == 0 && q.x0 > 0) zl = __ldg(a.invd + n - 1) * (sign * __ldg(a.grad + n - 1));
    if (lane == 31 && q.x0 + 4 < g.P2) zr = __ldg(a.invd + n + 4) * (sign * __ldg(a.grad + n + 4));
    float w[4];
    hz_group<P>(g, q, t, zc, z1m, z1p, z0m, z0p, zl, zr, a.dco, a.eco, w);
    if (own) {
      float ro[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const bool real = q.x0 + u < fe2;
        ro[u] = real ? rc[u] : 0.f;
        const float zk = real ? f4get(zc, u) : 0.f;
        t0[0] += ro[u] * zk;
        t0[1] += ro[u] * ro[u];
        t0[2] += zk * w[u];
      }
      reinterpret_cast<float4*>(a.rb[0])[t] = make_float4(ro[0], ro[1], ro[2], ro[3]);
      reinterpret_cast<float4*>(a.wb[0])[t] = make_float4(w[0], w[1], w[2], w[3]);
    }
  }
  if (!grid_allreduce<3>(t0, a.sync, ++gen, shf, shd)) { timed_out(); return; }
  const float rr0 = t0[1];
  float rho = t0[0], pq = t0[2];   // p_0 = z_0, q_0 = w_0
  float al = 0.f, be = 0.f, beta = 0.f, relres = rr0 > 0.f ? 1.f : 0.f;
  bool done = !(rr0 > 0.f) || !(pq > 0.f) || a.max_it < 1;
  if (!done) al = rho / pq;
  int it = 0;

  for (int k = 1; !done; ++k) {
    const bool last = k == a.max_it, has_q = k > 1;
    const float* rold = a.rb[(k - 1) & 1];
    const float* wold = a.wb[(k - 1) & 1];
    const float* qold = a.qb[k & 1];
    float* rnew = a.rb[k & 1];
    float* wnew = a.wb[k & 1];
    float* qnew = a.qb[(k - 1) & 1];
    float v[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};   // r.z, r.r, z.w, z.q_old, p_old.w, p_old.q_old
    for (int base = wbase; base < n4; base += T) {
      const int t = min(base + lane, n4 - 1);
      const bool own = base + lane < n4;
      const GroupPos q = group_pos(g, t);
      const int n = 4 * t;
      const float4 r4 = reinterpret_cast<const float4*>(rold)[t];
      const float4 w4 = reinterpret_cast<const float4*>(wold)[t];
      const float4 q4 = has_q ? reinterpret_cast<const float4*>(qold)[t] : make_float4(0.f, 0.f, 0.f, 0.f);
      const float4 p4 = has_q ? reinterpret_cast<const float4*>(a.p)[t] : make_float4(0.f, 0.f, 0.f, 0.f);
      const float4 x4 = has_q ? reinterpret_cast<const float4*>(a.x)[t] : make_float4(0.f, 0.f, 0.f, 0.f);
      const float4 i4 = __ldg(reinterpret_cast<const float4*>(a.invd) + t);
      float pn[4], qn[4], xn[4], rn[4], zn[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const float ri = f4get(r4, u), ii = f4get(i4, u);
        qn[u] = fmaf(be, f4get(q4, u), f4get(w4, u));
        rn[u] = fmaf(-al, qn[u], ri);
        zn[u] = ii * rn[u];
        pn[u] = fmaf(be, f4get(p4, u), ii * ri);
        xn[u] = fmaf(al, pn[u], f4get(x4, u));
      }
      float w[4] = {0.f, 0.f, 0.f, 0.f};
      if (!last) {
        const float4 zc = make_float4(zn[0], zn[1], zn[2], zn[3]);
        const float4 z1m = q.i1 > 0 ? z_next4(rold, wold, qold, a.invd, t - s1, al, be, has_q) : zc;
        const float4 z1p = q.i1 < g.fe[1] - 1 ? z_next4(rold, wold, qold, a.invd, t + s1, al, be, has_q) : zc;
        const float4 z0m = q.i0 > 0 ? z_next4(rold, wold, qold, a.invd, t - s0, al, be, has_q) : zc;
        const float4 z0p = q.i0 < g.fe[0] - 1 ? z_next4(rold, wold, qold, a.invd, t + s0, al, be, has_q) : zc;
        float zl = __shfl_up_sync(full, zc.w, 1), zr = __shfl_down_sync(full, zc.x, 1);
        if (lane == 0 && q.x0 > 0)
          zl = z_next(rold[n - 1], wold[n - 1], has_q ? qold[n - 1] : 0.f, __ldg(a.invd + n - 1), al, be);
        if (lane == 31 && q.x0 + 4 < g.P2)
          zr = z_next(rold[n + 4], wold[n + 4], has_q ? qold[n + 4] : 0.f, __ldg(a.invd + n + 4), al, be);
        hz_group<P>(g, q, t, zc, z1m, z1p, z0m, z0p, zl, zr, a.dco, a.eco, w);
      }
      if (own) {
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          if (q.x0 + u >= fe2) { pn[u] = qn[u] = xn[u] = rn[u] = zn[u] = 0.f; }
          v[0] += rn[u] * zn[u];
          v[1] += rn[u] * rn[u];
          v[2] += zn[u] * w[u];
          v[3] += zn[u] * qn[u];
          v[4] += pn[u] * w[u];
          v[5] += pn[u] * qn[u];
        }
        reinterpret_cast<float4*>(a.x)[t] = make_float4(xn[0], xn[1], xn[2], xn[3]);
        reinterpret_cast<float4*>(a.p)[t] = make_float4(pn[0], pn[1], pn[2], pn[3]);
        reinterpret_cast<float4*>(qnew)[t] = make_float4(qn[0], qn[1], qn[2], qn[3]);
        reinterpret_cast<float4*>(rnew)[t] = make_float4(rn[0], rn[1], rn[2], rn[3]);
        if (!last) reinterpret_cast<float4*>(wnew)[t] = make_float4(w[0], w[1], w[2], w[3]);
      }
    }
    if (!grid_allreduce<6>(v, a.sync, ++gen, shf, shd)) { timed_out(); return; }
    it = k;
    relres = sqrtf(v[1]) / sqrtf(rr0);
    if (relres < (float)a.rtol || last) break;
    beta = v[0] / rho;
    rho = v[0];
    const float den = v[2] + beta * (v[3] + v[4]) + beta * beta * v[5];
    if (!(den > 0.f)) break;
    be = beta;
    al = rho / den;
  }
  if (it == 0) {   // no iteration ran: x = 0
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < n4; t += T)
      reinterpret_cast<float4*>(a.x)[t] = make_float4(0.f, 0.f, 0.f, 0.f);
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    st->rr0 = rr0;
    st->rho = rho;
    st->beta_cg = beta;
    st->pcg_iter = it;
    st->relres = relres;
    st->pcg_done = 1;
  }
}

template <int P>
static PcgPlan plan_for(int device, int n4) {
  PcgPlan pl{0, 0};
  int sms = 0, per_sm = 0, coop = 0, optin = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess)
    return pl;
  if (cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, device) != cudaSuccess || !coop)
    return pl;
  if (cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, device) !=
      cudaSuccess)
    optin = 48 * 1024;
  // blocks per SM as the registers allow (at most kPcgBlocksPerSm: the barriers' latency grows
  // with the number of blocks), then as many on-chip slots as keep that occupancy
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_pcg_persistent<P>, kPcgBlock, 0) !=
          cudaSuccess || per_sm < 1)
    return pl;
  per_sm = std::min(per_sm, kPcgBlocksPerSm);
  const int grid = std::min(sms * per_sm, 32 * kTagWordsPerLane);
  const long long T = (long long)grid * kPcgBlock;
  // the launch limit is the device's opt-in maximum less the static shared memory (the same for
  // every handle); the occupancy test below takes each candidate size explicitly
  int G = 0;
  cudaFuncAttributes fa;
  const int dyn_max = cudaFuncGetAttributes(&fa, k_pcg_persistent<P>) == cudaSuccess
                          ? optin - (int)fa.sharedSizeBytes
                          : 0;
  if (dyn_max > 0 && cudaFuncSetAttribute(k_pcg_persistent<P>,
                                          cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          dyn_max) == cudaSuccess) {
    G = (int)std::min<long long>((n4 + T - 1) / T, dyn_max / pcg_onchip_bytes(1));
    for (; G > 0; --G) {
      int got = 0;
      if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&got, k_pcg_persistent<P>, kPcgBlock,
                                                        pcg_onchip_bytes(G)) == cudaSuccess &&
          got * sms >= grid)
        break;
    }
  }
  cudaGetLastError();
  pl.grid = grid;
  pl.onchip = G;
  return pl;
}

template <int P>
static int fused_grid_for(int device) {
  int sms = 0, per_sm = 0, coop = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) return 0;
  if (cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, device) != cudaSuccess || !coop)
    return 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_pcg_fused<P>, kBlock, 0) !=
      cudaSuccess)
    return 0;
  return sms * per_sm;
}

int pcg_fused_grid(int device, int pe_axis) {
  return pe_axis == 0 ? fused_grid_for<0>(device) : (pe_axis == 1 ? fused_grid_for<1>(device)
                                                                  : fused_grid_for<2>(device));
}

cudaError_t launch_pcg_fused(const Geo& g, int grid, const float* grad, float rhs_sign, float* x,
                             float* p, float* const rb[2], float* const wb[2], float* const qb[2],
                             const float* dco, const float* eco, const float* invd,
                             unsigned* sync, int max_it, double rtol, DevState* st,
                             cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(sync, 0, pcg_sync_words(grid) * sizeof(unsigned), s);
  if (e != cudaSuccess) return e;
  FusedArgs a{grad, rhs_sign, x, p, {rb[0], rb[1]}, {wb[0], wb[1]}, {qb[0], qb[1]},
              dco, eco, invd, sync, st, max_it, rtol};
  Geo gg = g;
  void* args[] = {&gg, &a};
  void* fn = g.p == 0 ? (void*)k_pcg_fused<0>
                      : (g.p == 1 ? (void*)k_pcg_fused<1> : (void*)k_pcg_fused<2>);
  return cudaLaunchCooperativeKernel(fn, dim3(grid), dim3(kBlock), args, 0, s);
}

int pcg_wave_setup(int device) {
  int sms = 0, coop = 0, optin = 0, per_sm = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess ||
      cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, device) != cudaSuccess ||
      !coop ||
      cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, device) !=
          cudaSuccess)
    return 0;
  cudaFuncAttributes fa;
  if (cudaFuncGetAttributes(&fa, k_pcg_wave) != cudaSuccess ||
      cudaFuncSetAttribute(k_pcg_wave, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           optin - (int)fa.sharedSizeBytes) != cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_pcg_wave, kPcgBlock,
                                                    pcg_onchip_bytes(kWaveSlots)) != cudaSuccess ||
      per_sm < 1) {
    cudaGetLastError();
    return 0;
  }
  return std::min(sms, 32 * kTagWordsPerLane);   // one block per SM
}

cudaError_t launch_pcg_wave(const PcgWave& w, int grid, int onchip_max, unsigned* sync,
                            size_t sync_words, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(sync, 0, sync_words * sizeof(unsigned), s);
  if (e != cudaSuccess) return e;
  PcgWave copy = w;
  void* args[] = {&copy};
  return cudaLaunchCooperativeKernel((void*)k_pcg_wave, dim3(grid), dim3(kPcgBlock), args,
                                     pcg_onchip_bytes(onchip_max), s);
}

PcgPlan pcg_persistent_plan(int device, int pe_axis, int n4) {
  return pe_axis == 0 ? plan_for<0>(device, n4)
                      : (pe_axis == 1 ? plan_for<1>(device, n4) : plan_for<2>(device, n4));
}

cudaError_t launch_pcg_persistent(const Geo& g, const PcgPlan& pl, const float* grad,
                                  float rhs_sign, float* x, float* r, float* z, float* p0,
                                  float* p1, float* Hp, const float* dco, const float* eco,
                                  const float* invd, unsigned* sync, int max_it, double rtol,
                                  DevState* st, cudaStream_t s, int promote, int clear) {
  // the words of this launch and, after them, as many for the step's halvings-and-update launch
  if (clear) {
    cudaError_t e = cudaMemsetAsync(sync, 0, 2 * pcg_sync_words(pl.grid) * sizeof(unsigned), s);
    if (e != cudaSuccess) return e;
  }
  PcgArgs a{grad, rhs_sign, x, r, z, p0, p1, Hp, dco, eco, invd, sync, st, max_it, rtol,
            pl.onchip, promote};
  Geo gg = g;
  void* args[] = {&gg, &a};
  void* fn = g.p == 0 ? (void*)k_pcg_persistent<0>
                      : (g.p == 1 ? (void*)k_pcg_persistent<1> : (void*)k_pcg_persistent<2>);
  return cudaLaunchCooperativeKernel(fn, dim3(pl.grid), dim3(kPcgBlock), args,
                                     pcg_onchip_bytes(pl.onchip), s);
}

}  // namespace hysco
