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
// After each barrier every block adds all blocks' partials itself, in the same fixed order and in
// double-float (compensated single precision), so every block takes the same scalar decisions
// (alpha, beta, the relative-residual stop, p.Hp <= 0) without another round trip.  H p is kept by the recurrence
// H p = H z + beta H p_old (H is linear), so the stencil reads one array (z) and p, Hp are
// updated in place.  The arithmetic per node is that of the separate kernels in k_pcg.cu.
//
// Memory: arrays written inside the launch (x, r, z, p, Hp) are read with ordinary (coherent)
// loads after a barrier, never through the read-only path; d, e, 1/diag and grad are read-only.
// Barriers spin with a bounded clock budget: on expiry a block records an error in the device
// state and returns; every other block then also times out at its next barrier, so the launch
// always ends.
#include <cuda/atomic>

#include "hysco_internal.cuh"

namespace hysco {

constexpr long long kBarrierSpinCycles = 4000000000LL;   // ~2 s at 2 GHz
constexpr int kPcgUnroll = 4;

struct PcgArgs {
  const float* grad;     // right-hand side is rhs_sign * grad
  float rhs_sign;
  float* x;
  float* r;
  float* z;
  float* p0;
  float* p1;
  float* Hp;
  const float* dco;
  const float* eco;
  const float* invd;
  float* part;           // 2 slots x gridDim.x x 2 floats
  unsigned* bar;         // [0] arrival count, [1] generation; zeroed before every launch
  DevState* st;
  int max_it;
  double rtol;
};

// Device-wide barrier.  Returns false (in every thread of the block) when the spin budget ran
// out; the block must then stop.
__device__ __forceinline__ bool grid_barrier(unsigned* bar, unsigned& gen) {
  __shared__ int ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    ok = 1;
    cuda::atomic_ref<unsigned, cuda::thread_scope_device> count(bar[0]), g(bar[1]);
    unsigned arrived = count.fetch_add(1u, cuda::memory_order_acq_rel);
    if (arrived == gridDim.x - 1) {
      count.store(0u, cuda::memory_order_relaxed);
      g.store(gen + 1, cuda::memory_order_release);
    } else {
      long long t0 = clock64();
      while (g.load(cuda::memory_order_acquire) == gen) {
        if (clock64() - t0 > kBarrierSpinCycles) { ok = 0; break; }
      }
    }
  }
  __syncthreads();
  gen += 1;
  return ok != 0;
}

// block sum of K floats, result broadcast through shared memory to every thread
template <int K>
__device__ __forceinline__ void block_reduce_f(float (&v)[K], float* sh) {
  block_sum<K, float>(v, sh);
  __syncthreads();
  if (threadIdx.x == 0)
#pragma unroll
    for (int i = 0; i < K; ++i) sh[i] = v[i];
  __syncthreads();
#pragma unroll
  for (int i = 0; i < K; ++i) v[i] = sh[i];
  __syncthreads();
}

// every block: sum of the K-float partials of all blocks in a fixed order (double-float), so
// that every block obtains the same totals
template <int K>
__device__ __forceinline__ void all_partials(const float* part, float (&tot)[K], df32* sh) {
  df32 acc[K];
#pragma unroll
  for (int i = 0; i < K; ++i) acc[i] = df32{0.f, 0.f};
  for (int b = linear_tid(); b < (int)gridDim.x; b += block_threads())
#pragma unroll
    for (int i = 0; i < K; ++i) acc[i] = df_add(acc[i], df32{part[b * K + i], 0.f});
  block_sum_df<K>(acc, sh);
  __syncthreads();
  if (linear_tid() == 0)
#pragma unroll
    for (int i = 0; i < K; ++i) sh[i] = acc[i];
  __syncthreads();
#pragma unroll
  for (int i = 0; i < K; ++i) tot[i] = sh[i].hi + sh[i].lo;
  __syncthreads();
}

template <int P>
__global__ void __launch_bounds__(kBlock)
k_pcg_persistent(Geo g, PcgArgs a) {
  __shared__ float shf[32 * 2];
  __shared__ df32 shd[32 * 2];
  DevState* st = a.st;
  if (st->stop) return;
  const int T = gridDim.x * blockDim.x;
  const int gtid = blockIdx.x * blockDim.x + threadIdx.x;
  const int n4 = g.nfp >> 2;   // float4 groups of the pitched field (padding is zero)
  unsigned gen = 0;
  int slot = 0;
  auto part = [&](int s) { return a.part + s * gridDim.x * 2; };

  // ---- init --------------------------------------------------------------------------------
  {
    float arr = 0.f, arz = 0.f;
    for (int i0 = gtid; i0 < n4; i0 += kPcgUnroll * T) {
      float4 gv[kPcgUnroll], dv[kPcgUnroll];
#pragma unroll
      for (int u = 0; u < kPcgUnroll; ++u) {
        int i = min(i0 + u * T, n4 - 1);
        gv[u] = __ldg(reinterpret_cast<const float4*>(a.grad) + i);
        dv[u] = __ldg(reinterpret_cast<const float4*>(a.invd) + i);
      }
#pragma unroll
      for (int u = 0; u < kPcgUnroll; ++u) {
        int i = i0 + u * T;
        float4 rv = make_float4(a.rhs_sign * gv[u].x, a.rhs_sign * gv[u].y, a.rhs_sign * gv[u].z,
                                a.rhs_sign * gv[u].w);
        float4 zv = make_float4(rv.x * dv[u].x, rv.y * dv[u].y, rv.z * dv[u].z, rv.w * dv[u].w);
        if (i < n4) {
          reinterpret_cast<float4*>(a.x)[i] = make_float4(0.f, 0.f, 0.f, 0.f);
          reinterpret_cast<float4*>(a.r)[i] = rv;
          reinterpret_cast<float4*>(a.z)[i] = zv;
          arr += rv.x * rv.x + rv.y * rv.y + rv.z * rv.z + rv.w * rv.w;
          arz += rv.x * zv.x + rv.y * zv.y + rv.z * zv.z + rv.w * zv.w;
        }
      }
    }
    float v[2] = {arr, arz};
    block_reduce_f<2>(v, shf);
    if (threadIdx.x == 0) { part(slot)[blockIdx.x * 2] = v[0]; part(slot)[blockIdx.x * 2 + 1] = v[1]; }
  }
  if (!grid_barrier(a.bar, gen)) { if (threadIdx.x == 0) { st->status = -6; st->stop = 1; } return; }
  // scalars in single precision (the sums themselves are double-float accurate)
  float tot[2];
  all_partials<2>(part(slot), tot, shd);
  slot ^= 1;
  const float rr0 = tot[0];
  float rho = tot[1], beta = 0.f, relres = rr0 > 0.f ? 1.f : 0.f;
  bool done = !(rr0 > 0.f);
  int it = 0;

  for (int i = 0; i < a.max_it && !done; ++i) {
    const bool first = i == 0;
    float* pv_ = a.p0;
    const float fb = beta;
    // ---- A: w = H z; p = z + beta p; Hp = w + beta Hp (groups of 4 pitched nodes) ----------
    float acc = 0.f;
    for (int t = gtid; t < n4; t += T) acc += hv_group<P, true>(g, t, a.z, pv_, a.Hp, a.dco, a.eco, fb, first);
    {
      float v[1] = {acc};
      block_reduce_f<1>(v, shf);
      if (threadIdx.x == 0) part(slot)[blockIdx.x] = v[0];
    }
    if (!grid_barrier(a.bar, gen)) { if (threadIdx.x == 0) { st->status = -6; st->stop = 1; } return; }
    {
      float t1[1];
      all_partials<1>(part(slot), t1, shd);
      slot ^= 1;
      if (!(t1[0] > 0.f)) { done = true; break; }
      const float al = rho / t1[0];
      // ---- B: x += alpha p, r -= alpha Hp, z = r / diag ----------------------------------
      float arr = 0.f, arz = 0.f;
      for (int j0 = gtid; j0 < n4; j0 += kPcgUnroll * T) {
        float4 pv[kPcgUnroll], hv[kPcgUnroll], dv[kPcgUnroll], rv[kPcgUnroll], xv[kPcgUnroll];
#pragma unroll
        for (int u = 0; u < kPcgUnroll; ++u) {
          int j = min(j0 + u * T, n4 - 1);
          pv[u] = reinterpret_cast<const float4*>(pv_)[j];
          hv[u] = reinterpret_cast<const float4*>(a.Hp)[j];
          dv[u] = __ldg(reinterpret_cast<const float4*>(a.invd) + j);
          rv[u] = reinterpret_cast<const float4*>(a.r)[j];
          xv[u] = first ? make_float4(0.f, 0.f, 0.f, 0.f) : reinterpret_cast<const float4*>(a.x)[j];
        }
#pragma unroll
        for (int u = 0; u < kPcgUnroll; ++u) {
          int j = j0 + u * T;
          float4 X = xv[u], R = rv[u];
          X.x = fmaf(al, pv[u].x, X.x); X.y = fmaf(al, pv[u].y, X.y);
          X.z = fmaf(al, pv[u].z, X.z); X.w = fmaf(al, pv[u].w, X.w);
          R.x = fmaf(-al, hv[u].x, R.x); R.y = fmaf(-al, hv[u].y, R.y);
          R.z = fmaf(-al, hv[u].z, R.z); R.w = fmaf(-al, hv[u].w, R.w);
          float4 Z = make_float4(R.x * dv[u].x, R.y * dv[u].y, R.z * dv[u].z, R.w * dv[u].w);
          if (j < n4) {
            reinterpret_cast<float4*>(a.x)[j] = X;
            reinterpret_cast<float4*>(a.r)[j] = R;
            reinterpret_cast<float4*>(a.z)[j] = Z;
            arr += R.x * R.x + R.y * R.y + R.z * R.z + R.w * R.w;
            arz += R.x * Z.x + R.y * Z.y + R.z * Z.z + R.w * Z.w;
          }
        }
      }
      float v2[2] = {arr, arz};
      block_reduce_f<2>(v2, shf);
      if (threadIdx.x == 0) { part(slot)[blockIdx.x * 2] = v2[0]; part(slot)[blockIdx.x * 2 + 1] = v2[1]; }
    }
    if (!grid_barrier(a.bar, gen)) { if (threadIdx.x == 0) { st->status = -6; st->stop = 1; } return; }
    all_partials<2>(part(slot), tot, shd);
    slot ^= 1;
    it = i + 1;
    relres = sqrtf(tot[0]) / sqrtf(rr0);
    if (relres < (float)a.rtol) {
      done = true;
    } else {
      beta = tot[1] / rho;
      rho = tot[1];
    }
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
static int grid_for(int device) {
  int sms = 0, per_sm = 0, coop = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) return 0;
  if (cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, device) != cudaSuccess || !coop)
    return 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_pcg_persistent<P>, kBlock, 0) !=
      cudaSuccess)
    return 0;
  return sms * per_sm;
}

int pcg_persistent_grid(int device, int pe_axis) {
  return pe_axis == 0 ? grid_for<0>(device) : (pe_axis == 1 ? grid_for<1>(device)
                                                            : grid_for<2>(device));
}

cudaError_t launch_pcg_persistent(const Geo& g, int grid, const float* grad, float rhs_sign,
                                  float* x, float* r, float* z, float* p0, float* p1, float* Hp,
                                  const float* dco, const float* eco, const float* invd,
                                  float* part, unsigned* bar, int max_it, double rtol,
                                  DevState* st, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(bar, 0, 2 * sizeof(unsigned), s);
  if (e != cudaSuccess) return e;
  PcgArgs a{grad, rhs_sign, x, r, z, p0, p1, Hp, dco, eco, invd, part, bar, st, max_it, rtol};
  Geo gg = g;
  void* args[] = {&gg, &a};
  void* fn = g.p == 0 ? (void*)k_pcg_persistent<0>
                      : (g.p == 1 ? (void*)k_pcg_persistent<1> : (void*)k_pcg_persistent<2>);
  return cudaLaunchCooperativeKernel(fn, dim3(grid), dim3(kBlock), args, 0, s);
}

}  // namespace hysco
