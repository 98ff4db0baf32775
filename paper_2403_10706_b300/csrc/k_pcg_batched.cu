// Jacobi PCG (Sec. 2.3.1) of one Gauss-Newton step for many volume pairs of uneven sizes in one
// persistent, cooperatively launched kernel.
//
// The grid's blocks are split into contiguous ranges, one range per pair (sizes chosen on the
// host, roughly proportional to the pair's field size).  A block works only on its own pair:
// grid-stride loops run over that pair's float4 groups with the pair's block range as the grid,
// and every phase ends in the device-wide grid_allreduce, each block adding only its own pair's
// block sums (in a fixed order, so the pair's blocks take identical decisions).  The barriers are
// shared by all pairs, so their cost is paid once per phase for the whole batch instead of once
// per pair.  The iteration is that of k_pcg_persistent (two phases per PCG iteration, H p by the
// recurrence H z + beta H p_old), per pair; a pair that has converged, stopped or was already
// stopped before the launch keeps passing the barriers without work, since every block must
// arrive at each of them.
#include "grid_sync.cuh"

namespace hysco {

namespace {

template <bool PCG>
__device__ __forceinline__ float hv_any(const Geo& g, int t, const float* z, float* p, float* Hp,
                                        const float* dco, const float* eco, float beta,
                                        bool first) {
  switch (g.p) {
    case 0: return hv_group<0, PCG>(g, t, z, p, Hp, dco, eco, beta, first);
    case 1: return hv_group<1, PCG>(g, t, z, p, Hp, dco, eco, beta, first);
    default: return hv_group<2, PCG>(g, t, z, p, Hp, dco, eco, beta, first);
  }
}

}  // namespace

__global__ void __launch_bounds__(kBlock)
k_pcg_batched(const BatchPair* __restrict__ pairs, const int* __restrict__ block_pair,
              int max_it, float rtol, unsigned* sync) {
  __shared__ float shf[32 * 2];
  __shared__ df32 shd[32 * 2];
  __shared__ BatchPair sp;
  const int pi = block_pair[blockIdx.x];
  if (threadIdx.x == 0) sp = pairs[pi];
  __syncthreads();
  const Geo& g = sp.g;
  DevState* st = sp.st;
  const int T = sp.nblk * blockDim.x;
  const int gtid = (blockIdx.x - sp.blk0) * blockDim.x + threadIdx.x;
  const int n4 = g.nfp >> 2;
  const int first = sp.blk0, count = sp.nblk;
  const bool stopped = st->stop != 0;   // the pair's solve has stopped: no work, no state update
  unsigned gen = 0;
  auto timed_out = [&]() { if (threadIdx.x == 0) { st->status = -6; st->stop = 1; } };

  // ---- init: r = -grad, x = 0, z = r / diag; r.r, r.z ---------------------------------------
  float tot[2] = {0.f, 0.f};
  if (!stopped) {
    for (int i = gtid; i < n4; i += T) {
      const float4 gv = __ldg(reinterpret_cast<const float4*>(sp.grad) + i);
      const float4 dv = __ldg(reinterpret_cast<const float4*>(sp.invd) + i);
      const float4 rv = make_float4(-gv.x, -gv.y, -gv.z, -gv.w);
      const float4 zv = make_float4(rv.x * dv.x, rv.y * dv.y, rv.z * dv.z, rv.w * dv.w);
      reinterpret_cast<float4*>(sp.x)[i] = make_float4(0.f, 0.f, 0.f, 0.f);
      reinterpret_cast<float4*>(sp.r)[i] = rv;
      reinterpret_cast<float4*>(sp.z)[i] = zv;
      tot[0] += rv.x * rv.x + rv.y * rv.y + rv.z * rv.z + rv.w * rv.w;
      tot[1] += rv.x * zv.x + rv.y * zv.y + rv.z * zv.z + rv.w * zv.w;
    }
  }
  if (!grid_allreduce<2>(tot, sync, ++gen, shf, shd, first, count)) { timed_out(); return; }
  const float rr0 = tot[0];
  float rho = tot[1], beta = 0.f, relres = rr0 > 0.f ? 1.f : 0.f;
  bool done = stopped || !(rr0 > 0.f);
  int it = 0;

  for (int i = 0; i < max_it; ++i) {
    const bool first_it = i == 0;
    // ---- A: w = H z; p = z + beta p; Hp = w + beta Hp; partial p.Hp -------------------------
    float acc[1] = {0.f};
    if (!done)
      for (int t = gtid; t < n4; t += T)
        acc[0] += hv_any<true>(g, t, sp.z, sp.p, sp.Hp, sp.dco, sp.eco, beta, first_it);
    // only p.Hp crosses blocks here (phase B reads the thread's own groups)
    if (!grid_allreduce_unordered(acc[0], sync, ++gen, shf, shd, first, count)) {
      timed_out();
      return;
    }
    float al = 0.f;
    if (!done) {
      if (!(acc[0] > 0.f)) done = true;
      else al = rho / acc[0];
    }
    // ---- B: x += alpha p, r -= alpha Hp, z = r / diag; r.r, r.z ----------------------------
    float v[2] = {0.f, 0.f};
    if (!done) {
      for (int j = gtid; j < n4; j += T) {
        const float4 pv = reinterpret_cast<const float4*>(sp.p)[j];
        const float4 hv = reinterpret_cast<const float4*>(sp.Hp)[j];
        const float4 dv = __ldg(reinterpret_cast<const float4*>(sp.invd) + j);
        float4 R = reinterpret_cast<const float4*>(sp.r)[j];
        float4 X = first_it ? make_float4(0.f, 0.f, 0.f, 0.f) : reinterpret_cast<const float4*>(sp.x)[j];
        X.x = fmaf(al, pv.x, X.x); X.y = fmaf(al, pv.y, X.y);
        X.z = fmaf(al, pv.z, X.z); X.w = fmaf(al, pv.w, X.w);
        R.x = fmaf(-al, hv.x, R.x); R.y = fmaf(-al, hv.y, R.y);
        R.z = fmaf(-al, hv.z, R.z); R.w = fmaf(-al, hv.w, R.w);
        const float4 Z = make_float4(R.x * dv.x, R.y * dv.y, R.z * dv.z, R.w * dv.w);
        reinterpret_cast<float4*>(sp.x)[j] = X;
        reinterpret_cast<float4*>(sp.r)[j] = R;
        reinterpret_cast<float4*>(sp.z)[j] = Z;
        v[0] += R.x * R.x + R.y * R.y + R.z * R.z + R.w * R.w;
        v[1] += R.x * Z.x + R.y * Z.y + R.z * Z.z + R.w * Z.w;
      }
    }
    if (!grid_allreduce<2>(v, sync, ++gen, shf, shd, first, count)) { timed_out(); return; }
    if (!done) {
      it = i + 1;
      relres = sqrtf(v[0]) / sqrtf(rr0);
      if (relres < rtol) {
        done = true;
      } else {
        beta = v[1] / rho;
        rho = v[1];
      }
    }
  }
  if (!stopped && blockIdx.x == first && threadIdx.x == 0) {
    st->rr0 = rr0;
    st->rho = rho;
    st->beta_cg = beta;
    st->pcg_iter = it;
    st->relres = relres;
    st->pcg_done = 1;
  }
}

// Self-test of the barrier's timeout path: every block but `missing` takes part in one
// grid_allreduce with a spin budget of `budget` cycles; block `missing` (if any) returns at once,
// so the others give up and raise *flag.  Bounded: the launch always ends.
__global__ void __launch_bounds__(kBlock)
k_barrier_selftest(unsigned* sync, int missing, long long budget, int* flag) {
  __shared__ float shf[32];
  __shared__ df32 shd[32];
  if ((int)blockIdx.x == missing) return;
  float v[1] = {1.f};
  if (!grid_allreduce<1>(v, sync, 1u, shf, shd, 0, -1, budget)) {
    if (threadIdx.x == 0) atomicExch(flag, 1);
    return;
  }
  if (threadIdx.x == 0 && blockIdx.x == 0 && v[0] != (float)(gridDim.x * blockDim.x))
    atomicExch(flag, 2);   // the sum over all threads is wrong
}

cudaError_t launch_barrier_selftest(int grid, int missing, long long budget, unsigned* sync,
                                    int* flag, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(sync, 0, pcg_sync_words(grid) * sizeof(unsigned), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(flag, 0, sizeof(int), s);
  if (e != cudaSuccess) return e;
  void* args[] = {&sync, &missing, &budget, &flag};
  return cudaLaunchCooperativeKernel((void*)k_barrier_selftest, dim3(grid), dim3(kBlock), args, 0,
                                     s);
}

int pcg_batched_blocks_per_sm(int device) {
  int coop = 0, per_sm = 0;
  if (cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, device) != cudaSuccess || !coop)
    return 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_pcg_batched, kBlock, 0) !=
      cudaSuccess)
    return 0;
  return per_sm;
}

cudaError_t launch_pcg_batched(int grid, const BatchPair* pairs, const int* block_pair,
                               int max_it, double rtol, unsigned* sync, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(sync, 0, pcg_sync_words(grid) * sizeof(unsigned), s);
  if (e != cudaSuccess) return e;
  float rt = (float)rtol;
  void* args[] = {&pairs, &block_pair, &max_it, &rt, &sync};
  return cudaLaunchCooperativeKernel((void*)k_pcg_batched, dim3(grid), dim3(kBlock), args, 0, s);
}

}  // namespace hysco
