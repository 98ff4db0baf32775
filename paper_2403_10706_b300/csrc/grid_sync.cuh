// Device-wide barrier fused with a deterministic reduction, for persistent cooperative kernels
// (all blocks of the grid are co-resident).  See grid_allreduce.
#pragma once

#include "hysco_internal.cuh"

namespace hysco {

constexpr long long kBarrierSpinCycles = 4000000000LL;   // ~2 s at 2 GHz
constexpr int kSumChunk = 8;   // partial-sum loads in flight per lane in grid_allreduce

__device__ __forceinline__ void red_release_add(unsigned* p, unsigned v) {
  asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ unsigned ld_acquire(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// Device-wide barrier fused with the sum of K floats over all threads of the grid.  Every thread
// of every block calls it with its own values v and the barrier's generation gen (1, 2, ... within
// a launch).  Layout of `sync`: an arrival counter (its own 128-byte line), then two slots of
// gridDim.x x kSyncMaxK floats.  Block b stores its block sums at slot gen & 1, b * K, then
// adds one to the counter with release semantics; the barrier of generation gen is complete when
// the counter
// reaches gen * gridDim.x.  A block can overwrite a slot only two generations later, by which
// time every block has read it.  Warp 0 then reads the sums of blocks first .. first + count - 1
// (default: all) through L2 and adds them in a fixed order (lane l takes blocks first + l,
// first + l + 32, ... in turn, then a fixed shuffle tree), in double-float.  On return v holds
// those totals, identical in every thread of every block that passed the same range.
// Returns false in every thread of the block when the spin budget (clock cycles) ran out.
// grid_allreduce_then runs `work()` in every thread after the block's arrival and before the
// wait: block-local work that the barrier neither orders nor waits for (its writes are not
// released to other blocks), overlapped with the barrier's latency.
// A barrier group is the whole grid by default; `grp` names a subset of the grid instead (a block
// range that works on one problem): the block's rank within it and its size.  The group's sync
// words (a counter and slots for grp.size blocks) are its own.
struct NoWork {
  __device__ void operator()() const {}
};
struct BarrierGroup {
  int rank, size;
};
__device__ __forceinline__ BarrierGroup whole_grid() {
  return BarrierGroup{(int)blockIdx.x, (int)gridDim.x};
}
template <int K, typename F>
__device__ __forceinline__ bool grid_allreduce_then(float (&v)[K], unsigned* sync, unsigned gen,
                                                    float* shf, df32* shd, F&& work,
                                                    int first = 0, int count = -1,
                                                    long long budget = kBarrierSpinCycles,
                                                    BarrierGroup grp = whole_grid()) {
  static_assert(K >= 1 && K <= kSyncMaxK, "grid_allreduce: K exceeds the slot width");
  const int tid = threadIdx.x, nb = grp.size;
  if (count < 0) count = nb;
  unsigned* counter = sync;
  float* slot = reinterpret_cast<float*>(sync + kSyncHeader) + (size_t)(gen & 1u) * nb * kSyncMaxK;
  __shared__ int ok_sh;
  block_sum<K, float>(v, shf);   // its barrier orders this block's phase writes before the release
  if (tid == 0) {
#pragma unroll
    for (int i = 0; i < K; ++i) __stcg(slot + grp.rank * K + i, v[i]);
    red_release_add(counter, 1u);
  }
  work();
  if (tid == 0) {
    const unsigned target = gen * (unsigned)nb;
    const long long t0 = clock64();
    int ok = 1;
    while ((int)(ld_acquire(counter) - target) < 0) {
      if (clock64() - t0 > budget) { ok = 0; break; }
    }
    ok_sh = ok;
  }
  __syncthreads();
  if (!ok_sh) return false;
  if (tid < 32) {
    df32 acc[K];
#pragma unroll
    for (int i = 0; i < K; ++i) acc[i] = df32{0.f, 0.f};
    // kSumChunk blocks per lane in flight per round, then added in block order
    for (int b0 = first + tid; b0 < first + count; b0 += 32 * kSumChunk) {
      float x[kSumChunk][K];
#pragma unroll
      for (int j = 0; j < kSumChunk; ++j) {
        const int b = b0 + 32 * j;
#pragma unroll
        for (int i = 0; i < K; ++i) x[j][i] = b < first + count ? __ldcg(slot + b * K + i) : 0.f;
      }
#pragma unroll
      for (int j = 0; j < kSumChunk; ++j)
        if (b0 + 32 * j < first + count)
#pragma unroll
          for (int i = 0; i < K; ++i) acc[i] = df_add(acc[i], df32{x[j][i], 0.f});
    }
#pragma unroll
    for (int i = 0; i < K; ++i)
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) acc[i] = df_add(acc[i], df_shfl_down(acc[i], off));
    if (tid == 0)
#pragma unroll
      for (int i = 0; i < K; ++i) shd[i] = acc[i];
  }
  __syncthreads();
#pragma unroll
  for (int i = 0; i < K; ++i) v[i] = shd[i].hi + shd[i].lo;
  return true;
}
template <int K>
__device__ __forceinline__ bool grid_allreduce(float (&v)[K], unsigned* sync, unsigned gen,
                                               float* shf, df32* shd, int first = 0,
                                               int count = -1,
                                               long long budget = kBarrierSpinCycles,
                                               BarrierGroup grp = whole_grid()) {
  return grid_allreduce_then<K>(v, sync, gen, shf, shd, NoWork{}, first, count, budget, grp);
}

// grid_allreduce over the group (next generation of gen) with the totals also in double: hi + lo
// of the double-float sums
template <int K>
__device__ __forceinline__ bool group_sum_d(float (&v)[K], double (&tot)[K], unsigned* sync,
                                            unsigned& gen, float* shf, df32* shd,
                                            BarrierGroup grp = whole_grid()) {
  if (!grid_allreduce<K>(v, sync, ++gen, shf, shd, 0, -1, kBarrierSpinCycles, grp)) return false;
#pragma unroll
  for (int i = 0; i < K; ++i) tot[i] = (double)shd[i].hi + (double)shd[i].lo;
  return true;
}

__device__ __forceinline__ void st_relaxed_u64(unsigned long long* p, unsigned long long v) {
  asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ unsigned long long ld_relaxed_u64(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void red_relaxed_add(unsigned* p, unsigned v) {
  asm volatile("red.relaxed.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ unsigned ld_relaxed_u32(const unsigned* p) {
  unsigned v;
  asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

constexpr int kTagWordsPerLane = kTagWordsPerLaneHost;   // block ranges of up to 512 blocks

// The barrier + sum of one float per thread for a phase after which no block reads another
// block's memory writes: only the sums cross blocks, so no release / acquire ordering is needed
// and the arrival does not wait for the block's outstanding stores.  Block b's sum travels as a
// 64-bit word (gen << 32 | bits) in the tagged-word area of `sync` (after the float slots), the
// arrival count uses the same counter as grid_allreduce (relaxed).  Warp 0 reads all words; a
// word not yet carrying this generation (its store still in flight when the count completed) is
// read again.  Same fixed order and double-float sums as grid_allreduce, over the blocks first ..
// first + count - 1 (default: all).  Requires count <= 32 * kTagWordsPerLane.  Returns false in
// every thread of the block when the budget ran out.
__device__ __forceinline__ bool grid_allreduce_unordered(float& v, unsigned* sync, unsigned gen,
                                                         float* shf, df32* shd, int first = 0,
                                                         int count = -1,
                                                         long long budget = kBarrierSpinCycles,
                                                         BarrierGroup grp = whole_grid()) {
  const int tid = threadIdx.x, nb = grp.size;
  if (count < 0) count = nb;
  unsigned* counter = sync;
  unsigned long long* words = reinterpret_cast<unsigned long long*>(
      sync + kSyncHeader + 2 * (size_t)nb * kSyncMaxK) + (size_t)(gen & 1u) * nb;
  __shared__ int ok_sh, ok2_sh;
  float vv[1] = {v};
  block_sum<1, float>(vv, shf);
  if (tid == 0) {
    st_relaxed_u64(words + grp.rank, ((unsigned long long)gen << 32) | __float_as_uint(vv[0]));
    red_relaxed_add(counter, 1u);
    const unsigned target = gen * (unsigned)nb;
    const long long t0 = clock64();
    int ok = 1;
    while ((int)(ld_relaxed_u32(counter) - target) < 0) {
      if (clock64() - t0 > budget) { ok = 0; break; }
    }
    ok_sh = ok;
  }
  __syncthreads();
  if (!ok_sh) return false;
  if (tid < 32) {
    unsigned long long w[kTagWordsPerLane];
    unsigned need = 0;
#pragma unroll
    for (int j = 0; j < kTagWordsPerLane; ++j) {
      const int b = tid + 32 * j;
      w[j] = b < count ? ld_relaxed_u64(words + first + b) : 0ull;
      if (b < count && (unsigned)(w[j] >> 32) != gen) need |= 1u << j;
    }
    const long long t0 = clock64();
    bool ok = true;
    while (need) {
#pragma unroll
      for (int j = 0; j < kTagWordsPerLane; ++j)
        if (need & (1u << j)) {
          w[j] = ld_relaxed_u64(words + first + tid + 32 * j);
          if ((unsigned)(w[j] >> 32) == gen) need &= ~(1u << j);
        }
      if (need && clock64() - t0 > budget) { ok = false; break; }
    }
    df32 acc{0.f, 0.f};
#pragma unroll
    for (int j = 0; j < kTagWordsPerLane; ++j)
      if (tid + 32 * j < count) acc = df_add(acc, df32{__uint_as_float((unsigned)w[j]), 0.f});
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) acc = df_add(acc, df_shfl_down(acc, off));
    if (tid == 0) { shd[0] = acc; ok2_sh = ok ? 1 : 0; }
  }
  __syncthreads();
  if (!ok2_sh) return false;
  v = shd[0].hi + shd[0].lo;
  return true;
}

}  // namespace hysco
