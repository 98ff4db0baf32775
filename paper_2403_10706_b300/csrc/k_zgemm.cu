// ADMM z-update products on the tensor cores (Sec. 2.3.2): the four real Fourier-basis products of
// the per-plane inversion of alpha H_G + rho I, each one tall GEMM D = A B^T over all PE planes,
// computed by tcgen05.mma (kind::tf32, accumulator in tensor memory) from tiles that TMA copies into
// 64-byte-swizzled shared memory.
//
// Single precision from TF32 products (three-term split): an operand x is held as hi + lo with
// hi = x truncated to TF32 (10 fraction bits) and lo = x - hi (exact in FP32), and
//   A B^T ~= Ahi Bhi^T + Ahi Blo^T + Alo Bhi^T,
// the dropped Alo Blo^T and lo's own truncation being below 2^-20 of |A||B| per term; every
// product is accumulated in FP32 in tensor memory.  The MMA reads an FP32 word as TF32 by dropping
// its 13 low mantissa bits, so the copied x itself serves as hi and only lo is written.  The
// operands travel in FP32; each stage is split in shared memory after its TMA copy lands, so the
// pairs never pass through L2 or HBM.  The four launches (and the one before them, which forms
// X and G2's scale table) are a chain of programmatic dependent launches.
//
// Chain (planes k < E, in-plane axes A (n_A, fastest) and B (n_B)); X = b + u:
//   G1  D(k cB, jA) = sum_cA X(k, cB, cA) Q_A(cA, jA)                 forward, axis A
//   G2  D(k jA, jB) = sum_cB Y1(k, jA, cB) Q_B(cB, jB) . rho / lambda  forward, axis B, scaled
//   G3  D(k jB, cA) = sum_jA Y2(k, jB, jA) Q_A(cA, jA)                 inverse, axis A
//   G4  D(k cA, cB) = sum_jB Y3(k, cA, jB) Q_B(cB, jB) = z(k, cB, cA)  inverse, axis B
// Each product's rows (the tile's TMEM lanes, one per thread in the epilogue) run along the next
// product's contraction index, so every epilogue store is coalesced across a warp: G1-G3 write the
// next A operand transposed, and G4's rows put whichever of cA and k has unit stride in the
// pitched field fastest (cA unless the PE axis is the innermost one).
#include <cuda.h>

#include <algorithm>
#include <vector>

#include "hysco_internal.cuh"

namespace hysco {

constexpr int kZgM = 128;          // tile rows (the MMA's M; TMEM lane = row)
constexpr int kZgKB = 16;          // contraction depth per stage: one 64-byte swizzled row of floats
constexpr int kZgThreads = 320;    // warp 0: TMA copies, warp 1: MMAs, warps 2-9: the split of
                                   // each stage, then the epilogue (two warps per TMEM lane quarter)
constexpr int kZgConvThreads = 256;
constexpr int kZgMaxStages = 12;
constexpr int kZgMaxN = 256;       // the MMA's largest N (one tile spans all output columns)
constexpr long long kZgSpin = 1LL << 31;   // clock cycles a wait may take before the launch gives up
                                           // (about a second)

// where the epilogue puts D(r, j): row r -> (q, x) = (r / n_row, r % n_row), element
// q sq + x sx + j sj of out; SCALE multiplies by scale[j ss + x]
struct ZgEpi {
  float* out;
  int n_row;
  long long sq, sx, sj;
  const float* scale;
  int ss;
};

__device__ __forceinline__ uint32_t zg_smem(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void zg_bar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void zg_bar_expect(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool zg_bar_try(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}

// wait for the phase of the given parity to complete; false once `spin` clock cycles have passed
__device__ __forceinline__ bool zg_bar_wait(uint32_t bar, uint32_t parity, long long spin) {
  if (zg_bar_try(bar, parity)) return true;
  const long long t0 = clock64();
  while (!zg_bar_try(bar, parity))
    if (clock64() - t0 > spin) return false;
  return true;
}

// 2D tiled TMA load of the box at (x, y) (x: the inner, contiguous coordinate) into shared memory,
// completing on the mbarrier's transaction count
__device__ __forceinline__ void zg_tma_load(uint32_t dst, const CUtensorMap* map, uint32_t bar,
                                            int x, int y) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, "
      "%4}], [%2];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(bar), "r"(x), "r"(y)
      : "memory");
}

__device__ __forceinline__ void zg_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void zg_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// shared-memory matrix descriptor of a K-major tile with the 64-byte swizzle: rows of 64 bytes,
// groups of eight rows 512 bytes apart (stride byte offset), leading byte offset unused (1),
// descriptor version 1 (bits 46-47), swizzle mode 4 = 64 bytes (bits 61-63)
__device__ __forceinline__ uint64_t zg_desc(uint32_t saddr) {
  return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)1 << 16) | ((uint64_t)(512 >> 4) << 32) |
         ((uint64_t)1 << 46) | ((uint64_t)4 << 61);
}

// instruction descriptor of kind::tf32: D in F32 (bits 4-5 = 1), A and B TF32 (bits 7-9, 10-12 =
// 2), both K-major (bits 15, 16 = 0), N >> 3 in bits 17-22, M >> 4 in bits 24-28
__host__ __device__ constexpr uint32_t zg_idesc(int M, int N) {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) |
         ((uint32_t)(M >> 4) << 24);
}

// D (+)= A B^T for one K = 8 slice; acc = 0 overwrites D
__device__ __forceinline__ void zg_mma(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc,
                                       uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(d),
      "l"(a), "l"(b), "r"(idesc), "r"(acc)
      : "memory");
}

// the mbarrier receives one arrival once every MMA this thread issued so far has completed
__device__ __forceinline__ void zg_commit(uint32_t bar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
      : "memory");
}

// issue the load of 16 consecutive accumulator columns of the thread's TMEM lane (warp w reads
// lanes 32 w ..); the registers hold the values after zg_ld_wait
__device__ __forceinline__ void zg_ld16(uint32_t taddr, uint32_t* r) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, "
      "%12, %13, %14, %15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15])
      : "r"(taddr)
      : "memory");
}

// wait for the thread's outstanding TMEM loads; the registers pass through the wait so that no
// use of them is scheduled before it
__device__ __forceinline__ void zg_ld_wait(uint32_t (&r)[32]) {
  asm volatile(
      "tcgen05.wait::ld.sync.aligned;"
      : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]),
        "+r"(r[7]), "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]), "+r"(r[12]), "+r"(r[13]),
        "+r"(r[14]), "+r"(r[15]), "+r"(r[16]), "+r"(r[17]), "+r"(r[18]), "+r"(r[19]),
        "+r"(r[20]), "+r"(r[21]), "+r"(r[22]), "+r"(r[23]), "+r"(r[24]), "+r"(r[25]),
        "+r"(r[26]), "+r"(r[27]), "+r"(r[28]), "+r"(r[29]), "+r"(r[30]), "+r"(r[31])
      :
      : "memory");
}

// x truncated to TF32 (its 13 low mantissa bits cleared): the value the MMA reads for x
__device__ __forceinline__ float zg_tf32_trunc(float x) {
  return __uint_as_float(__float_as_uint(x) & 0xFFFFE000u);
}

// One 128-row tile of D = A B^T per block (A: M x K, B: N x K, both K-major FP32 behind the
// tensor maps; N <= BN <= 256, BN a multiple of 16).  Roles per stage of 16 contraction columns:
//   lane 0 of warp 0   TMA-copies the FP32 tiles of A (128 rows) and B (BN rows) into the stage's
//                      hi slots (rows past M and columns past K read as zeros);
//   warps 2-9          write lo = x - (x truncated to TF32) into the lo slots (the copy is hi;
//                      an elementwise map, so the 64-byte swizzle of the copies carries over),
//                      then fence the writes to the async proxy and arrive on the stage;
//   lane 0 of warp 1   issues three MMAs per K = 8 slice (hi hi, hi lo, lo hi) into one TMEM
//                      accumulator of BN columns and frees the stage by a commit.
// Then warps 2-9 take the accumulator's rows (TMEM lane quarter warp % 4, alternate 16-column
// chunks, 32 columns per wait) to global memory as ZgEpi says.  A wait that runs out of its
// budget (spin clock cycles) records HYSCO_ETIMEOUT in the device state and stops the solve; the
// launch then skips its stores, frees its tensor memory and ends.  no_copy (the failure self-test
// only): the producer issues no copies, so the first stage never fills and the waits on it run
// out — no copy or MMA is then in flight when the launch ends.
template <bool SCALE>
__global__ void __launch_bounds__(kZgThreads, 1)
k_zgemm(const __grid_constant__ CUtensorMap tA, const __grid_constant__ CUtensorMap tB, int M,
        int N, int K, int BN, int stages, ZgEpi ep, DevState* st, long long spin, int no_copy) {
  // the next launch of the chain may start its setup now
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  extern __shared__ unsigned char zg_dyn[];
  __shared__ __align__(8) unsigned long long bars[3 * kZgMaxStages + 1];
  __shared__ uint32_t tmem_slot;
  __shared__ int failed;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t raw = zg_smem(zg_dyn);
  const uint32_t base = (raw + 1023u) & ~1023u;   // tiles start on 1024-byte boundaries
  unsigned char* const gbase = zg_dyn + (base - raw);
  const uint32_t a_bytes = kZgM * kZgKB * 4, b_bytes = (uint32_t)BN * kZgKB * 4;
  const uint32_t stage_bytes = 2 * a_bytes + 2 * b_bytes;   // A hi, A lo, B hi, B lo
  const uint32_t full0 = zg_smem(&bars[0]), conv0 = zg_smem(&bars[kZgMaxStages]),
                 empty0 = zg_smem(&bars[2 * kZgMaxStages]), done = zg_smem(&bars[3 * kZgMaxStages]);
  const uint32_t ncols = BN <= 32 ? 32u : BN <= 64 ? 64u : BN <= 128 ? 128u : 256u;
  const int nkb = (K + kZgKB - 1) / kZgKB;
  const int row0 = blockIdx.x * kZgM;
  if (threadIdx.x == 0) {
    for (int s = 0; s < stages; ++s) {
      zg_bar_init(full0 + 8 * s, 1);
      zg_bar_init(conv0 + 8 * s, kZgConvThreads);
      zg_bar_init(empty0 + 8 * s, 1);
    }
    zg_bar_init(done, 1);
    failed = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     zg_smem(&tmem_slot)),
                 "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  zg_fence_before();
  __syncthreads();
  zg_fence_after();
  const uint32_t tmem = tmem_slot;
  // the setup above overlapped the previous launch's tail (programmatic dependent launch); every
  // global access below waits for that launch to complete.  A stopped solve skips the work (a
  // block-wide decision, taken after the wait so that every thread sees the same state).
  asm volatile("griddepcontrol.wait;" ::: "memory");
  if (threadIdx.x == 0 && st->stop) failed = 2;
  __syncthreads();
  const bool run = *(volatile int*)&failed == 0;

  if (run && warp == 0 && lane == 0 && !no_copy) {
    // producer: stage s takes K block kb, kb + stages, ...; a refill waits for the MMAs that read
    // the stage's previous block
    for (int kb = 0; kb < nkb; ++kb) {
      const int s = kb % stages;
      if (kb >= stages && !zg_bar_wait(empty0 + 8 * s, (uint32_t)(kb / stages - 1) & 1u, spin)) {
        failed = 1;
        break;
      }
      const uint32_t sa = base + (uint32_t)s * stage_bytes, bar = full0 + 8 * s;
      zg_bar_expect(bar, a_bytes + b_bytes);
      zg_tma_load(sa, &tA, bar, kb * kZgKB, row0);
      zg_tma_load(sa + 2 * a_bytes, &tB, bar, kb * kZgKB, 0);
    }
  } else if (run && warp == 1 && lane == 0) {
    // MMA issuer: hi hi, hi lo, lo hi per K = 8 slice (the next slice 32 bytes along the rows)
    const uint32_t idesc = zg_idesc(kZgM, BN);
    for (int kb = 0; kb < nkb; ++kb) {
      const int s = kb % stages;
      if (!zg_bar_wait(conv0 + 8 * s, (uint32_t)(kb / stages) & 1u, spin)) {
        failed = 1;
        break;
      }
      zg_fence_after();
      const uint32_t sa = base + (uint32_t)s * stage_bytes;
      const int nk8 = min(kZgKB / 8, (K - kb * kZgKB + 7) / 8);
      for (int q = 0; q < nk8; ++q) {
        const uint32_t off = (uint32_t)q * 32u;
        const uint64_t ah = zg_desc(sa + off), al = zg_desc(sa + a_bytes + off);
        const uint64_t bh = zg_desc(sa + 2 * a_bytes + off);
        const uint64_t bl = zg_desc(sa + 2 * a_bytes + b_bytes + off);
        zg_mma(tmem, ah, bh, idesc, (kb > 0 || q > 0) ? 1u : 0u);
        zg_mma(tmem, ah, bl, idesc, 1u);
        zg_mma(tmem, al, bh, idesc, 1u);
      }
      zg_commit(empty0 + 8 * s);
    }
    zg_commit(done);
  } else if (run && warp >= 2) {
    // converters: the lo half of each TF32 pair beside the stage's FP32 copy (its hi half)
    const int ct = threadIdx.x - 64;
    for (int kb = 0; kb < nkb; ++kb) {
      const int s = kb % stages;
      if (!zg_bar_wait(full0 + 8 * s, (uint32_t)(kb / stages) & 1u, spin)) {
        failed = 1;
        break;
      }
      float4* const ah = reinterpret_cast<float4*>(gbase + (size_t)s * stage_bytes);
      float4* const bh = reinterpret_cast<float4*>(gbase + (size_t)s * stage_bytes + 2 * a_bytes);
      const int na4 = (int)(a_bytes / 16), nb4 = (int)(b_bytes / 16);
      for (int i = ct; i < na4 + nb4; i += kZgConvThreads) {
        float4* const h = i < na4 ? ah + i : bh + (i - na4);
        float4* const l = i < na4 ? ah + na4 + i : bh + nb4 + (i - na4);
        const float4 x = *h;
        *l = make_float4(x.x - zg_tf32_trunc(x.x), x.y - zg_tf32_trunc(x.y),
                         x.z - zg_tf32_trunc(x.z), x.w - zg_tf32_trunc(x.w));
      }
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(conv0 + 8 * s) : "memory");
    }
  }
  __syncwarp();
  const bool ok = run && zg_bar_wait(done, 0, spin);
  __syncthreads();
  zg_fence_after();
  const int fl = *(volatile int*)&failed;
  const bool good = ok && fl == 0;
  if (warp >= 2) {
    // epilogue: thread = row r of the tile (TMEM lane 32 (warp % 4) + lane); warps 2-5 take the
    // even 16-column chunks, warps 6-9 the odd ones, two chunks per wait
    const int quad = warp & 3, grp = (warp - 2) >> 2;
    const int r = row0 + quad * 32 + lane;
    const bool rv = good && r < M;
    long long rb = 0;
    int x = 0;
    if (rv) {
      const int q = r / ep.n_row;
      x = r - q * ep.n_row;
      rb = (long long)q * ep.sq + (long long)x * ep.sx;
    }
    const uint32_t tl = tmem + ((uint32_t)(quad * 32) << 16);
    const int nch = BN / 16;
    __syncwarp();
    for (int ch = grp; ch < nch; ch += 4) {
      uint32_t v[32];
      zg_ld16(tl + (uint32_t)(ch * 16), v);
      const bool two = ch + 2 < nch;
      if (two) zg_ld16(tl + (uint32_t)((ch + 2) * 16), v + 16);
      // the chunk's scale factors, all loads in flight before the first store
      float sc[32];
      if (SCALE && rv) {
#pragma unroll
        for (int u = 0; u < 32; ++u) {
          const int j = min((u < 16 ? ch : ch + 2) * 16 + (u & 15), N - 1);
          sc[u] = __ldg(ep.scale + (long long)j * ep.ss + x);
        }
      }
      zg_ld_wait(v);
      if (rv) {
#pragma unroll
        for (int u = 0; u < 32; ++u) {
          const int j = (u < 16 ? ch : ch + 2) * 16 + (u & 15);
          if ((u < 16 || two) && j < N) {
            float val = __uint_as_float(v[u]);
            if (SCALE) val *= sc[u];
            ep.out[rb + (long long)j * ep.sj] = val;
          }
        }
      }
      __syncwarp();
    }
  }
  zg_fence_before();
  __syncthreads();
  if (warp == 0) {
    zg_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(ncols)
                 : "memory");
  }
  if (run && !good && threadIdx.x == 0) {   // a wait ran out of its budget
    st->status = -6;   // HYSCO_ETIMEOUT
    st->stop = 1;
  }
}

// X = b + u as G1's A operand (row k nB + cB, column cA, row pitch Kp); the blocks of the first
// node segment also write G2's scale rho / lambda(jB, jA) with lambda = rho + alpha (wB muB[jB] +
// wA muA[jA]) at S[jB Kp + jA] (rho from the device state)
__global__ void __launch_bounds__(kBlock)
k_zrhs_tc(Geo g, const float* __restrict__ b, const float* __restrict__ u, float* __restrict__ X,
          int Kp, const float* __restrict__ muA, const float* __restrict__ muB,
          float* __restrict__ S, const DevState* st) {
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");   // G1 may start its setup
  if (st->stop) return;
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= g.ncols) return;
  const int fb = col_base(c, g.inner, g.fld_ostride), pb = col_pbase(g, c);
  const int cB = c / g.nA, cA = c - cB * g.nA;
  if (blockIdx.y == 0) {
    const float rho = st->admm_rho;
    S[(long long)cB * Kp + cA] =
        rho / (rho + g.alpha * (g.wB * __ldg(muB + cB) + g.wA * __ldg(muA + cA)));
  }
  const int k0 = blockIdx.y * 8, k1 = min(k0 + 8, g.E);
  for (int k = k0; k < k1; ++k)
    X[((long long)k * g.nB + cB) * Kp + cA] = __ldg(b + fb + k * g.inner) + __ldg(u + pb + k * g.psP);
}

// ------------------------------------------------------------------------------------------
// host: tensor maps, split bases, the four launches
// ------------------------------------------------------------------------------------------

using ZgEncode = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                              const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                              const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                              CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

// the driver's tensor-map encoder, looked up once through the runtime (null if unavailable)
ZgEncode zg_encoder() {
  static const ZgEncode fn = []() -> ZgEncode {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess) {
      cudaGetLastError();
      return nullptr;
    }
    return reinterpret_cast<ZgEncode>(p);
  }();
  return fn;
}

// map of a rows x K float array (row pitch Kp floats, Kp a multiple of 4) in boxes of 16 columns
// x box_rows rows, 64-byte swizzle, zeros outside the array
bool zg_map(CUtensorMap* m, const float* p, int K, long long rows, int Kp, int box_rows) {
  const ZgEncode enc = zg_encoder();
  if (!enc) return false;
  const cuuint64_t dims[2] = {(cuuint64_t)K, (cuuint64_t)rows};
  const cuuint64_t strides[1] = {(cuuint64_t)Kp * sizeof(float)};
  const cuuint32_t box[2] = {(cuuint32_t)kZgKB, (cuuint32_t)box_rows};
  const cuuint32_t es[2] = {1, 1};
  return enc(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float*>(p), dims, strides, box, es,
             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B,
             CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

struct ZgPlan {
  CUtensorMap tP, tQ, tB[4];           // A operands and the four bases
  float* P = nullptr;                   // X and Y2: E nB rows x KpA
  float* Q = nullptr;                   // Y1 and Y3: E nA rows x KpB
  float* Bm = nullptr;                  // the bases
  float* S = nullptr;                   // G2's scale rho / lambda, nB rows x KpA
  int nA = 0, nB = 0, E = 0, KpA = 0, KpB = 0, BNA = 0, BNB = 0;
  int stA = 0, stB = 0, smA = 0, smB = 0;   // stages and shared memory of G1/G3 and of G2/G4
};

void zg_destroy(ZgPlan* p) {
  if (!p) return;
  for (float* b : {p->P, p->Q, p->Bm, p->S})
    if (b) cudaFree(b);
  delete p;
}

namespace {

// stages of BN-column tiles: with no more tiles than SMs, as many as one block may hold (220 KB,
// the 1024 bytes of alignment slack included) so that all of a tile's copies are in flight at
// once; otherwise as many as let two blocks share an SM (110 KB each), so that one block's
// epilogue overlaps the other's copies
int zg_stages(int BN, int K, int tiles, int sms) {
  const int stage = 2 * kZgM * kZgKB * 4 + 2 * BN * kZgKB * 4;
  const int fit = ((tiles <= sms ? 220 : 110) * 1024 - 1024) / stage;
  return std::max(1, std::min({fit, kZgMaxStages, (K + kZgKB - 1) / kZgKB}));
}

int zg_smem_bytes(int BN, int stages) {
  return stages * (2 * kZgM * kZgKB * 4 + 2 * BN * kZgKB * 4) + 1024;
}

}  // namespace

// The tensor-core plan for a geometry's z-update, or null where it does not apply (an in-plane
// axis longer than the MMA's largest N, no tensor-map encoder, or an allocation failure).  QA, QB:
// the host bases (row = position, column = basis function).
ZgPlan* zg_create(const Geo& g, const std::vector<float>& QA, const std::vector<float>& QB) {
  const int nA = g.nA, nB = g.nB, E = g.E;
  if (nA > kZgMaxN || nB > kZgMaxN || nA < 1 || nB < 1 || !zg_encoder()) return nullptr;
  ZgPlan* p = new ZgPlan();
  p->nA = nA;
  p->nB = nB;
  p->E = E;
  p->KpA = (nA + 3) & ~3;
  p->KpB = (nB + 3) & ~3;
  p->BNA = (nA + 15) & ~15;
  p->BNB = (nB + 15) & ~15;
  int dev = 0, sms = 148;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
    cudaGetLastError();
    delete p;
    return nullptr;
  }
  p->stA = zg_stages(p->BNA, nA, ceil_div(E * nB, kZgM), sms);
  p->stB = zg_stages(p->BNB, nB, ceil_div(E * nA, kZgM), sms);
  p->smA = zg_smem_bytes(p->BNA, p->stA);
  p->smB = zg_smem_bytes(p->BNB, p->stB);
  const size_t np = (size_t)E * nB * p->KpA, nq = (size_t)E * nA * p->KpB;
  const size_t nbA = (size_t)nA * p->KpA, nbB = (size_t)nB * p->KpB;
  // pitch padding is never read (the maps stop at K), but keep it defined
  bool ok = cudaMalloc((void**)&p->P, np * sizeof(float)) == cudaSuccess &&
            cudaMalloc((void**)&p->Q, nq * sizeof(float)) == cudaSuccess &&
            cudaMemset(p->P, 0, np * sizeof(float)) == cudaSuccess &&
            cudaMemset(p->Q, 0, nq * sizeof(float)) == cudaSuccess &&
            cudaMalloc((void**)&p->Bm, (2 * nbA + 2 * nbB) * sizeof(float)) == cudaSuccess &&
            cudaMalloc((void**)&p->S, (size_t)nB * p->KpA * sizeof(float)) == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    zg_destroy(p);
    return nullptr;
  }
  // B operands as N x K (K-major): G1 Q_A^T, G2 Q_B^T, G3 Q_A, G4 Q_B
  std::vector<float> hb(2 * nbA + 2 * nbB, 0.f);
  const size_t off[4] = {0, nbA, nbA + nbB, 2 * nbA + nbB};
  for (int t = 0; t < 4; ++t) {
    const int n = (t % 2 == 0) ? nA : nB, Kp = (t % 2 == 0) ? p->KpA : p->KpB;
    const std::vector<float>& Q = (t % 2 == 0) ? QA : QB;
    for (int row = 0; row < n; ++row)   // row = output index, col = contraction index
      for (int col = 0; col < n; ++col)
        hb[off[t] + (size_t)row * Kp + col] =
            (t < 2) ? Q[(size_t)col * n + row] : Q[(size_t)row * n + col];
  }
  ok = cudaMemcpy(p->Bm, hb.data(), hb.size() * sizeof(float), cudaMemcpyHostToDevice) ==
           cudaSuccess &&
       zg_map(&p->tP, p->P, nA, (long long)E * nB, p->KpA, kZgM) &&
       zg_map(&p->tQ, p->Q, nB, (long long)E * nA, p->KpB, kZgM);
  for (int t = 0; t < 4 && ok; ++t) {
    const int n = (t % 2 == 0) ? nA : nB, Kp = (t % 2 == 0) ? p->KpA : p->KpB;
    const int BN = (t % 2 == 0) ? p->BNA : p->BNB;
    ok = zg_map(&p->tB[t], p->Bm + off[t], n, n, Kp, BN);
  }
  if (ok) {
    const int sm = std::max(p->smA, p->smB);
    ok = cudaFuncSetAttribute(k_zgemm<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm) ==
             cudaSuccess &&
         cudaFuncSetAttribute(k_zgemm<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm) ==
             cudaSuccess;
  }
  if (!ok) {
    cudaGetLastError();
    zg_destroy(p);
    return nullptr;
  }
  return p;
}

// one product of the chain, launched as a programmatic dependent of the launch before it (its
// prologue overlaps that launch's tail; its global accesses wait for it to complete)
template <bool SCALE>
cudaError_t zg_launch(const ZgPlan* p, const CUtensorMap& tA, const CUtensorMap& tB, int M, int N,
                      int BN, int stages, int smem, const ZgEpi& ep, DevState* st,
                      cudaStream_t s) {
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = dim3(ceil_div(M, kZgM));
  cfg.blockDim = dim3(kZgThreads);
  cfg.dynamicSmemBytes = (size_t)smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  (void)p;
  return cudaLaunchKernelEx(&cfg, k_zgemm<SCALE>, tA, tB, M, N, N, BN, stages, ep, st, kZgSpin, 0);
}

// The failure self-test: one launch of the first product whose producer issues no copies, with a
// wait budget of `spin` clock cycles; its converters and its MMA issuer give up on the unfilled
// stage, and the launch records HYSCO_ETIMEOUT in st and ends (nothing in flight, TMEM freed).
cudaError_t zg_selftest(const ZgPlan* p, DevState* st, long long spin, cudaStream_t s) {
  const ZgEpi e{p->Q, p->nB, (long long)p->nA * p->KpB, 1, p->KpB, nullptr, 0};
  k_zgemm<false><<<ceil_div(p->E * p->nB, kZgM), kZgThreads, p->smA, s>>>(
      p->tP, p->tB[0], p->E * p->nB, p->nA, p->nA, p->BNA, p->stA, e, st, spin, 1);
  return cudaGetLastError();
}

#define ZG_TRY(expr)                 \
  do {                               \
    cudaError_t e_ = (expr);         \
    if (e_ != cudaSuccess) return e_; \
  } while (0)

// z = rho (alpha H_G + rho I)^{-1} (b + u) in the pitched field, by the chain G1-G4
cudaError_t launch_zgemm_zsolve(const ZgPlan* p, const Geo& g, const float* b, const float* u,
                                const AdmmBasis& q, float* z, DevState* st, cudaStream_t s) {
  const int nA = p->nA, nB = p->nB, E = p->E;
  k_zrhs_tc<<<dim3(ceil_div(g.ncols, kBlock), ceil_div(E, 8)), kBlock, 0, s>>>(
      g, b, u, p->P, p->KpA, q.muA, q.muB, p->S, st);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const ZgEpi e1{p->Q, nB, (long long)nA * p->KpB, 1, p->KpB, nullptr, 0};
  ZG_TRY(zg_launch<false>(p, p->tP, p->tB[0], E * nB, nA, p->BNA, p->stA, p->smA, e1, st, s));
  const ZgEpi e2{p->P, nA, (long long)nB * p->KpA, 1, p->KpA, p->S, p->KpA};
  ZG_TRY(zg_launch<true>(p, p->tQ, p->tB[1], E * nA, nB, p->BNB, p->stB, p->smB, e2, st, s));
  // G4's rows: (k, cA) with cA fastest where cA has unit stride in the pitched field, else
  // (cA, k) with k fastest (PE axis innermost); G3 writes its output in that row order
  const bool afast = g.psA == 1 || g.psP != 1;
  const ZgEpi e3 = afast ? ZgEpi{p->Q, nB, (long long)nA * p->KpB, 1, p->KpB, nullptr, 0}
                         : ZgEpi{p->Q, nB, p->KpB, 1, (long long)E * p->KpB, nullptr, 0};
  ZG_TRY(zg_launch<false>(p, p->tP, p->tB[2], E * nB, nA, p->BNA, p->stA, p->smA, e3, st, s));
  const ZgEpi e4 = afast ? ZgEpi{z, nA, g.psP, g.psA, g.psB, nullptr, 0}
                         : ZgEpi{z, E, g.psA, g.psP, g.psB, nullptr, 0};
  ZG_TRY(zg_launch<false>(p, p->tQ, p->tB[3], nA * E, nB, p->BNB, p->stB, p->smB, e4, st, s));
  return cudaSuccess;
}

}  // namespace hysco
