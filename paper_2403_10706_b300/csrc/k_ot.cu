// Optimal-transport field-map initialisation (Sec. 2.2) and the 3x3x3 Gaussian blur (Sec. 2.4).
//
// k_ot_shift: one pass over both images for min and max|I|; the last block forms the positivity
//   shift s = max(0, -min) + eps * max|I| in single precision.
// k_ot: one CTA per tile of CW consecutive PE columns.  The shifted intensities of both images are
//   staged in shared memory with coalesced row loads; one thread per column forms the cumulative
//   sums left to right (single precision, the order a sequential loop uses, so the result is
//   bit-reproducible); all threads normalise, and every node k looks up
//     k* = min{j in [0, m-1] : C(j+1) >= r}    (binary search on the other image's CDF)
//   and C^{-1}(r) = k* + (r - C(k*)) / (C(k*+1) - C(k*)), capped at m.  Then
//     b0_k = 1/4 [ (C+^{-1}(C-(k)) - k) - (C-^{-1}(C+(k)) - k) ].
// k_blur3: the separable 3-tap weights [e^-1/2, 1, e^-1/2] / (1 + 2 e^-1/2) per axis (sigma = 1
//   voxel), replicate boundary, as one launch: a CTA stages an 8 x 8 x 32 brick of the field with
//   a one-node halo in shared memory (clamped coordinates, so the halo replicates the boundary)
//   and applies the passes along axis 0, 1 and 2 in that order, each pass's values rounded to
//   single precision as three separate passes would round them.
#include <algorithm>
#include <cmath>

#include "hysco_internal.cuh"

namespace hysco {

template <typename TI>
__global__ void __launch_bounds__(kBlock)
k_ot_shift(const TI* __restrict__ Ip, const TI* __restrict__ Im, int n, float eps,
           float* partials, unsigned* counter, DevState* st) {
  float mn = __int_as_float(0x7f800000), mx = 0.f;
  const int T = gridDim.x * blockDim.x;
  // four independent loads per image in flight per thread
  for (int i0 = blockIdx.x * blockDim.x + threadIdx.x; i0 < n; i0 += 4 * T) {
    float a[4], b[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      int i = min(i0 + u * T, n - 1);
      a[u] = ldf(Ip + i);
      b[u] = ldf(Im + i);
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      mn = fminf(mn, fminf(a[u], b[u]));
      mx = fmaxf(mx, fmaxf(fabsf(a[u]), fabsf(b[u])));
    }
  }
  // min / max reduction through the same deterministic machinery (max(-min) and max|I|)
  __shared__ float smn[32], smx[32];
  __shared__ int is_last;
  for (int off = 16; off > 0; off >>= 1) {
    mn = fminf(mn, __shfl_down_sync(0xffffffffu, mn, off));
    mx = fmaxf(mx, __shfl_down_sync(0xffffffffu, mx, off));
  }
  int tid = threadIdx.x, nw = blockDim.x >> 5;
  if ((tid & 31) == 0) { smn[tid >> 5] = mn; smx[tid >> 5] = mx; }
  __syncthreads();
  if (tid < 32) {
    mn = tid < nw ? smn[tid] : __int_as_float(0x7f800000);
    mx = tid < nw ? smx[tid] : 0.f;
    for (int off = 16; off > 0; off >>= 1) {
      mn = fminf(mn, __shfl_down_sync(0xffffffffu, mn, off));
      mx = fmaxf(mx, __shfl_down_sync(0xffffffffu, mx, off));
    }
  }
  if (tid == 0) {
    partials[2 * blockIdx.x] = mn;
    partials[2 * blockIdx.x + 1] = mx;
    __threadfence();
    unsigned t = atomicAdd(counter, 1u);
    is_last = (t == gridDim.x - 1);
  }
  __syncthreads();
  if (!is_last) return;
  __threadfence();
  // warp 0 of the last block: lane l takes blocks l, l + 32, ... (eight loads in flight), then a
  // shuffle tree; min and max are exact in any order
  if (tid < 32) {
    float gmn = __int_as_float(0x7f800000), gmx = 0.f;
    const int nblk = gridDim.x;
    for (int b0 = tid; b0 < nblk; b0 += 32 * 8) {
      float lo[8], hi[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int b = b0 + 32 * u;
        lo[u] = b < nblk ? __ldcg(partials + 2 * b) : __int_as_float(0x7f800000);
        hi[u] = b < nblk ? __ldcg(partials + 2 * b + 1) : 0.f;
      }
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        gmn = fminf(gmn, lo[u]);
        gmx = fmaxf(gmx, hi[u]);
      }
    }
    for (int off = 16; off > 0; off >>= 1) {
      gmn = fminf(gmn, __shfl_down_sync(0xffffffffu, gmn, off));
      gmx = fmaxf(gmx, __shfl_down_sync(0xffffffffu, gmx, off));
    }
    if (tid == 0) {
      float neg = -gmn > 0.f ? -gmn : 0.f;
      float s = __fadd_rn(neg, __fmul_rn(eps, gmx));
      st->ot_shift = (double)s;
      *counter = 0u;
    }
  }
}

int ot_tile_width(int E) {
  if (8LL * E * 32 <= 200 * 1024) return 32;
  if (8LL * E * 16 <= 200 * 1024) return 16;
  if (8LL * E * 8 <= 200 * 1024) return 8;
  return 4;
}

// smallest j in [0, m-1] with C[j+1] >= r (m - 1 if none); C has stride CW
__device__ __forceinline__ int cdf_bracket(const float* C, int CW, int m, float r) {
  int lo = 0, hi = m - 1;
  while (lo < hi) {
    int mid = (lo + hi) >> 1;
    if (C[(mid + 1) * CW] >= r) hi = mid; else lo = mid + 1;
  }
  return lo;
}

// C^{-1}(r) on the bracket k = k*: k + (r - C(k)) / (C(k+1) - C(k)), capped at m.  The bracket
// gives C(k) < r <= C(k+1) (C(0) = 0 < r), so the fraction lies in (0, 1]; it is formed with the
// fast reciprocal (at most 2 ulp of error for a divisor in [2^-126, 2^126]) and saturated to
// [0, 1], which also covers a divisor below that range
__device__ __forceinline__ float spline_inverse(const float* C, int CW, int m, float r, int k) {
  const float c0 = C[k * CW], c1 = C[(k + 1) * CW];
  const float x = (float)k + __saturatef(__fdividef(r - c0, c1 - c0));
  return fminf(x, (float)m);
}

__device__ __forceinline__ float cdf_inverse(const float* C, int CW, int m, float r, int& kstar) {
  if (r <= 0.f) { kstar = 0; return 0.f; }
  int k = cdf_bracket(C, CW, m, r);
  kstar = k;
  return spline_inverse(C, CW, m, r, k);
}

// the same lookup with the bracket search started at kstar (a bracket of a smaller or equal r);
// kstar is updated in place
__device__ __forceinline__ float cdf_inverse_from(const float* C, int CW, int m, float r,
                                                  int& kstar) {
  if (r <= 0.f) { kstar = 0; return 0.f; }
  int k = kstar;
  while (k < m - 1 && !(C[(k + 1) * CW] >= r)) ++k;
  kstar = k;
  return spline_inverse(C, CW, m, r, k);
}

template <typename TI, bool INDICES>
__global__ void __launch_bounds__(kBlock)
k_ot(Geo g, const TI* __restrict__ Ip, const TI* __restrict__ Im, float* __restrict__ b0,
     int* __restrict__ kp, int* __restrict__ km, const DevState* st) {
  extern __shared__ float sm[];
  const int CW = blockDim.x, E = g.E, m = g.m;
  float* Cp = sm;            // [E][CW]
  float* Cm = sm + E * CW;   // [E][CW]
  int tx = threadIdx.x, ty = threadIdx.y;
  int c = blockIdx.x * CW + tx;
  bool act = c < g.ncols;
  float s = (float)st->ot_shift;
  int ib = act ? col_base(c, g.inner, g.img_ostride) : 0;
  // eight rows of both images in flight per thread (loads first, then the shifted stores)
  const int RY = blockDim.y;
  for (int k0 = ty; k0 < m; k0 += 8 * RY) {
    float a[8], b[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int k = k0 + u * RY;
      const bool in = act && k < m;
      a[u] = in ? ldf(Ip + ib + k * g.inner) : 0.f;
      b[u] = in ? ldf(Im + ib + k * g.inner) : 0.f;
    }
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int k = k0 + u * RY;
      if (k < m) {
        Cp[(k + 1) * CW + tx] = act ? __fadd_rn(a[u], s) : 0.f;
        Cm[(k + 1) * CW + tx] = act ? __fadd_rn(b[u], s) : 0.f;
      }
    }
  }
  __syncthreads();
  // cumulative sums, single precision, left to right: row 0 of threads scans I+, row 1 I-
  // (eight rows loaded ahead of their dependent additions)
  if (ty < 2) {
    float* C = ty == 0 ? Cp : Cm;
    float acc = 0.f;
    C[tx] = 0.f;
    int k = 1;
    for (; k + 7 <= m; k += 8) {
      float v[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) v[u] = C[(k + u) * CW + tx];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        acc = __fadd_rn(acc, v[u]);
        C[(k + u) * CW + tx] = acc;
      }
    }
    for (; k <= m; ++k) {
      acc = __fadd_rn(acc, C[k * CW + tx]);
      C[k * CW + tx] = acc;
    }
  }
  __syncthreads();
  float tp = Cp[m * CW + tx], tm = Cm[m * CW + tx];
  bool ok = tp > 0.f && tm > 0.f;
  __syncthreads();
  if (ok)
    for (int k = ty; k <= m; k += blockDim.y) {
      Cp[k * CW + tx] = __fdiv_rn(Cp[k * CW + tx], tp);
      Cm[k * CW + tx] = __fdiv_rn(Cm[k * CW + tx], tm);
    }
  __syncthreads();
  if (!act) return;
  int fb = col_base(c, g.inner, g.fld_ostride);
  // thread row ty takes the nodes [ka, kb): C+(k) and C-(k) do not decrease with k, so each
  // bracket min{j : C(j+1) >= r} is found from the previous node's by walking forward (the same
  // index a binary search finds), after one binary search at the run's first node
  const int L = ceil_div(E, (int)blockDim.y), ka = ty * L, kb = min(ka + L, E);
  int jp = -1, jm = -1;
  for (int k = ka; k < kb; ++k) {
    int i = fb + k * g.inner;
    if (!ok) {
      b0[i] = 0.f;
      if (INDICES) { kp[i] = 0; km[i] = 0; }
      continue;
    }
    const float rp = Cp[k * CW + tx], rm = Cm[k * CW + tx];
    float xp, xm;
    if (jp < 0) {
      xp = cdf_inverse(Cm + tx, CW, m, rp, jp);   // C-^{-1}(C+(k))
      xm = cdf_inverse(Cp + tx, CW, m, rm, jm);   // C+^{-1}(C-(k))
    } else {
      xp = cdf_inverse_from(Cm + tx, CW, m, rp, jp);
      xm = cdf_inverse_from(Cp + tx, CW, m, rm, jm);
    }
    float kf = (float)k;
    b0[i] = 0.25f * ((xm - kf) - (xp - kf));
    if (INDICES) { kp[i] = jp; km[i] = jm; }
  }
}

// The 3x3x3 Gaussian in one launch.  CTA (bx, by, bz) owns the brick of BZ x BY x BX nodes at
// (bz BZ, by BY, bx BX) (axes 0, 1, 2 of the field, caller's layout); it stages the brick and a
// one-node halo on every side, coordinates clamped into the field (replicate boundary), then
//   A = pass along axis 0 over the staged brick's BZ planes, all halo rows and columns,
//   B = pass along axis 1 of A (into the staging buffer), all halo columns,
//   out = pass along axis 2 of B,
// each value y = w1 x_- + w0 x + w1 x_+ rounded to single precision, as three one-axis passes
// through global memory would compute it.  Nodes of the brick outside the field are computed
// from clamped copies and not stored.
constexpr int kBlurX = 32, kBlurY = 8, kBlurZ = 8;
constexpr int kBlurHX = kBlurX + 2, kBlurHY = kBlurY + 2, kBlurHZ = kBlurZ + 2;
static_assert(kBlurX * kBlurY == kBlock && kBlurX == 32,
              "a warp per brick row, a thread per node of a brick plane");

__global__ void __launch_bounds__(kBlock)
k_blur3(Geo g, const float* __restrict__ in, float* __restrict__ out, float w0, float w1) {
  __shared__ float X[kBlurHZ * kBlurHY * kBlurHX];   // staged brick; later B
  __shared__ float A[kBlurZ * kBlurHY * kBlurHX];
  const int n0 = g.fe[0], n1 = g.fe[1], n2 = g.fe[2];
  const int x0 = blockIdx.x * kBlurX, y0 = blockIdx.y * kBlurY, z0 = blockIdx.z * kBlurZ;
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  constexpr int NR = kBlurHZ * kBlurHY;                        // staged rows of the brick
  constexpr int RW = (NR + kBlock / 32 - 1) / (kBlock / 32);                 // rows per warp
  // stage: warp w loads rows w, w + 8, ... (a row: 32 nodes by the lanes, the 2 right-most by
  // lanes 0 and 1), every load of the thread in flight at once
  const int cx0 = min(max(x0 - 1 + lane, 0), n2 - 1), cx1 = min(x0 + 31 + lane, n2 - 1);
  float v[RW], v2[RW];
#pragma unroll
  for (int u = 0; u < RW; ++u) {
    const int rr = warp + u * (kBlock / 32);
    v[u] = 0.f;
    v2[u] = 0.f;
    if (rr < NR) {
      const int z = rr / kBlurHY, y = rr - z * kBlurHY;
      const int i0 = min(max(z0 - 1 + z, 0), n0 - 1), i1 = min(max(y0 - 1 + y, 0), n1 - 1);
      const float* row = in + ((long long)i0 * n1 + i1) * n2;
      v[u] = __ldg(row + cx0);
      if (lane < 2) v2[u] = __ldg(row + cx1);
    }
  }
#pragma unroll
  for (int u = 0; u < RW; ++u) {
    const int rr = warp + u * (kBlock / 32);
    if (rr < NR) {
      X[rr * kBlurHX + lane] = v[u];
      if (lane < 2) X[rr * kBlurHX + 32 + lane] = v2[u];
    }
  }
  __syncthreads();
  // axis 0: A[z][y][x] from planes z, z + 1, z + 2 of the staged brick
  constexpr int NA = kBlurZ * kBlurHY * kBlurHX, PL = kBlurHY * kBlurHX;
  for (int e = t; e < NA; e += kBlock) {
    const float xm = X[e], xc = X[e + PL], xp = X[e + 2 * PL];
    A[e] = w1 * xm + w0 * xc + w1 * xp;
  }
  __syncthreads();
  // axis 1: B[z][y][x] (y < kBlurY) from rows y, y + 1, y + 2 of A, into X
  constexpr int NB = kBlurZ * kBlurY * kBlurHX;
  for (int e = t; e < NB; e += kBlock) {
    const int z = e / (kBlurY * kBlurHX), r = e - z * (kBlurY * kBlurHX);
    const int a = z * PL + r;   // A[z][y][x] with r = y * kBlurHX + x
    const float xm = A[a], xc = A[a + kBlurHX], xp = A[a + 2 * kBlurHX];
    X[e] = w1 * xm + w0 * xc + w1 * xp;
  }
  __syncthreads();
  // axis 2: thread (tx, ty) writes nodes (z, ty, tx) of the brick, a warp per 32-node row
  const int tx = t % kBlurX, ty = t / kBlurX;
  const int i1 = y0 + ty, i2 = x0 + tx;
  if (i1 >= n1 || i2 >= n2) return;
#pragma unroll
  for (int z = 0; z < kBlurZ; ++z) {
    const int i0 = z0 + z;
    if (i0 >= n0) break;
    const int bidx = (z * kBlurY + ty) * kBlurHX + tx;
    const float xm = X[bidx], xc = X[bidx + 1], xp = X[bidx + 2];
    out[((long long)i0 * n1 + i1) * n2 + i2] = w1 * xm + w0 * xc + w1 * xp;
  }
}

// ------------------------------------------------------------------------------------------

cudaError_t launch_ot_shift(const Geo& g, int dtype, const void* Ip, const void* Im,
                            long long n, double eps, const Work& w, cudaStream_t s) {
  (void)g;
  int blocks = (int)((n + kBlock - 1) / kBlock);
  if (blocks > 148 * 8) blocks = 148 * 8;
  if (dtype == 0)
    k_ot_shift<float><<<blocks, kBlock, 0, s>>>((const float*)Ip, (const float*)Im, n, (float)eps,
                                                w.partials, w.counter, w.st);
  else if (dtype == 1)
    k_ot_shift<__nv_bfloat16><<<blocks, kBlock, 0, s>>>((const __nv_bfloat16*)Ip,
                                                        (const __nv_bfloat16*)Im, n, (float)eps,
                                                        w.partials, w.counter, w.st);
  else
    k_ot_shift<__half><<<blocks, kBlock, 0, s>>>((const __half*)Ip, (const __half*)Im, n,
                                                 (float)eps, w.partials, w.counter, w.st);
  return cudaGetLastError();
}

template <typename T, bool IDX>
static cudaError_t ot_one(const Geo& g, const void* Ip, const void* Im, float* b0, int* kp,
                          int* km, const Work& w, cudaStream_t s) {
  int CW = ot_tile_width(g.E);
  size_t smem = 2ull * g.E * CW * sizeof(float);
  cudaError_t e = cudaFuncSetAttribute(k_ot<T, IDX>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  k_ot<T, IDX><<<ceil_div(g.ncols, CW), dim3(CW, kBlock / CW), smem, s>>>(
      g, (const T*)Ip, (const T*)Im, b0, kp, km, w.st);
  return cudaGetLastError();
}

cudaError_t launch_ot(const Geo& g, int dtype, const void* Ip, const void* Im, float* b0,
                      int* kp, int* km, const Work& w, cudaStream_t s) {
  bool idx = kp != nullptr;
  if (dtype == 0) return idx ? ot_one<float, true>(g, Ip, Im, b0, kp, km, w, s)
                             : ot_one<float, false>(g, Ip, Im, b0, kp, km, w, s);
  if (dtype == 1) return idx ? ot_one<__nv_bfloat16, true>(g, Ip, Im, b0, kp, km, w, s)
                             : ot_one<__nv_bfloat16, false>(g, Ip, Im, b0, kp, km, w, s);
  return idx ? ot_one<__half, true>(g, Ip, Im, b0, kp, km, w, s)
             : ot_one<__half, false>(g, Ip, Im, b0, kp, km, w, s);
}

// the three passes (axis 0, 1, 2) in one launch: in -> out (in is not modified)
cudaError_t launch_blur(const Geo& g, float* in, float* out, cudaStream_t s) {
  double e = std::exp(-0.5);   // the sigma = 1 Gaussian at distance 1 voxel
  float w0 = (float)(1.0 / (1.0 + 2.0 * e)), w1 = (float)(e / (1.0 + 2.0 * e));
  const dim3 grid(ceil_div(g.fe[2], kBlurX), ceil_div(g.fe[1], kBlurY), ceil_div(g.fe[0], kBlurZ));
  if (grid.y > 65535u || grid.z > 65535u) return cudaErrorInvalidConfiguration;
  k_blur3<<<grid, kBlock, 0, s>>>(g, in, out, w0, w1);
  return cudaGetLastError();
}

// ------------------------------------------------------------------------------------------
// Feasible start of the GN loop (the barrier of Eq. 3 is +inf unless |delta| < 1 in every cell;
// b = 0 is feasible): the OT field is halved until max |delta| < 1.  k_start_max: largest
// |b_{j+1} - b_j| over all cells (exact: a maximum), the last block turns it into the factor
// 2^-k; k_start_scale applies it.
// ------------------------------------------------------------------------------------------
__global__ void __launch_bounds__(kBlock)
k_start_max(Geo g, const float* __restrict__ b, float* partials, unsigned* counter,
            DevState* st) {
  __shared__ float wmax[kBlock / 32];
  __shared__ int is_last;
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  const int j0 = blockIdx.y * kSeg, j1 = min(j0 + kSeg, g.m);
  float s = 0.f;
  if (c < g.ncols) {
    const int fb = col_base(c, g.inner, g.fld_ostride);
    for (int j = j0; j < j1; ++j)
      s = fmaxf(s, fabsf(__ldg(b + fb + (j + 1) * g.inner) - __ldg(b + fb + j * g.inner)));
  }
  for (int off = 16; off > 0; off >>= 1) s = fmaxf(s, __shfl_xor_sync(0xffffffffu, s, off));
  if ((threadIdx.x & 31) == 0) wmax[threadIdx.x >> 5] = s;
  __syncthreads();
  const int nblk = gridDim.x * gridDim.y, bid = blockIdx.x + gridDim.x * blockIdx.y;
  if (threadIdx.x == 0) {
    float m = 0.f;
    for (int w = 0; w < kBlock / 32; ++w) m = fmaxf(m, wmax[w]);
    partials[bid] = m;
    __threadfence();
    is_last = atomicAdd(counter, 1u) == (unsigned)(nblk - 1);
  }
  __syncthreads();
  if (!is_last) return;
  __threadfence();
  float m = 0.f;
  for (int i = threadIdx.x; i < nblk; i += blockDim.x) m = fmaxf(m, __ldcg(partials + i));
  for (int off = 16; off > 0; off >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, off));
  __syncthreads();
  if ((threadIdx.x & 31) == 0) wmax[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    float smax = 0.f;
    for (int w = 0; w < kBlock / 32; ++w) smax = fmaxf(smax, wmax[w]);
    float f = 1.f;
    for (int k = 0; k < 64 && smax * f >= 1.f; ++k) f *= 0.5f;
    st->start_scale = f;
    *counter = 0u;
  }
}

__global__ void __launch_bounds__(kBlock)
k_start_scale(int nf, float* __restrict__ b, const DevState* st) {
  const float f = st->start_scale;
  if (f == 1.f) return;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nf; i += gridDim.x * blockDim.x)
    b[i] *= f;
}

cudaError_t launch_feasible_start(const Geo& g, float* b, const Work& w, cudaStream_t s) {
  k_start_max<<<dim3(ceil_div(g.ncols, kBlock), ceil_div(g.m, kSeg)), kBlock, 0, s>>>(
      g, b, w.partials, w.counter, w.st);
  k_start_scale<<<ceil_div(g.nf, kBlock * 4), kBlock, 0, s>>>(g.nf, b, w.st);
  return cudaGetLastError();
}

}  // namespace hysco
