// Least-squares image correction (Sec. 2.4 "Image Correction"): per PE column, the true image I
// minimising |P+ I - I+|^2 + |P- I - I-|^2 + lambda |I|^2, where the push-forward matrix P+-
// spreads the mass of true cell j uniformly over its mapped interval
// [e_j, e_{j+1}] = [j - 1/2 +- b_j, j + 1/2 +- b_{j+1}] and distorted cell i collects the part
// inside [i - 1/2, i + 1/2]: P[i][j] = overlap / (e_{j+1} - e_j).
//
// One thread per column, streaming along it.  Row j of the normal matrix
// N = P+^T P+ + P-^T P- + lambda Id is formed directly: the distorted cells i that true cell j's
// mapped interval overlaps (at most three, |delta| < 1) give N_jk += P_ij P_ik for k = j .. j + 4
// (the band; edges kept in a rolling register window) and rhs_j += P_ij I[i].  Each row goes
// straight into one step of a banded LDL^T factorisation with the forward substitution L y = rhs
// fused in (the last four columns of L and D in registers); L and D^{-1} y go to scratch for the
// back substitution L^T x = D^{-1} y into the output.  A column whose field has |delta| >= 1 is
// set to 0 and counted.  The band a column needs grows with its compression (true cells j and
// j + d share a distorted cell when the d - 1 cells between them shrink by more than d - 2 in
// total): a first pass with half-width 4 (|delta| up to about 0.75) serves most columns and flags
// the others, which a second pass with half-width 16 (|delta| up to about 0.94) redoes; a column
// wider still is set to 0 and counted.
#include "eval_common.cuh"

namespace hysco {

constexpr int kLsColBlock = 64;

// |[i - 1/2, i + 1/2] ∩ [e0, e1]|
__device__ __forceinline__ float overlap(int i, float e0, float e1) {
  return fmaxf(0.f, fminf(e1, (float)i + 0.5f) - fmaxf(e0, (float)i - 0.5f));
}

// PASS 0: every column, half-width kLsBand, columns whose band is too narrow flagged in `wide`
// (their output left to pass 1).  PASS 1: the flagged columns only, half-width BAND.  STAGED: the
// block's two image columns are first copied to shared memory (rows of kLsColBlock consecutive
// columns, coalesced), so the per-row gathers of the sequential factorisation are shared loads.
template <typename TI, int BAND, int PASS, bool STAGED>
__global__ void __launch_bounds__(kLsColBlock)
k_ls_correct(Geo g, const TI* __restrict__ Ip, const TI* __restrict__ Im,
             const float* __restrict__ b, float lambda, float* __restrict__ band,
             long long bstride, float* __restrict__ rhs, float* __restrict__ out,
             int* __restrict__ nbad, int* __restrict__ wide) {
  constexpr int kLsBand = BAND;
  extern __shared__ float simg[];   // STAGED: [2][m][kLsColBlock]
  const int c0 = blockIdx.x * blockDim.x, tid = threadIdx.x;
  const int c = c0 + tid;
  bool live = c < g.ncols && (PASS == 0 || wide[c]);
  if (PASS == 1 && !__syncthreads_or(live)) return;   // no flagged column in this block
  const int inner = g.inner, m = g.m;
  if (STAGED) {
    // row i of both images for the block's columns (a lane per column; absent columns read 0)
    const int nw = blockDim.x >> 5, lane = tid & 31, w = tid >> 5;
    for (int s = 0; s < 2; ++s) {
      const TI* img = s == 0 ? Ip : Im;
      float* dst = simg + (size_t)s * m * kLsColBlock;
      for (int cc = lane; cc < kLsColBlock; cc += 32) {
        const int col = c0 + cc;
        const int cb = col < g.ncols ? col_base(col, inner, g.img_ostride) : 0;
        for (int i = w; i < m; i += nw)
          dst[i * kLsColBlock + cc] = col < g.ncols ? ldf(img + cb + i * inner) : 0.f;
      }
    }
    __syncthreads();
  }
  if (!live) return;
  const int ib = col_base(c, inner, g.img_ostride), fb = col_base(c, inner, g.fld_ostride);
  auto Lst = [&](int d, int j) -> float& { return band[d * bstride + ib + j * inner]; };   // L[j+1+d][j]
  auto Z = [&](int j) -> float& { return rhs[ib + j * inner]; };                 // D^-1 y
  bool ok = true, narrow = false;
  // rolling field window: bw[u] = b at node j + u, u = 0 .. kLsBand + 1; and the reciprocal
  // lengths 1 / (e_{j+u+1} - e_{j+u}) of the mapped cells for both directions
  float bw[kLsBand + 2], ilp[kLsBand + 1], ilm[kLsBand + 1];
#pragma unroll
  for (int u = 0; u < kLsBand + 2; ++u) bw[u] = __ldg(b + fb + min(u, m) * inner);
#pragma unroll
  for (int u = 0; u <= kLsBand; ++u) {
    ilp[u] = 1.0f / (1.0f + (bw[u + 1] - bw[u]));
    ilm[u] = 1.0f / (1.0f - (bw[u + 1] - bw[u]));
  }
  float Lw[kLsBand][kLsBand], Dw[kLsBand], yw[kLsBand];
#pragma unroll
  for (int t = 0; t < kLsBand; ++t) {
    Dw[t] = 1.f;
    yw[t] = 0.f;
#pragma unroll
    for (int d = 0; d < kLsBand; ++d) Lw[t][d] = 0.f;
  }
  for (int j = 0; j < m && ok; ++j) {
    // ---- row j of N and rhs_j -----------------------------------------------------------------
    float N[kLsBand + 1], r = 0.f;
#pragma unroll
    for (int d = 0; d <= kLsBand; ++d) N[d] = d == 0 ? lambda : 0.f;
    if (!(fabsf(bw[1] - bw[0]) < 1.0f)) { ok = false; narrow = false; }
#pragma unroll
    for (int s = 0; s < 2; ++s) {
      const float sg = s == 0 ? 1.0f : -1.0f;
      float e[kLsBand + 2];   // mapped edges of cells j .. j + kLsBand
#pragma unroll
      for (int u = 0; u < kLsBand + 2; ++u) e[u] = (float)(j + u) - 0.5f + sg * bw[u];
      const float* il = s == 0 ? ilp : ilm;
      const int ilo = max((int)floorf(e[0] + 0.5f), 0), ihi = min((int)floorf(e[1] + 0.5f), m - 1);
      // cells past j + kLsBand must not reach the last distorted cell of this row
      if (ok && j + kLsBand + 1 < m && (float)ihi + 0.5f > e[kLsBand + 1]) {
        ok = false;
        narrow = true;
      }
      const TI* img = (s == 0 ? Ip : Im) + ib;
      const float* simgc = simg + (size_t)s * m * kLsColBlock + tid;
      for (int i = ilo; i <= ihi; ++i) {
        const float pij = overlap(i, e[0], e[1]) * il[0];
        r += pij * (STAGED ? simgc[i * kLsColBlock] : ldf(img + i * inner));
#pragma unroll
        for (int d = 0; d <= kLsBand; ++d)
          if (j + d < m) N[d] += pij * overlap(i, e[d], e[d + 1]) * il[d];
      }
    }
    // ---- one step of N = L D L^T with L y = rhs -------------------------------------------------
    float dj = N[0], yj = r;
#pragma unroll
    for (int t = 0; t < kLsBand; ++t) {
      const float ljk = Lw[t][t];   // L[j][k], k = j - 1 - t
      dj -= ljk * ljk * Dw[t];
      yj -= ljk * yw[t];
    }
    const float idj = 1.0f / dj;
    float Lnew[kLsBand];
#pragma unroll
    for (int d = 0; d < kLsBand; ++d) {
      float a = N[d + 1];   // N[j+1+d][j]
#pragma unroll
      for (int t = 0; t + d + 1 < kLsBand; ++t) a -= Lw[t][t + d + 1] * Lw[t][t] * Dw[t];
      Lnew[d] = j + 1 + d < m ? a * idj : 0.f;
    }
#pragma unroll
    for (int t = kLsBand - 1; t > 0; --t) {
      Dw[t] = Dw[t - 1];
      yw[t] = yw[t - 1];
#pragma unroll
      for (int d = 0; d < kLsBand; ++d) Lw[t][d] = Lw[t - 1][d];
    }
    Dw[0] = dj;
    yw[0] = yj;
#pragma unroll
    for (int d = 0; d < kLsBand; ++d) {
      Lw[0][d] = Lnew[d];
      Lst(d, j) = Lnew[d];
    }
    Z(j) = yj * idj;
    // advance the field window
#pragma unroll
    for (int u = 0; u < kLsBand + 1; ++u) bw[u] = bw[u + 1];
    bw[kLsBand + 1] = __ldg(b + fb + min(j + kLsBand + 2, m) * inner);
#pragma unroll
    for (int u = 0; u < kLsBand; ++u) { ilp[u] = ilp[u + 1]; ilm[u] = ilm[u + 1]; }
    ilp[kLsBand] = 1.0f / (1.0f + (bw[kLsBand + 1] - bw[kLsBand]));
    ilm[kLsBand] = 1.0f / (1.0f - (bw[kLsBand + 1] - bw[kLsBand]));
  }
  if (!ok) {
    // a band too narrow in pass 0 (the field itself feasible so far): pass 1 redoes the column
    // (an infeasible cell further on is found there); otherwise the column is set to 0, counted
    if (PASS == 0 && narrow) {
      wide[c] = 1;
      return;
    }
    for (int j = 0; j < m; ++j) out[ib + j * inner] = 0.f;
    atomicAdd(nbad, 1);
    return;
  }
  // ---- L^T x = D^{-1} y (rows of L and D^{-1} y loaded ahead of the recurrence) --------------
  constexpr int kAhead = BAND <= 4 ? 8 : 2;
  float xw[kLsBand];
#pragma unroll
  for (int t = 0; t < kLsBand; ++t) xw[t] = 0.f;   // x_{j+1+t}
  for (int j1 = m - 1; j1 >= 0; j1 -= kAhead) {
    float zv[kAhead], lv[kAhead][kLsBand];
#pragma unroll
    for (int u = 0; u < kAhead; ++u) {
      const int j = max(j1 - u, 0);
      zv[u] = Z(j);
#pragma unroll
      for (int d = 0; d < kLsBand; ++d) lv[u][d] = Lst(d, j);
    }
#pragma unroll
    for (int u = 0; u < kAhead; ++u) {
      if (j1 - u < 0) break;
      float x = zv[u];
#pragma unroll
      for (int d = 0; d < kLsBand; ++d) x -= lv[u][d] * xw[d];
#pragma unroll
      for (int t = kLsBand - 1; t > 0; --t) xw[t] = xw[t - 1];
      xw[0] = x;
      out[ib + (j1 - u) * inner] = x;
    }
  }
}

cudaError_t launch_ls_correct(const Geo& g, int dtype, const void* Ip, const void* Im,
                              const float* b, float lambda, float* band, long long bstride,
                              float* rhs, float* out, int* nbad, int* wide, cudaStream_t s) {
  const dim3 grid(ceil_div(g.ncols, kLsColBlock));
  cudaError_t e = cudaMemsetAsync(wide, 0, sizeof(int) * (size_t)g.ncols, s);
  if (e != cudaSuccess) return e;
  // stage the images in shared memory when a block's two image columns fit
  const size_t smem = 2ull * g.m * kLsColBlock * sizeof(float);
  const bool staged = smem <= 160 * 1024;
  auto run = [&](auto tag) -> cudaError_t {
    using T = decltype(tag);
    if (staged) {
      for (const void* f : {(const void*)k_ls_correct<T, kLsBand, 0, true>,
                            (const void*)k_ls_correct<T, kLsBandWide, 1, true>})
        if (cudaError_t ea = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                  (int)smem))
          return ea;
      k_ls_correct<T, kLsBand, 0, true><<<grid, kLsColBlock, smem, s>>>(
          g, (const T*)Ip, (const T*)Im, b, lambda, band, bstride, rhs, out, nbad, wide);
      k_ls_correct<T, kLsBandWide, 1, true><<<grid, kLsColBlock, smem, s>>>(
          g, (const T*)Ip, (const T*)Im, b, lambda, band, bstride, rhs, out, nbad, wide);
    } else {
      k_ls_correct<T, kLsBand, 0, false><<<grid, kLsColBlock, 0, s>>>(
          g, (const T*)Ip, (const T*)Im, b, lambda, band, bstride, rhs, out, nbad, wide);
      k_ls_correct<T, kLsBandWide, 1, false><<<grid, kLsColBlock, 0, s>>>(
          g, (const T*)Ip, (const T*)Im, b, lambda, band, bstride, rhs, out, nbad, wide);
    }
    return cudaGetLastError();
  };
  switch (dtype) {
    case 0: return run(float{});
    case 1: return run(__nv_bfloat16{});
    default: return run(__half{});
  }
}

}  // namespace hysco
