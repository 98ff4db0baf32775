// Least-squares image correction (Sec. 2.4 "Image Correction"): per PE column, the true image I
// minimising |P+ I - I+|^2 + |P- I - I-|^2 + lambda |I|^2, where the push-forward matrix P+-
// spreads the mass of true cell j uniformly over its mapped interval
// [e_j, e_{j+1}] = [j - 1/2 +- b_j, j + 1/2 +- b_{j+1}] and distorted cell i collects the part
// inside [i - 1/2, i + 1/2]: P[i][j] = overlap / (e_{j+1} - e_j).
//
// Row j of the normal matrix N = P+^T P+ + P-^T P- + lambda Id is formed directly: the distorted
// cells i that true cell j's mapped interval overlaps (at most three, |delta| < 1) give
// N_jk += P_ij P_ik for k = j .. j + w (the band of half-width w) and rhs_j += P_ij I[i].  The band
// a column needs grows with its compression (true cells j and j + d share a distorted cell when
// the d - 1 cells between them shrink by more than d - 2 in total).
//
// Pass 0 (half-width kLsBand = 4, |delta| up to about 0.75, almost every column) runs in two
// kernels: k_ls_rows forms every row of every column at once (a thread per row: its band entries
// and right-hand side into the workspace, and the column's flags: a row whose band is too narrow,
// a cell with |delta| >= 1), then k_ls_solve walks each column once (a thread per column) through
// the banded LDL^T factorisation with the forward substitution L y = rhs fused in (the last four
// columns of L and D in registers, the workspace's rows loaded eight ahead) and the back
// substitution L^T x = D^{-1} y into the output; a column with |delta| >= 1 is set to 0 and
// counted.  Columns whose band was too narrow are redone by pass 1 (k_ls_correct, half-width 16,
// |delta| up to about 0.94: one thread per column forming and factoring its rows as it goes);
// a column wider still is set to 0 and counted.
#include "eval_common.cuh"

namespace hysco {

constexpr int kLsColBlock = 64;

// |[i - 1/2, i + 1/2] ∩ [e0, e1]|
__device__ __forceinline__ float overlap(int i, float e0, float e1) {
  return fmaxf(0.f, fminf(e1, (float)i + 0.5f) - fmaxf(e0, (float)i - 0.5f));
}

// Pass 1: the columns pass 0 flagged narrow (wide[c] == 1) only, half-width BAND, a thread per
// column forming each row as it factors it.  STAGED: the block's two image columns are first
// copied to shared memory (rows of kLsColBlock consecutive columns, coalesced), so the per-row
// gathers of the sequential factorisation are shared loads.
template <typename TI, int BAND, bool STAGED>
__global__ void __launch_bounds__(kLsColBlock)
k_ls_correct(Geo g, const TI* __restrict__ Ip, const TI* __restrict__ Im,
             const float* __restrict__ b, float lambda, float* __restrict__ band,
             long long bstride, float* __restrict__ rhs, float* __restrict__ out,
             int* __restrict__ nbad, int* __restrict__ wide) {
  constexpr int kLsBand = BAND;
  extern __shared__ float simg[];   // STAGED: [2][m][kLsColBlock]
  const int c0 = blockIdx.x * blockDim.x, tid = threadIdx.x;
  const int c = c0 + tid;
  bool live = c < g.ncols && wide[c] == 1;
  if (!__syncthreads_or(live)) return;   // no flagged column in this block
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
  bool ok = true;
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
    if (!(fabsf(bw[1] - bw[0]) < 1.0f)) ok = false;
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
  if (!ok) {   // a cell with |delta| >= 1, or a band still too narrow: set to 0, counted
    for (int j = 0; j < m; ++j) out[ib + j * inner] = 0.f;
    atomicAdd(nbad, 1);
    return;
  }
  // ---- L^T x = D^{-1} y (rows of L and D^{-1} y loaded ahead of the recurrence) --------------
  constexpr int kAhead = 2;
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

// Pass 0, step 1: row j of column c (thread j * ncols + c, so a warp's rows are one row of 32
// consecutive columns): the band entries N[j][j + d], d = 0 .. kLsBand, into ws[d], the
// right-hand side into ws[kLsBand + 1] (each array image-shaped), and the column's flags
// (bit 0: this row's band is too narrow, bit 1: cell j has |delta| >= 1).
template <typename TI>
__global__ void __launch_bounds__(kBlock)
k_ls_rows(Geo g, const TI* __restrict__ Ip, const TI* __restrict__ Im,
          const float* __restrict__ b, float lambda, float* __restrict__ ws, long long wstride,
          int* __restrict__ flag, FastDiv ncols_div) {
  constexpr int W = kLsBand;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;   // < m * ncols < 2^31
  if (t >= g.m * g.ncols) return;
  const int j = (int)fdiv((unsigned)t, ncols_div), c = t - j * g.ncols;
  const int inner = g.inner, m = g.m;
  const int o = (int)fdiv((unsigned)c, g.divIn), ci = c - o * inner;
  const int ib = o * (int)g.img_ostride + ci, fb = o * (int)g.fld_ostride + ci;
  // b at nodes j .. j + W + 1 (node m past the column's end) and the reciprocal lengths
  // 1 / (e_{u+1} - e_u) of the mapped cells j .. j + W for both directions
  float bw[W + 2], ilp[W + 1], ilm[W + 1];
#pragma unroll
  for (int u = 0; u < W + 2; ++u) bw[u] = __ldg(b + fb + min(j + u, m) * inner);
#pragma unroll
  for (int u = 0; u <= W; ++u) {
    ilp[u] = __frcp_rn(1.0f + (bw[u + 1] - bw[u]));   // = 1.0f / x, correctly rounded
    ilm[u] = __frcp_rn(1.0f - (bw[u + 1] - bw[u]));
  }
  int fl = fabsf(bw[1] - bw[0]) < 1.0f ? 0 : 2;
  float N[W + 1], r = 0.f;
#pragma unroll
  for (int d = 0; d <= W; ++d) N[d] = d == 0 ? lambda : 0.f;
#pragma unroll
  for (int s = 0; s < 2; ++s) {
    const float sg = s == 0 ? 1.0f : -1.0f;
    float e[W + 2];   // mapped edges of cells j .. j + W
#pragma unroll
    for (int u = 0; u < W + 2; ++u) e[u] = (float)(j + u) - 0.5f + sg * bw[u];
    const float* il = s == 0 ? ilp : ilm;
    const int ilo = max((int)floorf(e[0] + 0.5f), 0), ihi = min((int)floorf(e[1] + 0.5f), m - 1);
    // cells past j + W must not reach the last distorted cell of this row
    if (j + W + 1 < m && (float)ihi + 0.5f > e[W + 1]) fl |= 1;
    const TI* img = (s == 0 ? Ip : Im) + ib;
    for (int i = ilo; i <= ihi; ++i) {
      const float pij = overlap(i, e[0], e[1]) * il[0];
      r += pij * ldf(img + i * inner);
#pragma unroll
      for (int d = 0; d <= W; ++d)
        if (j + d < m) N[d] += pij * overlap(i, e[d], e[d + 1]) * il[d];
    }
  }
  if (fl) atomicOr(flag + c, fl);
  const int oj = ib + j * inner;
#pragma unroll
  for (int d = 0; d <= W; ++d) ws[d * wstride + oj] = N[d];
  ws[(W + 1) * wstride + oj] = r;
}

constexpr int kLsRing = 16;   // workspace rows a column's thread has in flight (shared ring)

// Pass 0, step 2: column c (a thread each, 32 per block): the banded LDL^T of N with L y = rhs
// fused (the last kLsBand columns of L and D in registers), L and D^-1 y written over the rows'
// workspace, then L^T x = D^-1 y into out.  The rows a step reads arrive kLsRing - 1 steps ahead
// through a shared-memory ring (cp.async: each thread its own words), so the sequential
// recurrence never waits on memory.  A column flagged narrow is left to pass 1; one with a cell
// of |delta| >= 1 is set to 0 and counted.
__global__ void __launch_bounds__(32)
k_ls_solve(Geo g, float* __restrict__ ws, long long wstride, const int* __restrict__ flag,
           float* __restrict__ out, int* __restrict__ nbad) {
  constexpr int W = kLsBand, R = kLsRing;
  __shared__ float ring[R][W + 2][32];
  const int lane = threadIdx.x, c = blockIdx.x * blockDim.x + lane;
  if (c >= g.ncols) return;
  const int f = flag[c], inner = g.inner, m = g.m;
  const int ib = col_base(c, inner, g.img_ostride);
  if (f & 2) {
    for (int j = 0; j < m; ++j) out[ib + j * inner] = 0.f;
    atomicAdd(nbad, 1);
    return;
  }
  if (f) return;
  auto at = [&](int k, int j) -> float* { return ws + k * wstride + ib + j * inner; };
  // ---- N = L D L^T with L y = rhs ---------------------------------------------------------------
  // row j (clamped to the column) into ring slot j % R: N[j][j + d] (d <= W) and rhs_j
  auto fetch_row = [&](int j) {
    const int jj = min(j, m - 1), sl = j % R;
#pragma unroll
    for (int k = 0; k < W + 2; ++k) cp_async4(&ring[sl][k][lane], at(k, jj), true);
    cp_async_commit();
  };
  float Lw[W][W], Dw[W], yw[W];
#pragma unroll
  for (int t = 0; t < W; ++t) {
    Dw[t] = 1.f;
    yw[t] = 0.f;
#pragma unroll
    for (int d = 0; d < W; ++d) Lw[t][d] = 0.f;
  }
  for (int u = 0; u < R - 1; ++u) fetch_row(u);
#pragma unroll 2
  for (int j = 0; j < m; ++j) {
    fetch_row(j + R - 1);
    cp_async_wait<R - 1>();   // row j has landed
    const int sl = j % R;
    float N[W + 1];
#pragma unroll
    for (int d = 0; d <= W; ++d) N[d] = ring[sl][d][lane];
    const float r = ring[sl][W + 1][lane];
    float dj = N[0], yj = r;
#pragma unroll
    for (int t = 0; t < W; ++t) {
      const float ljk = Lw[t][t];   // L[j][k], k = j - 1 - t
      dj -= ljk * ljk * Dw[t];
      yj -= ljk * yw[t];
    }
    const float idj = __frcp_rn(dj);   // = 1.0f / dj, correctly rounded
    float Lnew[W];
#pragma unroll
    for (int d = 0; d < W; ++d) {
      float a = N[d + 1];   // N[j+1+d][j]
#pragma unroll
      for (int t = 0; t + d + 1 < W; ++t) a -= Lw[t][t + d + 1] * Lw[t][t] * Dw[t];
      Lnew[d] = j + 1 + d < m ? a * idj : 0.f;
    }
#pragma unroll
    for (int t = W - 1; t > 0; --t) {
      Dw[t] = Dw[t - 1];
      yw[t] = yw[t - 1];
#pragma unroll
      for (int d = 0; d < W; ++d) Lw[t][d] = Lw[t - 1][d];
    }
    Dw[0] = dj;
    yw[0] = yj;
#pragma unroll
    for (int d = 0; d < W; ++d) {
      Lw[0][d] = Lnew[d];
      *at(d, j) = Lnew[d];
    }
    *at(W + 1, j) = yj * idj;
  }
  cp_async_wait<0>();
  __threadfence_block();   // this thread's L and D^-1 y stores before its copies read them back
  // ---- L^T x = D^-1 y, rows m - 1 .. 0 ----------------------------------------------------------
  auto fetch_back = [&](int j) {   // row m - 1 - j: L[.][d] (d < W) and D^-1 y
    const int jj = max(m - 1 - j, 0), sl = j % R;
#pragma unroll
    for (int d = 0; d < W; ++d) cp_async4(&ring[sl][d][lane], at(d, jj), true);
    cp_async4(&ring[sl][W][lane], at(W + 1, jj), true);
    cp_async_commit();
  };
  float xw[W];
#pragma unroll
  for (int t = 0; t < W; ++t) xw[t] = 0.f;   // x_{j+1+t}
  for (int u = 0; u < R - 1; ++u) fetch_back(u);
  for (int k = 0; k < m; ++k) {
    fetch_back(k + R - 1);
    cp_async_wait<R - 1>();
    const int sl = k % R, j = m - 1 - k;
    float x = ring[sl][W][lane];
#pragma unroll
    for (int d = 0; d < W; ++d) x -= ring[sl][d][lane] * xw[d];
#pragma unroll
    for (int t = W - 1; t > 0; --t) xw[t] = xw[t - 1];
    xw[0] = x;
    out[ib + j * inner] = x;
  }
  cp_async_wait<0>();
}

cudaError_t launch_ls_correct(const Geo& g, int dtype, const void* Ip, const void* Im,
                              const float* b, float lambda, float* band, long long bstride,
                              float* rhs, float* out, int* nbad, int* wide, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(wide, 0, sizeof(int) * (size_t)g.ncols, s);
  if (e != cudaSuccess) return e;
  // pass 1 stages the images in shared memory when a block's two image columns fit
  const size_t smem = 2ull * g.m * kLsColBlock * sizeof(float);
  const bool staged = smem <= 160 * 1024;
  const dim3 grid1(ceil_div(g.ncols, kLsColBlock));
  const long long rows = (long long)g.m * g.ncols;
  const dim3 grid0((unsigned)((rows + kBlock - 1) / kBlock));
  auto run = [&](auto tag) -> cudaError_t {
    using T = decltype(tag);
    k_ls_rows<T><<<grid0, kBlock, 0, s>>>(g, (const T*)Ip, (const T*)Im, b, lambda, band, bstride,
                                          wide, make_fastdiv((unsigned)g.ncols));
    k_ls_solve<<<ceil_div(g.ncols, 32), 32, 0, s>>>(g, band, bstride, wide, out, nbad);
    if (staged) {
      if (cudaError_t ea = cudaFuncSetAttribute(k_ls_correct<T, kLsBandWide, true>,
                                                cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                (int)smem))
        return ea;
      k_ls_correct<T, kLsBandWide, true><<<grid1, kLsColBlock, smem, s>>>(
          g, (const T*)Ip, (const T*)Im, b, lambda, band, bstride, rhs, out, nbad, wide);
    } else {
      k_ls_correct<T, kLsBandWide, false><<<grid1, kLsColBlock, 0, s>>>(
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
