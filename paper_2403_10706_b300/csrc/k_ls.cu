// Least-squares image correction (Sec. 2.4 "Image Correction"): per PE column, the true image I
// minimising |P+ I - I+|^2 + |P- I - I-|^2 + lambda |I|^2, where the push-forward matrix P+-
// spreads the mass of true cell j uniformly over its mapped interval
// [e_j, e_{j+1}] = [j - 1/2 +- b_j, j + 1/2 +- b_{j+1}] and distorted cell i collects the part
// inside [i - 1/2, i + 1/2]: P[i][j] = overlap / (e_{j+1} - e_j).
//
// One thread per column.  (1) Assembly of the normal equations N I = rhs with
// N = P+^T P+ + P-^T P- + lambda Id: the mapped edges increase with j (|delta| < 1), so a
// two-pointer march over distorted cells finds, for each, the contiguous run of true cells it
// overlaps; every pair in a run adds P_ij P_ik to the band of N (half-width kLsBand) and P_ij I[i]
// to rhs_j.  Band and rhs live in scratch arrays in the image layout.  (2) Banded LDL^T
// factorisation with the forward substitution L y = rhs fused in, the last kLsBand columns of L
// and D kept in registers; L, D^{-1} y written back to scratch.  (3) Back substitution
// L^T x = D^{-1} y into the output.  A column whose field has |delta| >= 1, or whose band would be
// wider than kLsBand (|delta| above about 0.75), is set to 0 and counted.
#include "eval_common.cuh"

namespace hysco {

constexpr int kLsColBlock = 64;

template <typename TI>
__global__ void __launch_bounds__(kLsColBlock)
k_ls_correct(Geo g, const TI* __restrict__ Ip, const TI* __restrict__ Im,
             const float* __restrict__ b, float lambda, LsBand band, float* __restrict__ rhs,
             float* __restrict__ out, int* __restrict__ nbad) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= g.ncols) return;
  const int inner = g.inner, m = g.m;
  const int ib = col_base(c, inner, g.img_ostride), fb = col_base(c, inner, g.fld_ostride);
  auto B = [&](int d, int j) -> float& { return band.d[d][ib + j * inner]; };
  auto R = [&](int j) -> float& { return rhs[ib + j * inner]; };
  bool ok = true;
  for (int j = 0; j < m; ++j) {
    if (!(fabsf(__ldg(b + fb + (j + 1) * inner) - __ldg(b + fb + j * inner)) < 1.0f)) ok = false;
#pragma unroll
    for (int d = 0; d <= kLsBand; ++d) B(d, j) = d == 0 ? lambda : 0.f;
    R(j) = 0.f;
  }
  // ---- (1) assembly ---------------------------------------------------------------------------
  for (int s = 0; s < 2 && ok; ++s) {
    const float sg = s == 0 ? 1.0f : -1.0f;
    const TI* img = (s == 0 ? Ip : Im) + ib;
    auto edge = [&](int j) { return (float)j - 0.5f + sg * __ldg(b + fb + j * inner); };
    int j0 = 0;
    for (int i = 0; i < m && ok; ++i) {
      const float lo = (float)i - 0.5f, hi = (float)i + 0.5f;
      while (j0 < m && edge(j0 + 1) <= lo) ++j0;
      int js[kLsBand + 1];
      float ps[kLsBand + 1];
      int n = 0;
      for (int j = j0; j < m; ++j) {
        const float e0 = edge(j), e1 = edge(j + 1);
        if (!(e0 < hi)) break;
        const float ov = fminf(e1, hi) - fmaxf(e0, lo);
        if (ov > 0.f) {
          if (n > kLsBand) { ok = false; break; }
          js[n] = j;
          ps[n] = ov / (e1 - e0);
          ++n;
        }
      }
      if (!ok) break;
      const float y = ldf(img + i * inner);
      for (int a = 0; a < n; ++a) {
        R(js[a]) += ps[a] * y;
        for (int q = a; q < n; ++q) B(js[q] - js[a], js[a]) += ps[a] * ps[q];
      }
    }
  }
  if (!ok) {
    for (int j = 0; j < m; ++j) out[ib + j * inner] = 0.f;
    atomicAdd(nbad, 1);
    return;
  }
  // ---- (2) N = L D L^T, L y = rhs --------------------------------------------------------------
  // window: column k = j - 1 - t (t = 0..kLsBand-1) of L below the diagonal (Lw[t][d] = L[k+1+d][k])
  // and D_k, y_k
  float Lw[kLsBand][kLsBand], Dw[kLsBand], yw[kLsBand];
#pragma unroll
  for (int t = 0; t < kLsBand; ++t) {
    Dw[t] = 1.f;
    yw[t] = 0.f;
#pragma unroll
    for (int d = 0; d < kLsBand; ++d) Lw[t][d] = 0.f;
  }
  for (int j = 0; j < m; ++j) {
    // D_j = N_jj - sum_k L[j][k]^2 D_k,  L[j][k] = Lw[j-1-k][j-1-k] for k = j-1-t
    float dj = B(0, j), yj = R(j);
#pragma unroll
    for (int t = 0; t < kLsBand; ++t) {
      const float ljk = Lw[t][t];   // L[j][k] with k = j - 1 - t (offset j - k - 1 = t)
      dj -= ljk * ljk * Dw[t];
      yj -= ljk * yw[t];
    }
    float Lnew[kLsBand];
#pragma unroll
    for (int d = 0; d < kLsBand; ++d) {
      // L[j+1+d][j] = (N[j+1+d][j] - sum_k L[j+1+d][k] L[j][k] D_k) / D_j
      float a = j + 1 + d < m ? B(d + 1, j) : 0.f;
#pragma unroll
      for (int t = 0; t + d + 1 < kLsBand; ++t)
        a -= Lw[t][t + d + 1] * Lw[t][t] * Dw[t];   // L[j+1+d][k] at offset (j+1+d) - k - 1
      Lnew[d] = j + 1 + d < m ? a / dj : 0.f;
    }
    // shift the window and store column j (L below the diagonal, and D_j^{-1} y_j)
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
      B(d + 1, j) = Lnew[d];
    }
    R(j) = yj / dj;
  }
  // ---- (3) L^T x = D^{-1} y ---------------------------------------------------------------------
  float xw[kLsBand];
#pragma unroll
  for (int t = 0; t < kLsBand; ++t) xw[t] = 0.f;   // x_{j+1+t}
  for (int j = m - 1; j >= 0; --j) {
    float x = R(j);
#pragma unroll
    for (int d = 0; d < kLsBand; ++d) x -= B(d + 1, j) * xw[d];
#pragma unroll
    for (int t = kLsBand - 1; t > 0; --t) xw[t] = xw[t - 1];
    xw[0] = x;
    out[ib + j * inner] = x;
  }
}

cudaError_t launch_ls_correct(const Geo& g, int dtype, const void* Ip, const void* Im,
                              const float* b, float lambda, LsBand band, float* rhs, float* out,
                              int* nbad, cudaStream_t s) {
  const dim3 grid(ceil_div(g.ncols, kLsColBlock));
  switch (dtype) {
    case 0:
      k_ls_correct<float><<<grid, kLsColBlock, 0, s>>>(g, (const float*)Ip, (const float*)Im, b,
                                                      lambda, band, rhs, out, nbad);
      break;
    case 1:
      k_ls_correct<__nv_bfloat16><<<grid, kLsColBlock, 0, s>>>(
          g, (const __nv_bfloat16*)Ip, (const __nv_bfloat16*)Im, b, lambda, band, rhs, out,
          nbad);
      break;
    default:
      k_ls_correct<__half><<<grid, kLsColBlock, 0, s>>>(g, (const __half*)Ip, (const __half*)Im,
                                                       b, lambda, band, rhs, out, nbad);
      break;
  }
  return cudaGetLastError();
}

}  // namespace hysco
