// Objective kernels: J(b) = D + alpha S + beta P with gradient and Gauss-Newton coefficients
// (Sec. 2.1 Eq. 1-5, Sec. 2.3.1), the multi-trial Armijo line search, the GN update, the
// corrected images (Sec. 2.4) and the interpolation cell indices.
//
// Thread mapping ("column march"): thread = (PE column c, segment of `seg` nodes along PE).
// Consecutive threads own consecutive columns, so for pe_dim != 2 every PE step is a coalesced
// row access.  A thread walks its segment keeping the two field nodes of the current cell and the
// previous cell's residual row in registers; in-plane Laplacian neighbours are read through L1.
// Per cell j (nodes j, j+1):
//   bc = (b_j + b_{j+1}) / 2, delta = b_{j+1} - b_j, t+- = j +- bc      (averaging / FD operators)
//   I(t) = I[i] + w (I[i+1] - I[i]), i = floor(t), w = t - i, I = 0 outside 0..m-1
//   T+ = I+(t+)(1 + delta), T- = I-(t-)(1 - delta), r = T+ - T-         (Eq. 1)
//   a = I+'(1 + delta) + I-'(1 - delta), c = I+(t+) + I-(t-);  dr/db_j = a/2 - c, dr/db_{j+1} = a/2 + c
// Per node k the Gauss-Newton Hessian restricted to the column is tridiagonal:
//   d_k = (dr_{k-1}/db_k)^2 + (dr_k/db_k)^2 + psi_{k-1} + psi_k,   e_k = dr_k/db_k * dr_k/db_{k+1} - psi_k
// with psi = beta/2 phi''(delta); H v = vol [e_{k-1} v_{k-1} + d_k v_k + e_k v_{k+1} + alpha (L v)_k].
#include "hysco_internal.cuh"

namespace hysco {

// positions of cell j: single-precision, no contraction (bit-reproducible cell indices)
__device__ __forceinline__ void cell_positions(float bj, float bj1, int j, float& tp, float& tm) {
  float bc = __fmul_rn(__fadd_rn(bj, bj1), 0.5f);
  float jf = (float)j;
  tp = __fadd_rn(jf, bc);
  tm = __fsub_rn(jf, bc);
}

// floor(t) clamped to [-2, m + 1] (zero interpolation beyond), and the exact weight t - floor(t)
__device__ __forceinline__ int cell_index(float t, int m, float& w) {
  float f = floorf(t);
  w = __fsub_rn(t, f);
  f = fminf(fmaxf(f, -2.0f), (float)(m + 1));
  return (int)f;
}

template <typename TI>
__device__ __forceinline__ void interp(const TI* col, int inner, int m, int i, float w,
                                       float& val, float& slope) {
  float I0 = (i >= 0 && i < m) ? ldf(col + (long long)i * inner) : 0.0f;
  float I1 = (i >= -1 && i + 1 < m) ? ldf(col + (long long)(i + 1) * inner) : 0.0f;
  slope = I1 - I0;
  val = fmaf(w, slope, I0);
}

// phi(z) = z^4 / (1 - z^2) on (-1, 1), +inf outside (Eq. 3), and its first two derivatives
__device__ __forceinline__ void barrier(float z, float& f, float& df, float& d2f) {
  if (!(fabsf(z) < 1.0f)) {
    f = (z != z) ? z : __int_as_float(0x7f800000);
    df = 0.0f;
    d2f = 0.0f;
    return;
  }
  float z2 = z * z;
  float q = (1.0f - z) * (1.0f + z);
  float iq = 1.0f / q;
  float z4 = z2 * z2;
  f = z4 * iq;
  df = (4.0f * z2 * z - 2.0f * z4 * z) * (iq * iq);
  d2f = (12.0f * z2 - 6.0f * z4 + 2.0f * z4 * z2) * (iq * iq * iq);
}

struct CellLin {
  float r, jl, jr, dphi, psi, phi;
};

template <typename TI>
__device__ __forceinline__ CellLin cell_lin(const TI* Ipc, const TI* Imc, int inner, int m, int j,
                                            float bj, float bj1, float half_beta) {
  float tp, tm, wp, wm;
  cell_positions(bj, bj1, j, tp, tm);
  int ip = cell_index(tp, m, wp), im = cell_index(tm, m, wm);
  float vp, sp, vm, sm;
  interp(Ipc, inner, m, ip, wp, vp, sp);
  interp(Imc, inner, m, im, wm, vm, sm);
  float delta = bj1 - bj;
  float op = 1.0f + delta, om = 1.0f - delta;
  CellLin q;
  q.r = vp * op - vm * om;
  float a = sp * op + sm * om;
  float c = vp + vm;
  q.jl = 0.5f * a - c;
  q.jr = 0.5f * a + c;
  float d2;
  barrier(delta, q.phi, q.dphi, d2);
  q.psi = half_beta * d2;
  return q;
}

// r and phi only (line-search trials)
template <typename TI>
__device__ __forceinline__ void cell_residual(const TI* Ipc, const TI* Imc, int inner, int m,
                                              int j, float bj, float bj1, float& r, float& phi) {
  float tp, tm, wp, wm;
  cell_positions(bj, bj1, j, tp, tm);
  int ip = cell_index(tp, m, wp), im = cell_index(tm, m, wm);
  float vp, sp, vm, sm;
  interp(Ipc, inner, m, ip, wp, vp, sp);
  interp(Imc, inner, m, im, wm, vm, sm);
  float delta = bj1 - bj;
  r = vp * (1.0f + delta) - vm * (1.0f - delta);
  float df, d2;
  barrier(delta, phi, df, d2);
}

struct Nbrs {   // in-plane neighbour columns of the field (base pointers, nullptr if absent)
  const float *Am, *Ap, *Bm, *Bp;
  float nin;    // wA * (#A neighbours) + wB * (#B neighbours)
};

__device__ __forceinline__ Nbrs make_nbrs(const Geo& g, const float* f, int c) {
  int cA = c % g.nA, cB = c / g.nA;
  Nbrs n;
  n.Am = cA > 0 ? f + col_base(c - 1, g.inner, g.fld_ostride) : nullptr;
  n.Ap = cA < g.nA - 1 ? f + col_base(c + 1, g.inner, g.fld_ostride) : nullptr;
  n.Bm = cB > 0 ? f + col_base(c - g.nA, g.inner, g.fld_ostride) : nullptr;
  n.Bp = cB < g.nB - 1 ? f + col_base(c + g.nA, g.inner, g.fld_ostride) : nullptr;
  n.nin = g.wA * (float)((cA > 0) + (cA < g.nA - 1)) + g.wB * (float)((cB > 0) + (cB < g.nB - 1));
  return n;
}

// ------------------------------------------------------------------------------------------
// J, grad J and the tridiagonal GN coefficients (d, e)
// ------------------------------------------------------------------------------------------

template <typename TI>
__global__ void __launch_bounds__(kBlock)
k_eval(Geo g, const TI* __restrict__ Ip, const TI* __restrict__ Im, const float* __restrict__ b,
       float* __restrict__ grad, float* __restrict__ dco, float* __restrict__ eco, int seg,
       int it, double* partials, unsigned* counter, DevState* st) {
  if (it >= 0 && st->stop) return;
  int c = blockIdx.x * blockDim.x + threadIdx.x;
  int k0 = blockIdx.y * seg, k1 = min(k0 + seg, g.E);
  float accD = 0.f, accS = 0.f, accP = 0.f, accG = 0.f;
  if (c < g.ncols) {
    const int inner = g.inner, m = g.m;
    long long ib = col_base(c, inner, g.img_ostride), fb = col_base(c, inner, g.fld_ostride);
    const TI* Ipc = Ip + ib;
    const TI* Imc = Im + ib;
    const float* bc = b + fb;
    Nbrs nb = make_nbrs(g, b, c);
    float jr_prev = 0.f, r_prev = 0.f, dphi_prev = 0.f, psi_prev = 0.f, b_prev = 0.f;
    float bk = __ldg(bc + (long long)k0 * inner);
    if (k0 > 0) {
      b_prev = __ldg(bc + (long long)(k0 - 1) * inner);
      CellLin q = cell_lin(Ipc, Imc, inner, m, k0 - 1, b_prev, bk, g.half_beta);
      jr_prev = q.jr; r_prev = q.r; dphi_prev = q.dphi; psi_prev = q.psi;
    }
    for (int k = k0; k < k1; ++k) {
      long long o = (long long)k * inner;
      float bn = 0.f, jl = 0.f, jr = 0.f, r = 0.f, dphi = 0.f, psi = 0.f;
      float lap = 0.f;
      if (k < m) {
        bn = __ldg(bc + o + inner);
        CellLin q = cell_lin(Ipc, Imc, inner, m, k, bk, bn, g.half_beta);
        jl = q.jl; jr = q.jr; r = q.r; dphi = q.dphi; psi = q.psi;
        accD += r * r;
        accP += q.phi;
        float dd = bn - bk;
        accS += dd * dd;
        lap += bk - bn;
      }
      if (k > 0) lap += bk - b_prev;
      float la = 0.f, lb = 0.f;
      if (nb.Am) la += bk - __ldg(nb.Am + o);
      if (nb.Ap) { float v = __ldg(nb.Ap + o); la += bk - v; accS += g.wA * (v - bk) * (v - bk); }
      if (nb.Bm) lb += bk - __ldg(nb.Bm + o);
      if (nb.Bp) { float v = __ldg(nb.Bp + o); lb += bk - v; accS += g.wB * (v - bk) * (v - bk); }
      lap += g.wA * la + g.wB * lb;
      float gk = g.vol * (jr_prev * r_prev + jl * r + g.alpha * lap + g.half_beta * (dphi_prev - dphi));
      if (grad) grad[fb + o] = gk;
      accG += gk * gk;
      dco[fb + o] = jr_prev * jr_prev + jl * jl + psi_prev + psi;
      eco[fb + o] = jl * jr - psi;
      b_prev = bk; bk = bn;
      jr_prev = jr; r_prev = r; dphi_prev = dphi; psi_prev = psi;
    }
  }
  double v[4] = {accD, accS, accP, accG}, tot[4];
  if (grid_sum<4>(v, partials, counter, tot)) {
    double hv = 0.5 * (double)g.vol;
    double D = hv * tot[0], S = hv * tot[1], P = hv * tot[2];
    double J = D + g.alpha_d * S + g.beta_d * P;
    st->J = J; st->D = D; st->S = S; st->P = P;
    st->gnorm = sqrt(tot[3]);
    st->status = isnan(J) ? -4 : (isinf(J) ? 1 : 0);
    st->ls_done = 0; st->ls_trials = 0; st->gamma = 0.0; st->gq = 0.0;
    st->pcg_done = 0; st->pcg_iter = 0; st->relres = 0.0;
    if (it >= 0 && !isfinite(J)) { st->stop = 1; st->stop_iter = it; }
  }
}

// ------------------------------------------------------------------------------------------
// Armijo line search: J(b + gamma_t q) for gamma_t = 2^-t, t = t0 .. t0+kLsBatch-1, in one pass;
// the first accepted trial in order wins, exactly as sequential halving would pick it.
// ------------------------------------------------------------------------------------------

template <typename TI>
__global__ void __launch_bounds__(kBlock)
k_linesearch(Geo g, const TI* __restrict__ Ip, const TI* __restrict__ Im,
             const float* __restrict__ b, const float* __restrict__ q,
             const float* __restrict__ grad, int t0, int ls_max, double c1, int seg,
             double* partials, unsigned* counter, DevState* st) {
  if (st->stop || st->ls_done) return;
  constexpr int T = kLsBatch;
  int c = blockIdx.x * blockDim.x + threadIdx.x;
  int k0 = blockIdx.y * seg, k1 = min(k0 + seg, g.E);
  float gam[T];
#pragma unroll
  for (int t = 0; t < T; ++t) gam[t] = ldexpf(1.0f, -(t0 + t));
  float aD[T], aS[T], aP[T];
#pragma unroll
  for (int t = 0; t < T; ++t) { aD[t] = 0.f; aS[t] = 0.f; aP[t] = 0.f; }
  float agq = 0.f;
  if (c < g.ncols) {
    const int inner = g.inner, m = g.m;
    long long ib = col_base(c, inner, g.img_ostride), fb = col_base(c, inner, g.fld_ostride);
    const TI* Ipc = Ip + ib;
    const TI* Imc = Im + ib;
    Nbrs nbb = make_nbrs(g, b, c);
    Nbrs nbq = make_nbrs(g, q, c);
    float bk = __ldg(b + fb + (long long)k0 * inner), qk = __ldg(q + fb + (long long)k0 * inner);
    for (int k = k0; k < k1; ++k) {
      long long o = (long long)k * inner;
      if (t0 == 0) agq += __ldg(grad + fb + o) * qk;
      float bn = 0.f, qn = 0.f;
      if (k < m) { bn = __ldg(b + fb + o + inner); qn = __ldg(q + fb + o + inner); }
      float bAp = 0.f, qAp = 0.f, bBp = 0.f, qBp = 0.f;
      if (nbb.Ap) { bAp = __ldg(nbb.Ap + o); qAp = __ldg(nbq.Ap + o); }
      if (nbb.Bp) { bBp = __ldg(nbb.Bp + o); qBp = __ldg(nbq.Bp + o); }
#pragma unroll
      for (int t = 0; t < T; ++t) {
        float x0 = fmaf(gam[t], qk, bk);
        if (k < m) {
          float x1 = fmaf(gam[t], qn, bn);
          float r, phi;
          cell_residual(Ipc, Imc, inner, m, k, x0, x1, r, phi);
          aD[t] += r * r;
          aP[t] += phi;
          aS[t] += (x1 - x0) * (x1 - x0);
        }
        if (nbb.Ap) { float y = fmaf(gam[t], qAp, bAp) - x0; aS[t] += g.wA * y * y; }
        if (nbb.Bp) { float y = fmaf(gam[t], qBp, bBp) - x0; aS[t] += g.wB * y * y; }
      }
      bk = bn; qk = qn;
    }
  }
  double v[3 * T + 1], tot[3 * T + 1];
#pragma unroll
  for (int t = 0; t < T; ++t) { v[3 * t] = aD[t]; v[3 * t + 1] = aS[t]; v[3 * t + 2] = aP[t]; }
  v[3 * T] = agq;
  if (grid_sum<3 * T + 1>(v, partials, counter, tot)) {
    if (t0 == 0) st->gq = tot[3 * T];
    double gq = st->gq, J = st->J, hv = 0.5 * (double)g.vol;
    if (!(gq < 0.0)) { st->ls_done = 1; st->gamma = 0.0; st->ls_trials = 0; return; }
    for (int t = 0; t < T && t0 + t < ls_max; ++t) {
      double gm = ldexp(1.0, -(t0 + t));
      double Jt = hv * tot[3 * t] + g.alpha_d * hv * tot[3 * t + 1] + g.beta_d * hv * tot[3 * t + 2];
      st->ls_trials = t0 + t + 1;
      if (Jt <= J + c1 * gm * gq) { st->ls_done = 1; st->gamma = gm; return; }
    }
    if (t0 + T >= ls_max) { st->ls_done = 1; st->gamma = 0.0; }
  }
}

// b += gamma q; block 0 records the iteration's statistics row
__global__ void k_update(float* __restrict__ b, const float* __restrict__ q, long long nf, int it,
                         double* stats, DevState* st) {
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    const double nan = __longlong_as_double(0x7ff8000000000000LL);
    bool stopped_before = st->stop && st->stop_iter < it;
    bool stopped_now = st->stop && st->stop_iter == it;
    if (stats) {
      double* row = stats + (long long)it * 10;
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
    st->gn_iter = it + 1;
  }
  if (st->stop) return;
  float gam = (float)st->gamma;
  if (gam == 0.0f) return;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < nf;
       i += (long long)gridDim.x * blockDim.x)
    b[i] = fmaf(gam, q[i], b[i]);
}

// corrected images T+ = I+(t+)(1 + delta), T- = I-(t-)(1 - delta)
template <typename TI>
__global__ void __launch_bounds__(kBlock)
k_correct(Geo g, const TI* __restrict__ Ip, const TI* __restrict__ Im, const float* __restrict__ b,
          float* __restrict__ Tp, float* __restrict__ Tm, int seg) {
  int c = blockIdx.x * blockDim.x + threadIdx.x;
  int j0 = blockIdx.y * seg, j1 = min(j0 + seg, g.m);
  if (c >= g.ncols) return;
  const int inner = g.inner, m = g.m;
  long long ib = col_base(c, inner, g.img_ostride), fb = col_base(c, inner, g.fld_ostride);
  float bj = j0 < j1 ? __ldg(b + fb + (long long)j0 * inner) : 0.f;
  for (int j = j0; j < j1; ++j) {
    float bn = __ldg(b + fb + (long long)(j + 1) * inner);
    float tp, tm, wp, wm, vp, sp, vm, sm;
    cell_positions(bj, bn, j, tp, tm);
    int ip = cell_index(tp, m, wp), im = cell_index(tm, m, wm);
    interp(Ip + ib, inner, m, ip, wp, vp, sp);
    interp(Im + ib, inner, m, im, wm, vm, sm);
    float delta = bn - bj;
    Tp[ib + (long long)j * inner] = vp * (1.0f + delta);
    Tm[ib + (long long)j * inner] = vm * (1.0f - delta);
    bj = bn;
  }
}

__global__ void __launch_bounds__(kBlock)
k_cells(Geo g, const float* __restrict__ b, int* __restrict__ cp, int* __restrict__ cm, int seg) {
  int c = blockIdx.x * blockDim.x + threadIdx.x;
  int j0 = blockIdx.y * seg, j1 = min(j0 + seg, g.m);
  if (c >= g.ncols) return;
  long long ib = col_base(c, g.inner, g.img_ostride), fb = col_base(c, g.inner, g.fld_ostride);
  for (int j = j0; j < j1; ++j) {
    float tp, tm, wp, wm;
    cell_positions(__ldg(b + fb + (long long)j * g.inner), __ldg(b + fb + (long long)(j + 1) * g.inner),
                   j, tp, tm);
    cp[ib + (long long)j * g.inner] = cell_index(tp, g.m, wp);
    cm[ib + (long long)j * g.inner] = cell_index(tm, g.m, wm);
  }
}

__global__ void k_publish_terms(double* terms, const DevState* st) {
  terms[0] = st->J; terms[1] = st->D; terms[2] = st->S; terms[3] = st->P;
}

// ------------------------------------------------------------------------------------------

static dim3 march_grid(const Geo& g, int nodes, int seg) {
  return dim3(ceil_div(g.ncols, kBlock), ceil_div(nodes, seg));
}

#define HYSCO_DISPATCH(dtype, T, ...)                                                  \
  switch (dtype) {                                                                     \
    case 0: { using T = float; __VA_ARGS__; break; }                                   \
    case 1: { using T = __nv_bfloat16; __VA_ARGS__; break; }                           \
    default: { using T = __half; __VA_ARGS__; break; }                                 \
  }

cudaError_t launch_eval(const Geo& g, int dtype, const void* Ip, const void* Im, const float* b,
                        float* grad, float* dco, float* eco, int seg, int it, const Work& w,
                        cudaStream_t s) {
  HYSCO_DISPATCH(dtype, T,
    k_eval<T><<<march_grid(g, g.E, seg), kBlock, 0, s>>>(g, (const T*)Ip, (const T*)Im, b, grad,
                                                          dco, eco, seg, it, w.partials,
                                                          w.counter, w.st))
  return cudaGetLastError();
}

cudaError_t launch_linesearch(const Geo& g, int dtype, const void* Ip, const void* Im,
                              const float* b, const float* q, const float* grad, int t0,
                              int ls_max, double c1, int seg, const Work& w, cudaStream_t s) {
  HYSCO_DISPATCH(dtype, T,
    k_linesearch<T><<<march_grid(g, g.E, seg), kBlock, 0, s>>>(g, (const T*)Ip, (const T*)Im, b,
                                                                q, grad, t0, ls_max, c1, seg,
                                                                w.partials, w.counter, w.st))
  return cudaGetLastError();
}

cudaError_t launch_update(const Geo& g, float* b, const float* q, long long nf, int it,
                          double* stats, const Work& w, cudaStream_t s) {
  (void)g;
  int blocks = (int)((nf + kBlock - 1) / kBlock);
  if (blocks > 148 * 16) blocks = 148 * 16;
  k_update<<<blocks, kBlock, 0, s>>>(b, q, nf, it, stats, w.st);
  return cudaGetLastError();
}

cudaError_t launch_correct(const Geo& g, int dtype, const void* Ip, const void* Im,
                           const float* b, float* Tp, float* Tm, int seg, cudaStream_t s) {
  HYSCO_DISPATCH(dtype, T,
    k_correct<T><<<march_grid(g, g.m, seg), kBlock, 0, s>>>(g, (const T*)Ip, (const T*)Im, b, Tp,
                                                             Tm, seg))
  return cudaGetLastError();
}

cudaError_t launch_cells(const Geo& g, const float* b, int* cp, int* cm, int seg, cudaStream_t s) {
  k_cells<<<march_grid(g, g.m, seg), kBlock, 0, s>>>(g, b, cp, cm, seg);
  return cudaGetLastError();
}

cudaError_t launch_publish_terms(double* terms, const Work& w, cudaStream_t s) {
  k_publish_terms<<<1, 1, 0, s>>>(terms, w.st);
  return cudaGetLastError();
}

}  // namespace hysco
