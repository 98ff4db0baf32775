// Adjoints (vector-Jacobian products) of the corrected images of Eq. 1 and of J at fixed b.
//
// Per cell j of a PE column, T+_j = I+(t+_j)(1 + delta_j) with I+(t) = (1 - w) I+[i] + w I+[i+1],
// i = floor(t), w = t - i (zero outside the column), t+_j = j + (b_j + b_{j+1})/2,
// delta_j = b_{j+1} - b_j; T-_j likewise with t-_j = j - (b_j + b_{j+1})/2 and 1 - delta_j.
//   image part:  dI+[i] += g+_j (1 - w)(1 + delta_j),  dI+[i+1] += g+_j w (1 + delta_j)
//   field part:  dT+_j/db_j = 1/2 I+'(t+)(1 + delta) - I+(t+),  dT+_j/db_{j+1} = ... + I+(t+)
//                dT-_j/db_j = -1/2 I-'(t-)(1 - delta) + I-(t-), dT-_j/db_{j+1} = ... - I-(t-)
// Cells, weights and interpolated values are recomputed from b with the forward pass's own
// single-precision operations (eval_common.cuh), never stored.
//
// Image part: one thread per (column, image) marches the column's cells in order (both images in
// one launch).  While the cell index is non-decreasing (always, for a feasible field:
// t+_{j+1} - t+_j = 1 + (delta_j + delta_{j+1})/2 > 0) each voxel receives all its contributions
// inside a two-voxel window and is written once; if the index ever decreases, the thread writes
// its window and zeroes the rest of its column, then adds the remaining contributions in place
// (read-modify-write of its own column: no other thread touches it).  No atomics: the result is
// deterministic.
// Field part: thread = (column, segment of nodes), each node from its two adjacent cells.
#include "eval_common.cuh"

namespace hysco {

constexpr int kAdjBlock = 64;   // one column per thread: small blocks spread the columns over SMs

// coefficient of the image adjoint for cell j: MODE 0 takes the upstream sensitivity of T,
// MODE 1 the distance term of J (g+ = s vol r_j, g- = -s vol r_j, r recomputed).  blockIdx.y
// selects the image (0: I+, 1: I-).  The field and the sensitivities are loaded kAdjChunk cells
// ahead of their use, so that one memory latency covers a chunk of cells.
constexpr int kAdjChunk = 8;

// MODE 2: (svol / vol) d(v^T g)/dI+- (implicit differentiation): per cell, with
// u = jl v_j + jr v_{j+1}, voxel i+s (s = 0, 1) of the image gets vol (u dr/dI + r du/dI), where
// dr/dI = +-w_s (1 +- delta), du/dI = v_j (da/2 - dc) + v_{j+1} (da/2 + dc), da/dI = -+(1 +- delta)
// (the slope), dc/dI = w_s (w_0 = 1 - w, w_1 = w); svol carries vol and the sign.
template <typename TI, int MODE>
__global__ void __launch_bounds__(kAdjBlock)
k_image_adjoint(Geo g, const TI* __restrict__ Ip, const TI* __restrict__ Im,
                const float* __restrict__ b, const float* __restrict__ gTp,
                const float* __restrict__ gTm, float svol, float* __restrict__ dIp,
                float* __restrict__ dIm, const float* __restrict__ vfld = nullptr) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  const bool plus = blockIdx.y == 0;
  float* out = plus ? dIp : dIm;
  const float* gT = plus ? gTp : gTm;
  if (c >= g.ncols || out == nullptr) return;
  const int inner = g.inner, m = g.m;
  const int ib = col_base(c, inner, g.img_ostride), fb = col_base(c, inner, g.fld_ostride);
  const TI* Ipc = Ip + ib;
  const TI* Imc = Im + ib;
  float* oc = out + ib;
  int base = -2;              // voxel index of A0 (cell indices are clamped to [-2, m + 1])
  float A0 = 0.f, A1 = 0.f;   // pending sums of voxels base and base + 1
  bool rmw = false;
  auto put = [&](int k, float v) { if (k >= 0 && k < m) oc[k * inner] = v; };
  float bnext[kAdjChunk + 1], gnext[kAdjChunk], vnext[kAdjChunk + 1];
  auto fetch = [&](int j0) {
#pragma unroll
    for (int u = 0; u <= kAdjChunk; ++u) bnext[u] = __ldg(b + fb + min(j0 + u, m) * inner);
#pragma unroll
    for (int u = 0; u <= kAdjChunk; ++u)
      vnext[u] = MODE == 2 ? __ldg(vfld + fb + min(j0 + u, m) * inner) : 0.f;
#pragma unroll
    for (int u = 0; u < kAdjChunk; ++u)
      gnext[u] = MODE == 0 ? __ldg(gT + ib + min(j0 + u, m - 1) * inner) : 0.f;
  };
  fetch(0);
  for (int j0 = 0; j0 < m; j0 += kAdjChunk) {
    float bv[kAdjChunk + 1], gv[kAdjChunk], vv[kAdjChunk + 1];
#pragma unroll
    for (int u = 0; u <= kAdjChunk; ++u) bv[u] = bnext[u];
#pragma unroll
    for (int u = 0; u <= kAdjChunk; ++u) vv[u] = vnext[u];
#pragma unroll
    for (int u = 0; u < kAdjChunk; ++u) gv[u] = gnext[u];
    if (j0 + kAdjChunk < m) fetch(j0 + kAdjChunk);
#pragma unroll
    for (int u = 0; u < kAdjChunk; ++u) {
      const int j = j0 + u;
      if (j >= m) break;
      const float bj = bv[u], bn = bv[u + 1];
      float tp, tm;
      cell_positions(bj, bn, j, tp, tm);
      const float delta = bn - bj;
      const float mod = plus ? 1.0f + delta : 1.0f - delta;
      float w;
      const int i = cell_index(plus ? tp : tm, m, w);
      float c0, c1;
      if (MODE == 0) {
        const float coef = gv[u] * mod;
        c0 = (1.0f - w) * coef;
        c1 = w * coef;
      } else if (MODE == 1) {
        float wp, wm, vp, sp, vm, sm;
        const int ip = cell_index(tp, m, wp), im = cell_index(tm, m, wm);
        interp(Ipc, inner, m, ip, wp, vp, sp);
        interp(Imc, inner, m, im, wm, vm, sm);
        const float r = vp * (1.0f + delta) - vm * (1.0f - delta);
        const float coef = (plus ? svol : -svol) * r * mod;
        c0 = (1.0f - w) * coef;
        c1 = w * coef;
      } else {
        float wp, wm, vp, sp, vm, sm;
        const int ip = cell_index(tp, m, wp), im = cell_index(tm, m, wm);
        interp(Ipc, inner, m, ip, wp, vp, sp);
        interp(Imc, inner, m, im, wm, vm, sm);
        const float r = vp * (1.0f + delta) - vm * (1.0f - delta);
        const float a = sp * (1.0f + delta) + sm * (1.0f - delta);
        const float cc = vp + vm;
        const float vj = vv[u], vj1 = vv[u + 1];
        const float uu = (0.5f * a - cc) * vj + (0.5f * a + cc) * vj1;
        const float dr0 = (plus ? 1.0f : -1.0f) * (1.0f - w) * mod;
        const float dr1 = (plus ? 1.0f : -1.0f) * w * mod;
        const float du0 = vj * (-0.5f * mod - (1.0f - w)) + vj1 * (-0.5f * mod + (1.0f - w));
        const float du1 = vj * (0.5f * mod - w) + vj1 * (0.5f * mod + w);
        c0 = svol * (uu * dr0 + r * du0);
        c1 = svol * (uu * dr1 + r * du1);
      }
      if (!rmw && i < base) {   // index decreased: switch to in-place accumulation
        put(base, A0);
        put(base + 1, A1);
        for (int k = max(base + 2, 0); k < m; ++k) oc[k * inner] = 0.f;
        rmw = true;
      }
      if (rmw) {
        if (i >= 0 && i < m) oc[i * inner] += c0;
        if (i + 1 >= 0 && i + 1 < m) oc[(i + 1) * inner] += c1;
      } else {
        while (base < i) {
          put(base, A0);
          A0 = A1;
          A1 = 0.f;
          ++base;
        }
        A0 += c0;
        A1 += c1;
      }
    }
  }
  if (!rmw) {
    put(base, A0);
    put(base + 1, A1);
    for (int k = max(base + 2, 0); k < m; ++k) oc[k * inner] = 0.f;
  }
}

// field part of the corrected-image adjoint: node k of column c gets cell k-1's d/db_{j+1} term
// and cell k's d/db_j term
template <typename TI>
__global__ void __launch_bounds__(kBlock)
k_field_adjoint(Geo g, const TI* __restrict__ Ip, const TI* __restrict__ Im,
                const float* __restrict__ b, const float* __restrict__ gTp,
                const float* __restrict__ gTm, float* __restrict__ db) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= g.ncols) return;
  const int inner = g.inner, m = g.m;
  const int k0 = blockIdx.y * kSeg, k1 = min(k0 + kSeg, m + 1);
  const int ib = col_base(c, inner, g.img_ostride), fb = col_base(c, inner, g.fld_ostride);
  // d T_j / d b_j and d T_j / d b_{j+1}, weighted by the upstream sensitivities, for cell j
  auto cell = [&](int j, float& lo, float& hi) {
    lo = hi = 0.f;
    if (j < 0 || j >= m) return;
    const float bj = __ldg(b + fb + j * inner), bn = __ldg(b + fb + (j + 1) * inner);
    float tp, tm, wp, wm, vp, sp, vm, sm;
    cell_positions(bj, bn, j, tp, tm);
    const int ip = cell_index(tp, m, wp), im = cell_index(tm, m, wm);
    interp(Ip + ib, inner, m, ip, wp, vp, sp);
    interp(Im + ib, inner, m, im, wm, vm, sm);
    const float delta = bn - bj;
    const float gp = gTp ? __ldg(gTp + ib + j * inner) : 0.f;
    const float gm = gTm ? __ldg(gTm + ib + j * inner) : 0.f;
    const float ap = 0.5f * sp * (1.0f + delta), am = 0.5f * sm * (1.0f - delta);
    lo = gp * (ap - vp) + gm * (vm - am);
    hi = gp * (ap + vp) - gm * (am + vm);
  };
  float lo, hi;
  cell(k0 - 1, lo, hi);
  float carry = hi;
  for (int k = k0; k < k1; ++k) {
    cell(k, lo, hi);
    db[fb + k * inner] = carry + lo;
    carry = hi;
  }
}

// sign * v^T dg/dalpha and sign * v^T dg/dbeta (implicit differentiation): g = vol [Jr^T r + alpha lap(b)
// + beta/2 D^T phi'(delta)] in the eval kernel's units, so per node k the two sums take
// v_k vol lap_k and v_k vol/2 (phi'(delta_{k-1}) - phi'(delta_k)) (phi' of a missing cell: 0).
__global__ void __launch_bounds__(kBlock)
k_theta_dots(Geo g, const float* __restrict__ b, const float* __restrict__ v, double sign,
             float* partials, unsigned* counter, double* out) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  const int inner = g.inner, m = g.m;
  const int k0 = blockIdx.y * kSeg, k1 = min(k0 + kSeg, m + 1);
  float sa = 0.f, sb = 0.f;
  if (c < g.ncols) {
    const int fb = col_base(c, inner, g.fld_ostride);
    const ColNbrs nb = col_nbrs(g, c, fb);
    auto dphi = [&](int j) {   // phi'(delta_j), 0 outside the column
      if (j < 0 || j >= m) return 0.f;
      float f, df, d2f;
      barrier(__ldg(b + fb + (j + 1) * inner) - __ldg(b + fb + j * inner), f, df, d2f);
      return df;
    };
    float left = dphi(k0 - 1);
    for (int k = k0; k < k1; ++k) {
      const int o = k * inner;
      const float bk = __ldg(b + fb + o);
      const float bl = k > 0 ? __ldg(b + fb + o - inner) : bk;
      const float br = k < m ? __ldg(b + fb + o + inner) : bk;
      const float lap = (bk - bl) + (bk - br) +
                        g.wA * ((bk - __ldg(b + nb.Am + o)) + (bk - __ldg(b + nb.Ap + o))) +
                        g.wB * ((bk - __ldg(b + nb.Bm + o)) + (bk - __ldg(b + nb.Bp + o)));
      const float right = dphi(k);
      const float vk = __ldg(v + fb + o);
      sa += vk * lap;
      sb += vk * (left - right);
      left = right;
    }
  }
  float vals[2] = {sa, sb};
  double tot[2];
  if (grid_sum<2>(vals, partials, counter, tot)) {
    out[0] = sign * (double)g.vol * tot[0];
    out[1] = sign * 0.5 * (double)g.vol * tot[1];
  }
}

cudaError_t launch_theta_dots(const Geo& g, const float* b, const float* v, double sign,
                              double* out, const Work& w, cudaStream_t s) {
  k_theta_dots<<<dim3(ceil_div(g.ncols, kBlock), ceil_div(g.E, kSeg)), kBlock, 0, s>>>(
      g, b, v, sign, w.partials, w.counter, out);
  return cudaGetLastError();
}

cudaError_t launch_mixed_image_adjoint(const Geo& g, int dtype, const void* Ip, const void* Im,
                                       const float* b, const float* v, float svol, float* dIp,
                                       float* dIm, cudaStream_t s) {
  const dim3 cols(ceil_div(g.ncols, kAdjBlock), 2);
  auto run = [&](auto tag) -> cudaError_t {
    using T = decltype(tag);
    if (dIp || dIm)
      k_image_adjoint<T, 2><<<cols, kAdjBlock, 0, s>>>(g, (const T*)Ip, (const T*)Im, b, nullptr,
                                                       nullptr, svol, dIp, dIm, v);
    return cudaGetLastError();
  };
  switch (dtype) {
    case 0: return run(float{});
    case 1: return run(__nv_bfloat16{});
    default: return run(__half{});
  }
}

cudaError_t launch_correct_adjoint(const Geo& g, int dtype, const void* Ip, const void* Im,
                                   const float* b, const float* gTp, const float* gTm,
                                   float* dIp, float* dIm, float* db, size_t img_bytes,
                                   cudaStream_t s) {
  const dim3 cols(ceil_div(g.ncols, kAdjBlock), 2);
  const dim3 march(ceil_div(g.ncols, kBlock), ceil_div(g.E, kSeg));
  // an image without an upstream sensitivity has a zero adjoint
  float* dp = gTp ? dIp : nullptr;
  float* dm = gTm ? dIm : nullptr;
  if (dIp && !gTp)
    if (cudaError_t e = cudaMemsetAsync(dIp, 0, img_bytes, s)) return e;
  if (dIm && !gTm)
    if (cudaError_t e = cudaMemsetAsync(dIm, 0, img_bytes, s)) return e;
  auto run = [&](auto tag) -> cudaError_t {
    using T = decltype(tag);
    const T* P = (const T*)Ip;
    const T* M = (const T*)Im;
    if (dp || dm) k_image_adjoint<T, 0><<<cols, kAdjBlock, 0, s>>>(g, P, M, b, gTp, gTm, 0.f, dp, dm);
    if (db) k_field_adjoint<T><<<march, kBlock, 0, s>>>(g, P, M, b, gTp, gTm, db);
    return cudaGetLastError();
  };
  switch (dtype) {
    case 0: return run(float{});
    case 1: return run(__nv_bfloat16{});
    default: return run(__half{});
  }
}

cudaError_t launch_image_grad(const Geo& g, int dtype, const void* Ip, const void* Im,
                              const float* b, float svol, float* dIp, float* dIm,
                              cudaStream_t s) {
  const dim3 cols(ceil_div(g.ncols, kAdjBlock), 2);
  auto run = [&](auto tag) -> cudaError_t {
    using T = decltype(tag);
    if (dIp || dIm)
      k_image_adjoint<T, 1><<<cols, kAdjBlock, 0, s>>>(g, (const T*)Ip, (const T*)Im, b, nullptr,
                                                       nullptr, svol, dIp, dIm);
    return cudaGetLastError();
  };
  switch (dtype) {
    case 0: return run(float{});
    case 1: return run(__nv_bfloat16{});
    default: return run(__half{});
  }
}

}  // namespace hysco
