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
// Image part: eight lanes per (column, image) march the column's cells in segments (both images
// in one launch).  While the cell index is non-decreasing (always, for a feasible field:
// t+_{j+1} - t+_j = 1 + (delta_j + delta_{j+1})/2 > 0) each voxel receives its contributions in
// a two-voxel window and is written once, the voxels two neighbouring segments share summed
// after the march in a fixed order.  A column that folds (the index decreases) or squeezes a
// voxel between three segments is re-done by one lane that writes its window and zeroes the rest
// of the column, then adds the remaining contributions in place (read-modify-write of its own
// column: no other thread touches it).  No atomics: the result is deterministic.
// Field part: thread = (column, segment of nodes), each node from its two adjacent cells.
#include "eval_common.cuh"

namespace hysco {

constexpr int kAdjBlock = 64;   // threads per block of the image adjoint: 8 columns
constexpr int kAdjLanes = 8;    // lanes (segments) per column

// coefficient of the image adjoint for cell j: MODE 0 takes the upstream sensitivity of T,
// MODE 1 the distance term of J (g+ = s vol r_j, g- = -s vol r_j, r recomputed).  blockIdx.y
// selects the image (0: I+, 1: I-).  The field and the sensitivities are loaded kAdjChunk cells
// ahead of their use, so that one memory latency covers a chunk of cells.
constexpr int kAdjChunk = 8;

// MODE 2: (svol / vol) d(v^T g)/dI+- (implicit differentiation): per cell, with
// u = jl v_j + jr v_{j+1}, voxel i+s (s = 0, 1) of the image gets vol (u dr/dI + r du/dI), where
// dr/dI = +-w_s (1 +- delta), du/dI = v_j (da/2 - dc) + v_{j+1} (da/2 + dc), da/dI = -+(1 +- delta)
// (the slope), dc/dI = w_s (w_0 = 1 - w, w_1 = w); svol carries vol and the sign.
//
// Cell j's two contributions: c0 to voxel i, c1 to voxel i + 1; returns i (clamped to
// [-2, m + 1]).  gj: the upstream sensitivity of cell j (MODE 0); vj, vj1: v at its nodes (MODE 2).
template <typename TI, int MODE>
__device__ __forceinline__ int adj_cell(int m, int inner, const TI* Ipc, const TI* Imc, bool plus,
                                        int j, float bj, float bn, float gj, float vj, float vj1,
                                        float svol, float& c0, float& c1) {
  float tp, tm;
  cell_positions(bj, bn, j, tp, tm);
  const float delta = bn - bj;
  const float mod = plus ? 1.0f + delta : 1.0f - delta;
  float w;
  const int i = cell_index(plus ? tp : tm, m, w);
  if (MODE == 0) {
    const float coef = svol * gj * mod;   // svol: a factor on the upstream sensitivity
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
    const float uu = (0.5f * a - cc) * vj + (0.5f * a + cc) * vj1;
    const float dr0 = (plus ? 1.0f : -1.0f) * (1.0f - w) * mod;
    const float dr1 = (plus ? 1.0f : -1.0f) * w * mod;
    const float du0 = vj * (-0.5f * mod - (1.0f - w)) + vj1 * (-0.5f * mod + (1.0f - w));
    const float du1 = vj * (0.5f * mod - w) + vj1 * (0.5f * mod + w);
    c0 = svol * (uu * dr0 + r * du0);
    c1 = svol * (uu * dr1 + r * du1);
  }
  return i;
}

// One thread marches a whole column (every voxel of it written once, or read-modify-written
// after a fold): the fallback of k_image_adjoint for columns its segments cannot share out.
// The field and the sensitivities are loaded kAdjChunk cells ahead of their use.
template <typename TI, int MODE>
__device__ void march_column(int m, int inner, const TI* Ipc, const TI* Imc, const float* bc,
                             const float* gc, const float* vc, float svol, bool plus, float* oc) {
  int base = -2;              // voxel index of A0 (cell indices are clamped to [-2, m + 1])
  float A0 = 0.f, A1 = 0.f;   // pending sums of voxels base and base + 1
  bool rmw = false;
  auto put = [&](int k, float v) { if (k >= 0 && k < m) oc[k * inner] = v; };
  float bnext[kAdjChunk + 1], gnext[kAdjChunk], vnext[kAdjChunk + 1];
  auto fetch = [&](int j0) {
#pragma unroll
    for (int u = 0; u <= kAdjChunk; ++u) bnext[u] = __ldg(bc + min(j0 + u, m) * inner);
#pragma unroll
    for (int u = 0; u <= kAdjChunk; ++u)
      vnext[u] = MODE == 2 ? __ldg(vc + min(j0 + u, m) * inner) : 0.f;
#pragma unroll
    for (int u = 0; u < kAdjChunk; ++u)
      gnext[u] = MODE == 0 ? __ldg(gc + min(j0 + u, m - 1) * inner) : 0.f;
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
      float c0, c1;
      const int i = adj_cell<TI, MODE>(m, inner, Ipc, Imc, plus, j, bv[u], bv[u + 1], gv[u],
                                       vv[u], vv[u + 1], svol, c0, c1);
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

// Image part: eight lanes of a warp per (column, image), lane s marching the cells of segment s
// (ceil(m / 8) cells each; lanes past the last non-empty segment idle).  With a non-decreasing
// cell index the voxels a segment touches form a range that overlaps its neighbours' ranges in at
// most two voxels at each end: a lane writes its other voxels as the march completes them, zeroes
// the untouched gap to its left, keeps its partial sums of the shared voxels and, after the march,
// the left segment adds the right one's partials to its own (left first, a fixed order) and writes
// them.  If any segment of the column sees its index decrease, a fold across a segment boundary,
// or a voxel touched by three segments, lane 0 re-does the whole column with march_column (every
// voxel written again, after the others' writes).  No atomics: deterministic.
template <typename TI, int MODE>
__global__ void __launch_bounds__(kAdjBlock)
k_image_adjoint(Geo g, const TI* __restrict__ Ip, const TI* __restrict__ Im,
                const float* __restrict__ b, const float* __restrict__ gTp,
                const float* __restrict__ gTm, float svol, float* __restrict__ dIp,
                float* __restrict__ dIm, const float* __restrict__ vfld = nullptr) {
  const bool plus = blockIdx.y == 0;
  float* out = plus ? dIp : dIm;
  if (out == nullptr) return;   // the whole block: blockIdx.y picks the image
  const float* gT = plus ? gTp : gTm;
  const int lane = threadIdx.x & 31, s = lane & (kAdjLanes - 1);
  const int c = (blockIdx.x * blockDim.x + threadIdx.x) / kAdjLanes;
  const bool colok = c < g.ncols;   // the same for the column's eight lanes
  const int inner = g.inner, m = g.m;
  const int cc = colok ? c : g.ncols - 1;
  const int ib = col_base(cc, inner, g.img_ostride), fb = col_base(cc, inner, g.fld_ostride);
  const TI* Ipc = Ip + ib;
  const TI* Imc = Im + ib;
  const float* bc = b + fb;
  float* oc = out + ib;
  const int L = ceil_div(m, kAdjLanes), nseg = ceil_div(m, L);
  const bool act = colok && s < nseg;
  const int j0 = s * L, j1 = min(j0 + L, m);
  auto index_of = [&](int j) {
    float tp, tm, w;
    cell_positions(__ldg(bc + j * inner), __ldg(bc + (j + 1) * inner), j, tp, tm);
    return cell_index(plus ? tp : tm, m, w);
  };
  const int ifirst = act ? index_of(j0) : 0, ilast = act ? index_of(j1 - 1) : 0;
  const int iprev = __shfl_up_sync(0xffffffffu, ilast, 1);     // segment s - 1's last index
  const int inext = __shfl_down_sync(0xffffffffu, ifirst, 1);  // segment s + 1's first index
  const bool hasprev = s > 0, hasnext = s + 1 < nseg;
  bool bad = act && ((hasprev && ifirst < iprev) || (hasprev && hasnext && inext <= iprev + 1));
  // voxels shared with the segment before: [ifirst, iprev + 1]; after: [inext, ilast + 1]
  const int llo = ifirst, lhi = hasprev ? iprev + 1 : ifirst - 1;
  const int rlo = hasnext ? inext : ilast + 2, rhi = ilast + 1;
  float L0 = 0.f, L1 = 0.f, R0 = 0.f, R1 = 0.f;
  auto emit = [&](int v, float val) {
    if (v >= llo && v <= lhi) {
      if (v == llo) L0 += val; else L1 += val;
    } else if (v >= rlo && v <= rhi) {
      if (v == rlo) R0 += val; else R1 += val;
    } else if (v >= 0 && v < m) {
      oc[v * inner] = val;
    }
  };
  if (act && !bad) {
    // the untouched voxels before this segment's range (after the previous one's)
    for (int v = max(hasprev ? iprev + 2 : 0, 0); v < min(ifirst, m); ++v) oc[v * inner] = 0.f;
    int base = ifirst, iold = ifirst;
    float A0 = 0.f, A1 = 0.f;
    float bj = __ldg(bc + j0 * inner);
    float vj = MODE == 2 ? __ldg(vfld + fb + j0 * inner) : 0.f;
    for (int j = j0; j < j1; ++j) {
      const float bn = __ldg(bc + (j + 1) * inner);
      const float vn = MODE == 2 ? __ldg(vfld + fb + (j + 1) * inner) : 0.f;
      const float gj = MODE == 0 ? __ldg(gT + ib + j * inner) : 0.f;
      float c0, c1;
      const int i = adj_cell<TI, MODE>(m, inner, Ipc, Imc, plus, j, bj, bn, gj, vj, vn, svol,
                                       c0, c1);
      if (i < iold) { bad = true; break; }   // the index decreased: fold
      iold = i;
      while (base < i) {
        emit(base, A0);
        A0 = A1;
        A1 = 0.f;
        ++base;
      }
      A0 += c0;
      A1 += c1;
      bj = bn;
      vj = vn;
    }
    if (!bad) {
      emit(base, A0);
      emit(base + 1, A1);
      if (!hasnext)
        for (int v = max(ilast + 2, 0); v < m; ++v) oc[v * inner] = 0.f;
    }
  }
  // any lane of the column unable to finish its share sends the whole column to the fallback
  const unsigned grp = 0xffu << (lane & ~(kAdjLanes - 1));
  const bool fallback = (__ballot_sync(0xffffffffu, bad) & grp) != 0u;
  const float nL0 = __shfl_down_sync(0xffffffffu, L0, 1);
  const float nL1 = __shfl_down_sync(0xffffffffu, L1, 1);
  if (act && !fallback && hasnext) {
    if (rlo >= 0 && rlo < m && rlo <= rhi) oc[rlo * inner] = R0 + nL0;
    if (rlo + 1 >= 0 && rlo + 1 < m && rlo + 1 <= rhi) oc[(rlo + 1) * inner] = R1 + nL1;
  }
  __syncwarp();
  if (colok && fallback && s == 0)
    march_column<TI, MODE>(m, inner, Ipc, Imc, bc, gT ? gT + ib : nullptr,
                           MODE == 2 ? vfld + fb : nullptr, svol, plus, oc);
}

// field part of the corrected-image adjoint: node k of column c gets cell k-1's d/db_{j+1} term
// and cell k's d/db_j term
template <typename TI>
__global__ void __launch_bounds__(kBlock)
k_field_adjoint(Geo g, const TI* __restrict__ Ip, const TI* __restrict__ Im,
                const float* __restrict__ b, const float* __restrict__ gTp,
                const float* __restrict__ gTm, float scale, float* __restrict__ db) {
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
    const float gp = gTp ? scale * __ldg(gTp + ib + j * inner) : 0.f;
    const float gm = gTm ? scale * __ldg(gTm + ib + j * inner) : 0.f;
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
  const dim3 cols(ceil_div(g.ncols, kAdjBlock / kAdjLanes), 2);
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
                                   cudaStream_t s, float scale) {
  const dim3 cols(ceil_div(g.ncols, kAdjBlock / kAdjLanes), 2);
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
    if (dp || dm) k_image_adjoint<T, 0><<<cols, kAdjBlock, 0, s>>>(g, P, M, b, gTp, gTm, scale, dp, dm);
    if (db) k_field_adjoint<T><<<march, kBlock, 0, s>>>(g, P, M, b, gTp, gTm, scale, db);
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
  const dim3 cols(ceil_div(g.ncols, kAdjBlock / kAdjLanes), 2);
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
