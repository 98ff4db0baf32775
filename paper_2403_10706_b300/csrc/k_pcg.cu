// Gauss-Newton Hessian-vector products and the preconditioned CG steps (Sec. 2.3.1).
//
// The GN Hessian about the last evaluated field is
//   H = vol [T + alpha L],  T = per-column tridiagonal (d_k on the diagonal, e_k between k, k+1),
// with d, e written by the eval kernel and L the 7-point negative Laplacian in PE-voxel units
// (PE weight 1, in-plane weights wA, wB).  Vectors are field-shaped float32 in the pitched layout
// (Geo::P2): one thread handles one aligned group of 4 nodes of a row (see hv_group).
//
// PCG (Hestenes-Stiefel, x0 = 0) is split in two kernels per iteration i so that every global
// inner product is reduced exactly once, in the kernel that produces it:
//   k_pcg_hp:     w = H z, p = z + beta p, Hp = w + beta Hp (p = z, Hp = w when i = 0),
//                 partial p.Hp -> last block: alpha = rho / p.Hp (stop if p.Hp <= 0)
//   k_pcg_update: x += alpha p, r -= alpha Hp, partial r.r; z = M^{-1} r, partial r.z
//                 -> last block: stop if ||r|| / ||r0|| < rtol, else beta = r.z / rho, rho = r.z
// H p is kept by the recurrence H p = H z + beta H p_old (H is linear, so this is the same vector
// as applying the stencil to p, up to rounding): the stencil reads only z, and p, Hp are updated
// in place by their owning thread.
#include <algorithm>

#include "hysco_internal.cuh"

namespace hysco {

// ------------------------------------------------------------------------------------------
// H v: one thread per aligned group of 4 nodes of the pitched field (hv_group): neighbours along
// the two outer axes are float4 loads, along the row they come from the group and one scalar on
// each side; an absent neighbour (Neumann end) is the node itself, which zeroes its difference.
// ------------------------------------------------------------------------------------------

// Hv (PCG = false) or the PCG step (PCG = true): w = H z; p = z + beta p; Hp = w + beta Hp.
template <int P, bool PCG>
__global__ void __launch_bounds__(kBlock)
k_hv(Geo g, const float* z, float* p, float* Hp, const float* __restrict__ dco,
     const float* __restrict__ eco, int first, float* partials, unsigned* counter,
     DevState* st) {
  float beta = 0.f;
  if (PCG) {
    if (st->stop || st->pcg_done) return;
    beta = first ? 0.f : (float)st->beta_cg;
  }
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  float acc = 0.f;
  if (t < (g.nfp >> 2)) acc = hv_group<P, PCG>(g, t, z, p, Hp, dco, eco, beta, first != 0);
  if (!PCG) return;
  float v[1] = {acc};
  double tot[1];
  if (grid_sum<1>(v, partials, counter, tot)) {
    double pHp = tot[0];
    if (!(pHp > 0.0)) {
      st->pcg_done = 1;
    } else {
      st->alpha_cg = st->rho / pHp;
    }
  }
}

// ------------------------------------------------------------------------------------------
// elementwise PCG steps, float4 over the pitched field (a multiple of 4 long, padding zero);
// the inverse Jacobi diagonal comes from the eval kernel.
// ------------------------------------------------------------------------------------------

__device__ __forceinline__ float4 ld4(const float* p, int i) {
  return __ldg(reinterpret_cast<const float4*>(p) + i);
}
__device__ __forceinline__ void st4(float* p, int i, float4 v) {
  reinterpret_cast<float4*>(p)[i] = v;
}

// PCG init with Jacobi: r = sign * grad (sign = -1 in a GN step), x = 0, z = r / diag;
// rr0 = r.r, rho = r.z
__global__ void __launch_bounds__(kBlock)
k_pcg_init_jacobi(Geo g, const float* __restrict__ grad, float sign, float* __restrict__ x,
                  float* __restrict__ r, float* __restrict__ z, const float* __restrict__ invd,
                  float* partials, unsigned* counter, DevState* st) {
  if (st->stop) return;
  float arr = 0.f, arz = 0.f;
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < (g.nfp >> 2)) {
    float4 gv = ld4(grad, i), dv = ld4(invd, i);
    float4 rv = make_float4(sign * gv.x, sign * gv.y, sign * gv.z, sign * gv.w);
    float4 zv = make_float4(rv.x * dv.x, rv.y * dv.y, rv.z * dv.z, rv.w * dv.w);
    st4(x, i, make_float4(0.f, 0.f, 0.f, 0.f));
    st4(r, i, rv);
    st4(z, i, zv);
    arr = rv.x * rv.x + rv.y * rv.y + rv.z * rv.z + rv.w * rv.w;
    arz = rv.x * zv.x + rv.y * zv.y + rv.z * zv.z + rv.w * zv.w;
  }
  float v[2] = {arr, arz};
  double tot[2];
  if (grid_sum<2>(v, partials, counter, tot)) {
    st->rr0 = tot[0]; st->rr = tot[0]; st->rho = tot[1];
    st->pcg_iter = 0;
    st->pcg_done = !(tot[0] > 0.0);
    st->relres = tot[0] > 0.0 ? 1.0 : 0.0;
  }
}

__device__ __forceinline__ void pcg_finish(DevState* st, double rr, double rz, double rtol) {
  st->pcg_iter += 1;
  st->rr = rr;
  st->relres = sqrt(rr) / sqrt(st->rr0);
  if (st->relres < rtol) {
    st->pcg_done = 1;
  } else {
    st->beta_cg = rz / st->rho;
    st->rho = rz;
  }
}

// x += alpha p, r -= alpha Hp, z = r / diag
__global__ void __launch_bounds__(kBlock)
k_pcg_update_jacobi(Geo g, float* __restrict__ x, float* __restrict__ r,
                    const float* __restrict__ p, const float* __restrict__ Hp,
                    float* __restrict__ z, const float* __restrict__ invd, int first, double rtol,
                    float* partials, unsigned* counter, DevState* st) {
  if (st->stop || st->pcg_done) return;
  const float a = (float)st->alpha_cg;
  float arr = 0.f, arz = 0.f;
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < (g.nfp >> 2)) {
    float4 pv = ld4(p, i), hv = ld4(Hp, i), dv = ld4(invd, i);
    float4 rv = reinterpret_cast<const float4*>(r)[i];
    float4 xv = first ? make_float4(0.f, 0.f, 0.f, 0.f) : reinterpret_cast<const float4*>(x)[i];
    xv.x = fmaf(a, pv.x, xv.x); xv.y = fmaf(a, pv.y, xv.y);
    xv.z = fmaf(a, pv.z, xv.z); xv.w = fmaf(a, pv.w, xv.w);
    rv.x = fmaf(-a, hv.x, rv.x); rv.y = fmaf(-a, hv.y, rv.y);
    rv.z = fmaf(-a, hv.z, rv.z); rv.w = fmaf(-a, hv.w, rv.w);
    float4 zv = make_float4(rv.x * dv.x, rv.y * dv.y, rv.z * dv.z, rv.w * dv.w);
    st4(x, i, xv);
    st4(r, i, rv);
    st4(z, i, zv);
    arr = rv.x * rv.x + rv.y * rv.y + rv.z * rv.z + rv.w * rv.w;
    arz = rv.x * zv.x + rv.y * zv.y + rv.z * zv.z + rv.w * zv.w;
  }
  float v[2] = {arr, arz};
  double tot[2];
  if (grid_sum<2>(v, partials, counter, tot)) pcg_finish(st, tot[0], tot[1], rtol);
}

// z = r / diag with r and z in the caller's layout (1/diag pitched)
__global__ void __launch_bounds__(kBlock)
k_jacobi_caller(Geo g, const float* __restrict__ r, float* __restrict__ z,
                const float* __restrict__ invd) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= g.nf) return;
  const int row = (int)fdiv((unsigned)n, g.divfe2);
  z[n] = __ldg(r + n) * __ldg(invd + row * g.P2 + (n - row * g.fe[2]));
}

// caller layout <-> pitched layout (padding written as zero)
__global__ void __launch_bounds__(kBlock)
k_to_pitched(Geo g, const float* __restrict__ src, float* __restrict__ dst) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (g.nfp >> 2)) return;
  GroupPos q = group_pos(g, t);
  float v[4];
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    int x = q.x0 + u;
    v[u] = x < g.fe[2] ? __ldg(src + q.row * g.fe[2] + x) : 0.f;
  }
  reinterpret_cast<float4*>(dst)[t] = make_float4(v[0], v[1], v[2], v[3]);
}

__global__ void __launch_bounds__(kBlock)
k_from_pitched(Geo g, const float* __restrict__ src, float* __restrict__ dst) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (g.nfp >> 2)) return;
  GroupPos q = group_pos(g, t);
  float4 v = __ldg(reinterpret_cast<const float4*>(src) + t);
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    int x = q.x0 + u;
    if (x < g.fe[2]) dst[q.row * g.fe[2] + x] = f4get(v, u);
  }
}

// Per-column block preconditioner (end of Sec. 2.3.1): one thread per PE column marches along it
// (coalesced row accesses across the warp), the values of the next kColRing - 1 nodes already
// on their way through a per-thread shared-memory ring (cp.async: each thread its own words, so
// no block barrier), so the sequential recurrence waits on arithmetic, not on memory.
//   M = tridiag(vol (e_k - alpha), vol (d_k + alpha (npe_k + nin)), vol (e_k - alpha)), M = L D L^T:
//   D_0 = dia_0, l_k = off_k / D_k, D_{k+1} = dia_{k+1} - l_k off_k; stored 1 / D_k and l_k.
constexpr int kColRing = 16;
constexpr int kColGroup = 4;   // nodes per copy group (one commit and one wait per group)
// threads per block of the column kernels: a column per thread and one warp per block, so that
// the few thousand columns spread over every SM (the sequential recurrences are latency-bound)
constexpr int kColBlock = 32;

struct ColPos {
  int base;     // pitched offset of node 0
  float nin;    // in-plane part of L_kk
};
__device__ __forceinline__ ColPos col_pos(const Geo& g, int c) {
  const int cB = c / g.nA, cA = c - cB * g.nA;
  ColPos q;
  q.base = cB * g.psB + cA * g.psA;
  q.nin = g.wA * (float)((cA > 0) + (cA < g.nA - 1)) + g.wB * (float)((cB > 0) + (cB < g.nB - 1));
  return q;
}

__global__ void __launch_bounds__(kColBlock)
k_col_factor(Geo g, const float* __restrict__ dco, const float* __restrict__ eco,
             float* __restrict__ invD, float* __restrict__ lco) {
  constexpr int R = kColRing, NG = kColRing / kColGroup;
  __shared__ float ring[R][2][kColBlock];
  const int lane = threadIdx.x, c = blockIdx.x * kColBlock + lane;
  if (c >= g.ncols) return;
  const ColPos cp = col_pos(g, c);
  const int E = g.E, m = g.m, ps = g.psP, fb = cp.base;
  const float vol = g.vol, alpha = g.alpha;
  // step k (0 .. E - 2) reads e_k and d_{k+1}; copy group q holds steps kColGroup q .. + 3
  auto fetch = [&](int q) {
#pragma unroll
    for (int u = 0; u < kColGroup; ++u) {
      const int k = q * kColGroup + u, kk = min(k, E - 2), sl = k % R;
      cp_async4(&ring[sl][0][lane], eco + fb + kk * ps, true);
      cp_async4(&ring[sl][1][lane], dco + fb + (kk + 1) * ps, true);
    }
    cp_async_commit();
  };
  // dia_0 (npe = 1: node 0 has one PE neighbour)
  float D = vol * (__ldg(dco + fb) + alpha * (1.0f + cp.nin));
  for (int q = 0; q < NG - 1; ++q) fetch(q);
  for (int q = 0; q * kColGroup < E - 1; ++q) {
    fetch(q + NG - 1);
    cp_async_wait<NG - 1>();
    // no branch inside the group (steps past the column's end are predicated off), so the
    // compiler can issue the group's shared loads ahead of its recurrence
#pragma unroll
    for (int u = 0; u < kColGroup; ++u) {
      const int k = q * kColGroup + u, sl = k % R;
      const bool in = k < E - 1;
      const float ok = vol * (ring[sl][0][lane] - alpha);
      const float iD = __frcp_rn(D);   // = 1.0f / D, correctly rounded
      const float l = ok * iD;
      if (in) {
        invD[fb + k * ps] = iD;
        lco[fb + k * ps] = l;
      }
      const float npe = (float)(1 + (k + 1 < m));
      const float Dn = fmaf(-l, ok, vol * (ring[sl][1][lane] + alpha * (npe + cp.nin)));
      D = in ? Dn : D;
    }
  }
  cp_async_wait<0>();
  invD[fb + (E - 1) * ps] = __frcp_rn(D);
  lco[fb + (E - 1) * ps] = 0.f;
}

// z = M^{-1} r per column (forward L y = r, backward L^T z = D^{-1} y; y kept in z).  MODE 0:
// apply to r, r and z in the caller's layout (the API call); MODE 1: PCG init (r = sign * grad,
// x = 0); MODE 2: PCG update (x += alpha p, r -= alpha Hp) first.  MODE 1 / 2 work on pitched
// vectors, reduce r.r and r.z and take the PCG decisions.  The factors are pitched.
template <int MODE>
__global__ void __launch_bounds__(kColBlock)
k_col_solve(Geo g, const float* __restrict__ grad, float* __restrict__ x, float* r,
            const float* __restrict__ p, const float* __restrict__ Hp, float* __restrict__ z,
            const float* __restrict__ invD, const float* __restrict__ lco, int first,
            double rtol, float sign, float* partials, unsigned* counter, DevState* st) {
  if (MODE != 0 && st->stop) return;
  if (MODE == 2 && st->pcg_done) return;
  constexpr int R = kColRing, NA = 5, NG = kColRing / kColGroup;
  __shared__ float ring[R][NA][kColBlock];
  const int lane = threadIdx.x, c = blockIdx.x * kColBlock + lane;
  float arr = 0.f, arz = 0.f;
  if (c < g.ncols) {
    const int E = g.E, ps = g.psP, fb = col_pos(g, c).base;
    // the vectors' base and PE stride (the factors': fb, ps)
    const int db = MODE == 0 ? col_base(c, g.inner, g.fld_ostride) : fb;
    const int ds = MODE == 0 ? g.inner : ps;
    const float a = MODE == 2 ? (float)st->alpha_cg : 0.f;
    // the residual at pitched offset i from its inputs v (MODE 1 / 2 also update x and r there)
    auto resid = [&](int i, const float* v) {
      float rk;
      if (MODE == 0) {
        rk = v[0];
      } else if (MODE == 1) {
        rk = sign * v[0];
        x[i] = 0.f;
        r[i] = rk;
      } else {
        x[i] = first ? a * v[0] : fmaf(a, v[0], v[3]);
        rk = fmaf(-a, v[1], v[2]);
        r[i] = rk;
      }
      return rk;
    };
    // inputs at node i: r (MODE 0); grad (MODE 1); p, Hp, r, x (MODE 2)
    auto inputs = [&](int i, float* v) {
      if (MODE == 0) { v[0] = r[i]; }
      else if (MODE == 1) { v[0] = __ldg(grad + i); }
      else { v[0] = __ldg(p + i); v[1] = __ldg(Hp + i); v[2] = r[i]; v[3] = first ? 0.f : x[i]; }
    };
    auto fetch_inputs = [&](int i, int sl) {
      if (MODE == 0) {
        cp_async4(&ring[sl][1][lane], r + i, true);
      } else if (MODE == 1) {
        cp_async4(&ring[sl][1][lane], grad + i, true);
      } else {
        cp_async4(&ring[sl][1][lane], p + i, true);
        cp_async4(&ring[sl][2][lane], Hp + i, true);
        cp_async4(&ring[sl][3][lane], r + i, true);
        cp_async4(&ring[sl][4][lane], x + i, !first);
      }
    };
    // forward: y_0 = r_0, y_k = r_k - l_{k-1} y_{k-1}; step k (1 .. E - 1) reads l_{k-1} and the
    // inputs at node k
    float v0[4];
    inputs(db, v0);
    float y = resid(db, v0);
    arr += y * y;
    z[db] = y;
    auto ffetch = [&](int q) {   // steps 1 + kColGroup q .. + 3
#pragma unroll
      for (int u = 0; u < kColGroup; ++u) {
        const int k = 1 + q * kColGroup + u, kk = min(k, E - 1), sl = k % R;
        cp_async4(&ring[sl][0][lane], lco + fb + (kk - 1) * ps, true);
        fetch_inputs(db + kk * ds, sl);
      }
      cp_async_commit();
    };
    for (int q = 0; q < NG - 1; ++q) ffetch(q);
    for (int q = 0; 1 + q * kColGroup < E; ++q) {
      ffetch(q + NG - 1);
      cp_async_wait<NG - 1>();
#pragma unroll
      for (int u = 0; u < kColGroup; ++u) {   // predicated past the column's end, no branch
        const int k = 1 + q * kColGroup + u, sl = k % R, i = db + k * ds;
        if (MODE == 0 ? false : k >= E) break;   // MODE 1 / 2 write x and r in resid
        const bool in = k < E;
        float v[4];
#pragma unroll
        for (int w = 0; w < 4; ++w) v[w] = ring[sl][1 + w][lane];
        const float rk = resid(i, v);
        const float yn = fmaf(-ring[sl][0][lane], y, rk);
        if (in) {
          arr += rk * rk;
          y = yn;
          z[i] = y;
        }
      }
    }
    cp_async_wait<0>();
    __threadfence_block();   // this thread's y (in z) and r stores before its copies read them back
    // backward: z_{E-1} = y_{E-1} / D_{E-1}, z_k = y_k / D_k - l_k z_{k+1}; step t reads node
    // k = E - 2 - t: y_k, l_k, 1 / D_k (and r_k)
    float zz = y * __ldg(invD + fb + (E - 1) * ps);
    z[db + (E - 1) * ds] = zz;
    if (MODE != 0) arz += r[db + (E - 1) * ds] * zz;
    auto bfetch = [&](int q) {   // steps kColGroup q .. + 3
#pragma unroll
      for (int u = 0; u < kColGroup; ++u) {
        const int t = q * kColGroup + u, kk = max(E - 2 - t, 0), sl = t % R;
        const int i = fb + kk * ps, id = db + kk * ds;
        cp_async4(&ring[sl][0][lane], z + id, true);
        cp_async4(&ring[sl][1][lane], lco + i, true);
        cp_async4(&ring[sl][2][lane], invD + i, true);
        if (MODE != 0) cp_async4(&ring[sl][3][lane], r + id, true);
      }
      cp_async_commit();
    };
    for (int q = 0; q < NG - 1; ++q) bfetch(q);
    for (int q = 0; q * kColGroup < E - 1; ++q) {
      bfetch(q + NG - 1);
      cp_async_wait<NG - 1>();
#pragma unroll
      for (int u = 0; u < kColGroup; ++u) {   // predicated past the column's start, no branch
        const int t = q * kColGroup + u, sl = t % R, k = E - 2 - t;
        const float zn = fmaf(-ring[sl][1][lane], zz, ring[sl][0][lane] * ring[sl][2][lane]);
        if (k >= 0) {
          zz = zn;
          z[db + k * ds] = zz;
          if (MODE != 0) arz += ring[sl][3][lane] * zz;
        }
      }
    }
    cp_async_wait<0>();
  }
  if (MODE == 0) return;
  float v[2] = {arr, arz};
  double tot[2];
  if (grid_sum<2>(v, partials, counter, tot)) {
    if (MODE == 1) {
      st->rr0 = tot[0]; st->rr = tot[0]; st->rho = tot[1];
      st->pcg_iter = 0;
      st->pcg_done = !(tot[0] > 0.0);
      st->relres = tot[0] > 0.0 ? 1.0 : 0.0;
    } else {
      pcg_finish(st, tot[0], tot[1], rtol);
    }
  }
}

cudaError_t launch_col_factor(const Geo& g, const float* dco, const float* eco, float* invD,
                              float* lco, cudaStream_t s) {
  k_col_factor<<<ceil_div(g.ncols, kColBlock), kColBlock, 0, s>>>(g, dco, eco, invD, lco);
  return cudaGetLastError();
}

cudaError_t launch_col_solve(const Geo& g, int mode, const float* grad, float* x, float* r,
                             const float* p, const float* Hp, float* z, const float* invD,
                             const float* lco, int first, double rtol, float sign,
                             const Work& w, cudaStream_t s) {
  const dim3 grid(ceil_div(g.ncols, kColBlock));
#define HYSCO_COLSOLVE(M)                                                                       \
  k_col_solve<M><<<grid, kColBlock, 0, s>>>(g, grad, x, r, p, Hp, z, invD, lco, first, rtol, sign, \
                                         w.partials, w.counter, w.st);
  if (mode == 0) { HYSCO_COLSOLVE(0) }
  else if (mode == 1) { HYSCO_COLSOLVE(1) }
  else { HYSCO_COLSOLVE(2) }
#undef HYSCO_COLSOLVE
  return cudaGetLastError();
}

// ------------------------------------------------------------------------------------------

static int group_blocks(const Geo& g) { return ceil_div(g.nfp >> 2, kBlock); }

template <bool PCG>
static void hv_launch(const Geo& g, const float* z, float* p, float* Hp, const float* dco,
                      const float* eco, int first, const Work* w, cudaStream_t s) {
  float* pa = w ? w->partials : nullptr;
  unsigned* ct = w ? w->counter : nullptr;
  DevState* st = w ? w->st : nullptr;
  const int nb = group_blocks(g);
  if (g.p == 0) k_hv<0, PCG><<<nb, kBlock, 0, s>>>(g, z, p, Hp, dco, eco, first, pa, ct, st);
  else if (g.p == 1) k_hv<1, PCG><<<nb, kBlock, 0, s>>>(g, z, p, Hp, dco, eco, first, pa, ct, st);
  else k_hv<2, PCG><<<nb, kBlock, 0, s>>>(g, z, p, Hp, dco, eco, first, pa, ct, st);
}

// Hv = H_J v with v and Hv in the caller's layout and d, e in the pitched one: one node per thread
// (consecutive threads on consecutive nodes of axis 2), the same arithmetic as hv_core
template <int P>
__global__ void __launch_bounds__(kBlock)
k_hv_caller(Geo g, const float* __restrict__ v, const float* __restrict__ dco,
            const float* __restrict__ eco, float* __restrict__ Hv) {
  const int fe0 = g.fe[0], fe1 = g.fe[1], fe2 = g.fe[2], s0 = fe1 * fe2;
  for (int n = blockIdx.x * blockDim.x + threadIdx.x; n < g.nf; n += gridDim.x * blockDim.x) {
    const int row = (int)fdiv((unsigned)n, g.divfe2), i2 = n - row * fe2;
    const int i0 = (int)fdiv((unsigned)row, g.divfe1), i1 = row - i0 * fe1;
    const int pi = row * g.P2 + i2;
    const float vk = __ldg(v + n);
    const float a0m = i0 > 0 ? __ldg(v + n - s0) : vk, a0p = i0 < fe0 - 1 ? __ldg(v + n + s0) : vk;
    const float a1m = i1 > 0 ? __ldg(v + n - fe2) : vk, a1p = i1 < fe1 - 1 ? __ldg(v + n + fe2) : vk;
    const float a2m = i2 > 0 ? __ldg(v + n - 1) : vk, a2p = i2 < fe2 - 1 ? __ldg(v + n + 1) : vk;
    const float lap = g.w[0] * ((vk - a0m) + (vk - a0p)) + g.w[1] * ((vk - a1m) + (vk - a1p)) +
                      g.w[2] * ((vk - a2m) + (vk - a2p));
    const int iP = P == 0 ? i0 : (P == 1 ? i1 : i2);
    const float elo = iP > 0 ? __ldg(eco + pi - g.psP) : 0.f;
    const float zlo = P == 0 ? a0m : (P == 1 ? a1m : a2m);
    const float zhi = P == 0 ? a0p : (P == 1 ? a1p : a2p);
    Hv[n] = g.vol * (elo * zlo + __ldg(dco + pi) * vk + __ldg(eco + pi) * zhi + g.alpha * lap);
  }
}

cudaError_t launch_hessvec_caller(const Geo& g, const float* v, float* Hv, const float* dco,
                                  const float* eco, cudaStream_t s) {
  const int blocks = std::min(ceil_div(g.nf, kBlock), 148 * 8);
  if (g.p == 0) k_hv_caller<0><<<blocks, kBlock, 0, s>>>(g, v, dco, eco, Hv);
  else if (g.p == 1) k_hv_caller<1><<<blocks, kBlock, 0, s>>>(g, v, dco, eco, Hv);
  else k_hv_caller<2><<<blocks, kBlock, 0, s>>>(g, v, dco, eco, Hv);
  return cudaGetLastError();
}

cudaError_t launch_pcg_init_jacobi(const Geo& g, const float* grad, float sign, float* x, float* r,
                                   float* z, const float* invd, const Work& w, cudaStream_t s) {
  k_pcg_init_jacobi<<<group_blocks(g), kBlock, 0, s>>>(g, grad, sign, x, r, z, invd, w.partials,
                                                       w.counter, w.st);
  return cudaGetLastError();
}

cudaError_t launch_pcg_hp(const Geo& g, const float* z, float* p, float* Hp, const float* dco,
                          const float* eco, int first, const Work& w, cudaStream_t s) {
  hv_launch<true>(g, z, p, Hp, dco, eco, first, &w, s);
  return cudaGetLastError();
}

cudaError_t launch_pcg_update_jacobi(const Geo& g, float* x, float* r, const float* p,
                                     const float* Hp, float* z, const float* invd, int first,
                                     double rtol, const Work& w, cudaStream_t s) {
  k_pcg_update_jacobi<<<group_blocks(g), kBlock, 0, s>>>(g, x, r, p, Hp, z, invd, first, rtol,
                                                         w.partials, w.counter, w.st);
  return cudaGetLastError();
}

cudaError_t launch_jacobi_apply(const Geo& g, const float* r, float* z, const float* invd,
                                cudaStream_t s) {
  k_jacobi_caller<<<ceil_div(g.nf, kBlock), kBlock, 0, s>>>(g, r, z, invd);
  return cudaGetLastError();
}

cudaError_t launch_to_pitched(const Geo& g, const float* src, float* dst, cudaStream_t s) {
  k_to_pitched<<<group_blocks(g), kBlock, 0, s>>>(g, src, dst);
  return cudaGetLastError();
}

cudaError_t launch_from_pitched(const Geo& g, const float* src, float* dst, cudaStream_t s) {
  k_from_pitched<<<group_blocks(g), kBlock, 0, s>>>(g, src, dst);
  return cudaGetLastError();
}


}  // namespace hysco
