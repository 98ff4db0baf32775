// Per-cell arithmetic of the objective (Sec. 2.1, Eq. 1-3) shared by the objective kernels:
// cell positions and indices, the 1D linear image model, the barrier phi and its derivatives,
// and the in-plane neighbour columns.  Included by the translation units that evaluate J.
#pragma once

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

// the two taps are loaded only where they lie inside the column (predicated loads), 0 outside
template <typename TI>
__device__ __forceinline__ void interp(const TI* col, int inner, int m, int i, float w,
                                       float& val, float& slope) {
  const bool in0 = (unsigned)i < (unsigned)m, in1 = (unsigned)(i + 1) < (unsigned)m;
  const float I0 = in0 ? ldf(col + i * inner) : 0.0f;
  const float I1 = in1 ? ldf(col + (i + 1) * inner) : 0.0f;
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
  // phi = z^4 / q, phi' = 2 z^3 (2 - z^2) / q^2, phi'' = 2 z^2 (6 - 3 z^2 + z^4) / q^3, q = 1 - z^2
  float z2 = z * z;
  float q = (1.0f - z) * (1.0f + z);
  float iq = __fdividef(1.0f, q);
  float z2q = z2 * iq;
  f = z2 * z2q;
  df = 2.0f * z * z2q * (2.0f - z2) * iq;
  d2f = 2.0f * z2q * fmaf(z2, z2 - 3.0f, 6.0f) * (iq * iq);
}

struct CellLin {
  float r, jl, jr, dphi, psi, phi, dlt;   // dlt = delta = b_{j+1} - b_j
};

// the absent cells left of node 0 and right of node m: no residual, no barrier, delta = 0
__device__ __forceinline__ CellLin cell_zero() { return CellLin{0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f}; }

// cell arithmetic from the two images' taps at the cell's positions: I(t) = I0 + w (I1 - I0)
__device__ __forceinline__ CellLin cell_from_taps(float Ip0, float Ip1, float wp, float Im0,
                                                  float Im1, float wm, float delta,
                                                  float half_beta) {
  const float sp = Ip1 - Ip0, vp = fmaf(wp, sp, Ip0);
  const float sm = Im1 - Im0, vm = fmaf(wm, sm, Im0);
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
  q.dlt = delta;
  return q;
}

template <typename TI>
__device__ __forceinline__ CellLin cell_lin(const TI* Ipc, const TI* Imc, int inner, int m, int j,
                                            float bj, float bj1, float half_beta) {
  float tp, tm, wp, wm;
  cell_positions(bj, bj1, j, tp, tm);
  int ip = cell_index(tp, m, wp), im = cell_index(tm, m, wm);
  const bool p0 = (unsigned)ip < (unsigned)m, p1 = (unsigned)(ip + 1) < (unsigned)m;
  const bool m0 = (unsigned)im < (unsigned)m, m1 = (unsigned)(im + 1) < (unsigned)m;
  const float Ip0 = p0 ? ldf(Ipc + ip * inner) : 0.0f, Ip1 = p1 ? ldf(Ipc + (ip + 1) * inner) : 0.0f;
  const float Im0 = m0 ? ldf(Imc + im * inner) : 0.0f, Im1 = m1 ? ldf(Imc + (im + 1) * inner) : 0.0f;
  return cell_from_taps(Ip0, Ip1, wp, Im0, Im1, wm, bj1 - bj, half_beta);
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

// in-plane neighbour columns of column c, clamped: an absent neighbour is the column itself
struct ColNbrs {
  int Am, Ap, Bm, Bp;
  float nin;   // wA * (#A neighbours) + wB * (#B neighbours): in-plane part of L_kk
};

__device__ __forceinline__ ColNbrs col_nbrs(const Geo& g, int c, int own) {
  int cA = c % g.nA, cB = c / g.nA;
  ColNbrs n;
  n.Am = cA > 0 ? col_base(c - 1, g.inner, g.fld_ostride) : own;
  n.Ap = cA < g.nA - 1 ? col_base(c + 1, g.inner, g.fld_ostride) : own;
  n.Bm = cB > 0 ? col_base(c - g.nA, g.inner, g.fld_ostride) : own;
  n.Bp = cB < g.nB - 1 ? col_base(c + g.nA, g.inner, g.fld_ostride) : own;
  n.nin = g.wA * (float)((cA > 0) + (cA < g.nA - 1)) + g.wB * (float)((cB > 0) + (cB < g.nB - 1));
  return n;
}

// the same neighbours as pitched bases (solver arrays)
__device__ __forceinline__ ColNbrs col_nbrs_pitched(const Geo& g, int c, int own) {
  int cA = c % g.nA, cB = c / g.nA;
  ColNbrs n;
  n.Am = cA > 0 ? own - g.psA : own;
  n.Ap = cA < g.nA - 1 ? own + g.psA : own;
  n.Bm = cB > 0 ? own - g.psB : own;
  n.Bp = cB < g.nB - 1 ? own + g.psB : own;
  n.nin = g.wA * (float)((cA > 0) + (cA < g.nA - 1)) + g.wB * (float)((cB > 0) + (cB < g.nB - 1));
  return n;
}

}  // namespace hysco
