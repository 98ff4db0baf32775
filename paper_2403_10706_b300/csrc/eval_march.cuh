// Device bodies of the objective kernels (Sec. 2.1 Eq. 1-5, Sec. 2.3.1): the column-march
// evaluation of J, grad J and the GN coefficients, the Armijo halvings' J, and the GN update.
// Each is called by its own kernel (k_eval.cu) and by the persistent GN loop (k_gn.cu).  RO: the
// field arrays the body reads (b, q, grad) were written before the launch (read-only path);
// otherwise by the same launch, before a device-wide barrier (ordinary loads).
#pragma once

#include "eval_common.cuh"

namespace hysco {

constexpr int kEvalU = 4;           // nodes whose loads are issued together (evaluation)
constexpr int kEvalUTrial = 3;      // the same for the gamma = 1 trial (80 registers, no spill)
constexpr int kEvalUProx = 2;       // and for the prox variants (ADMM b-subproblem)

// per-thread partial sums of one objective evaluation: D, S, P (Eq. 2-4 without their factor
// vol/2), ||grad||^2, grad^T q (trial) and ||b - c||^2 (prox)
struct EvalAcc {
  float D = 0.f, S = 0.f, P = 0.f, G = 0.f, GQ = 0.f, R = 0.f;
};

// Work item `item` of the column march (item < g.ntile * g.nseg): the warp's 32 consecutive
// columns of tile item % ntile (lane = column) and the nodes of segment item / ntile.  Each
// thread walks its segment node by node with a rolling window of one cell (the cell right of
// node k is evaluated once and reused as the cell left of node k + 1); loads of U nodes are
// issued together before their arithmetic.  A lane past the last column repeats the last column
// (identical values stored to identical addresses) and adds nothing to `acc`.
// TRIAL: the evaluation at b + q (grad_p is read first for grad^T q).  PROX: the ADMM
// b-subproblem's prox term rho vol/2 ||b - c||^2 (c = cpx, pitched).  OUT bit 0: write grad in
// the caller's layout; bit 1: the pitched copy grad_p; bit 2: the field value the evaluation is
// at (b + q in the trial) into fout, caller layout.
template <typename TI, bool TRIAL, bool PROX, int U, int OUT, bool RO>
__device__ __forceinline__ void eval_item(const Geo& g, const TI* __restrict__ Ip,
                                          const TI* __restrict__ Im, const float* b,
                                          const float* q, const float* __restrict__ cpx,
                                          float* grad, float* grad_p, float* dco, float* eco,
                                          float* invd, float rho, int item, int lane,
                                          EvalAcc& acc, float* fout = nullptr) {
  const int inner = g.inner, m = g.m, psP = g.psP;
  const float wA = g.wA, wB = g.wB, alpha = g.alpha, hbeta = g.half_beta, vol = g.vol;
  float accD = 0.f, accS = 0.f, accP = 0.f, accG = 0.f, accGQ = 0.f, accR = 0.f;
  const int seg = item / g.ntile;
  {
    int c = (item - seg * g.ntile) * 32 + lane;
    const bool act = c < g.ncols;
    c = act ? c : g.ncols - 1;
    const int k0 = seg * g.mseg, k1 = min(k0 + g.mseg, g.E);
    // column geometry: caller-layout bases (image, field), pitched base, in-plane neighbours
    const int o = (int)fdiv((unsigned)c, g.divIn), ci = c - o * inner;
    const int ib = o * (int)g.img_ostride + ci, fb = o * (int)g.fld_ostride + ci;
    const int cB = (int)fdiv((unsigned)c, g.divA), cA = c - cB * g.nA;
    const bool hAm = cA > 0, hAp = cA < g.nA - 1, hBm = cB > 0, hBp = cB < g.nB - 1;
    auto fbase = [&](int cc) {
      const int oo = (int)fdiv((unsigned)cc, g.divIn);
      return oo * (int)g.fld_ostride + (cc - oo * inner);
    };
    // offsets of the neighbour columns from this one (0: absent, the node itself, so that its
    // Laplacian difference vanishes)
    const int uAm = hAm ? fbase(c - 1) - fb : 0, uAp = hAp ? fbase(c + 1) - fb : 0;
    const int uBm = hBm ? fbase(c - g.nA) - fb : 0, uBp = hBp ? fbase(c + g.nA) - fb : 0;
    const int pAm = hAm ? -g.psA : 0, pAp = hAp ? g.psA : 0;
    const int pBm = hBm ? -g.psB : 0, pBp = hBp ? g.psB : 0;
    const float nin = g.wA * (float)((int)hAm + (int)hAp) + g.wB * (float)((int)hBm + (int)hBp);
    const float dg2 = g.alpha * (2.0f + nin), dg1 = g.alpha * (1.0f + nin);
    const TI* Ipc = Ip + ib;
    const TI* Imc = Im + ib;
    // field value (b, or b + q in the trial) at caller offset uo / pitched offset po
    auto fld = [&](int uo, int po) {
      const float v = ld_in<RO>(b + uo);
      return TRIAL ? v + ld_in<RO>(q + po) : v;
    };
    auto cell = [&](int j, float bj, float bj1) {
      return cell_lin(Ipc, Imc, inner, m, j, bj, bj1, hbeta);
    };
    // node k from the cells left (P) and right (C) of it: gradient, GN coefficients, sums
    auto node = [&](int k, const CellLin& P, const CellLin& C, float bk, float bAm, float bAp,
                    float bBm, float bBp, float qk, float gpk, float ck, int uo, int po,
                    float dgk) {
      const float dAm = bk - bAm, dAp = bAp - bk, dBm = bk - bBm, dBp = bBp - bk;
      const float lap = (P.dlt - C.dlt) + wA * (dAm - dAp) + wB * (dBm - dBp);
      accS += C.dlt * C.dlt + wA * dAp * dAp + wB * dBp * dBp;
      accD += C.r * C.r;
      accP += C.phi;
      float prx = 0.f;
      if (PROX) {
        prx = bk - ck;
        accR += prx * prx;
      }
      float gsum = P.jr * P.r + C.jl * C.r + alpha * lap + hbeta * (P.dphi - C.dphi);
      if (PROX) gsum += rho * prx;
      const float gk = vol * gsum;
      float dk = P.jr * P.jr + C.jl * C.jl + P.psi + C.psi;
      if (PROX) dk += rho;
      const float ek = C.jl * C.jr - C.psi;
      const float diag = vol * (dk + dgk);
      if (TRIAL) accGQ += gpk * qk;
      if (OUT & 1) grad[uo] = gk;
      if (OUT & 2) grad_p[po] = gk;
      if (OUT & 4) fout[uo] = bk;
      dco[po] = dk;
      eco[po] = ek;
      invd[po] = diag > 0.f ? __fdividef(1.0f, diag) : 1.0f;
      accG += gk * gk;
    };

    int uo = fb + k0 * inner, po = col_pbase(g, c) + k0 * psP;
    float bk = fld(uo, po);
    float qk = TRIAL ? ld_in<RO>(q + po) : 0.f;
    CellLin P = cell_zero();
    if (k0 > 0) P = cell(k0 - 1, fld(uo - inner, po - psP), bk);
    const int kend = min(k1, m);   // nodes below kend have a cell on their right
    int k = k0;
    for (; k + U <= kend; k += U) {
      float bn[U], qn[U], bAm[U], bAp[U], bBm[U], bBp[U], gp[U], cc[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int uk = uo + u * inner, pk = po + u * psP;
        bn[u] = fld(uk + inner, pk + psP);
        qn[u] = TRIAL ? ld_in<RO>(q + pk + psP) : 0.f;
        bAm[u] = fld(uk + uAm, pk + pAm);
        bAp[u] = fld(uk + uAp, pk + pAp);
        bBm[u] = fld(uk + uBm, pk + pBm);
        bBp[u] = fld(uk + uBp, pk + pBp);
        gp[u] = TRIAL ? grad_p[pk] : 0.f;
        cc[u] = PROX ? __ldg(cpx + pk) : 0.f;
      }
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const CellLin C = cell(k + u, bk, bn[u]);
        node(k + u, P, C, bk, bAm[u], bAp[u], bBm[u], bBp[u], qk, gp[u], cc[u],
             uo + u * inner, po + u * psP, (k + u > 0) ? dg2 : dg1);
        P = C;
        bk = bn[u];
        qk = qn[u];
      }
      uo += U * inner;
      po += U * psP;
    }
    for (; k < k1; ++k) {   // the rest of the segment, and node m (no cell on its right)
      const bool cv = k < m;
      const float bn = cv ? fld(uo + inner, po + psP) : bk;
      const float qnx = (TRIAL && cv) ? ld_in<RO>(q + po + psP) : 0.f;
      const float gpk = TRIAL ? grad_p[po] : 0.f;
      const float ck = PROX ? __ldg(cpx + po) : 0.f;
      const CellLin C = cv ? cell(k, bk, bn) : cell_zero();
      node(k, P, C, bk, fld(uo + uAm, po + pAm), fld(uo + uAp, po + pAp),
           fld(uo + uBm, po + pBm), fld(uo + uBp, po + pBp), qk, gpk, ck, uo, po,
           (k > 0 && k < m) ? dg2 : dg1);
      P = C;
      bk = bn;
      qk = qnx;
      uo += inner;
      po += psP;
    }
    if (act) {
      acc.D += accD; acc.S += accS; acc.P += accP; acc.G += accG; acc.GQ += accGQ; acc.R += accR;
    }
  }
}

// The Armijo halvings' objective values J(b + gamma_t q), gamma_t = 2^-t, t = t0 .. t0 + T - 1,
// over work items vb, vb + nvb, ... (kBlock columns x SEG nodes each; lane = column within the
// item), accumulated into aD, aS, aP (and aR with PROX) per trial; t0 = 0 also adds grad^T q to
// agq.
template <typename TI, int SEG, int T, bool PROX, bool RO>
__device__ __forceinline__ void ls_items(const Geo& g, const TI* __restrict__ Ip,
                                         const TI* __restrict__ Im, const float* b,
                                         const float* q, const float* __restrict__ cpx,
                                         const float* grad, int t0, int vb, int nvb, int lane,
                                         float (&aD)[T], float (&aS)[T], float (&aP)[T],
                                         float (&aR)[T], float& agq) {
  const int inner = g.inner, m = g.m;
  const int ncb = ceil_div(g.ncols, kBlock), nitems = ncb * ceil_div(g.E, SEG);
  // grid-stride over work items (256 columns x SEG nodes); accumulators carry across items
  for (int item = vb; item < nitems; item += nvb) {
  int c = (item % ncb) * kBlock + lane;
  const bool act = c < g.ncols;
  c = act ? c : g.ncols - 1;
  const int k0 = (item / ncb) * SEG;
  const int ib = col_base(c, inner, g.img_ostride), fb = col_base(c, inner, g.fld_ostride);
  const TI* Ipc = Ip + ib;
  const TI* Imc = Im + ib;
  const ColNbrs nb = col_nbrs(g, c, fb);
  const int pb = col_pbase(g, c);
  const ColNbrs nq = col_nbrs_pitched(g, c, pb);   // q and grad are pitched solver arrays
  float bw[SEG + 1], qw[SEG + 1], bAp[SEG], qAp[SEG], bBp[SEG], qBp[SEG], cw[SEG];
#pragma unroll
  for (int j = 0; j <= SEG; ++j) {
    int kk = min(k0 + j, m);
    bw[j] = ld_in<RO>(b + fb + kk * inner);
    qw[j] = ld_in<RO>(q + pb + kk * g.psP);
    if (PROX && j < SEG) cw[j] = __ldg(cpx + pb + kk * g.psP);
  }
#pragma unroll
  for (int j = 0; j < SEG; ++j) {
    int kk = min(k0 + j, m);
    int o = kk * inner, op = kk * g.psP;
    bAp[j] = ld_in<RO>(b + nb.Ap + o); qAp[j] = ld_in<RO>(q + nq.Ap + op);
    bBp[j] = ld_in<RO>(b + nb.Bp + o); qBp[j] = ld_in<RO>(q + nq.Bp + op);
  }
  if (t0 == 0) {
#pragma unroll
    for (int j = 0; j < SEG; ++j)
      if (act && k0 + j <= m) agq += ld_in<RO>(grad + pb + (k0 + j) * g.psP) * qw[j];
  }
#pragma unroll
  for (int t = 0; t < T; ++t) {
    float gam = ldexpf(1.0f, -(t0 + t));
    float x[SEG + 1];
#pragma unroll
    for (int j = 0; j <= SEG; ++j) x[j] = fmaf(gam, qw[j], bw[j]);
#pragma unroll
    for (int j = 0; j < SEG; ++j) {
      int k = k0 + j;
      if (!act || k > m) continue;
      float r = 0.f, phi = 0.f;
      cell_residual(Ipc, Imc, inner, m, k, x[j], x[j + 1], r, phi);
      if (k < m) { aD[t] += r * r; aP[t] += phi; }
      float dPE = x[j + 1] - x[j];
      float dA = fmaf(gam, qAp[j], bAp[j]) - x[j], dB = fmaf(gam, qBp[j], bBp[j]) - x[j];
      aS[t] += dPE * dPE + g.wA * dA * dA + g.wB * dB * dB;
      if (PROX) aR[t] += (x[j] - cw[j]) * (x[j] - cw[j]);
    }
  }
  }   // work items
}

// b += gam q over the caller-layout nodes gtid, gtid + T, ... (q pitched); UN nodes' loads in
// flight per thread
template <bool RO, int UN = 4>
__device__ __forceinline__ void update_nodes(const Geo& g, float* b, const float* q, float gam,
                                             int gtid, int T) {
  // lanes walk consecutive caller-layout nodes (coalesced b); q's pitched index by one division
  for (int i0 = gtid; i0 < g.nf; i0 += UN * T) {
    float bv[UN], qv[UN];
    int idx[UN];
#pragma unroll
    for (int u = 0; u < UN; ++u) {
      int i = min(i0 + u * T, g.nf - 1);
      int row = (int)fdiv((unsigned)i, g.divfe2);
      idx[u] = i;
      bv[u] = b[i];
      qv[u] = ld_in<RO>(q + row * g.P2 + (i - row * g.fe[2]));
    }
#pragma unroll
    for (int u = 0; u < UN; ++u)
      if (i0 + u * T < g.nf) b[idx[u]] = fmaf(gam, qv[u], bv[u]);
  }
}

}  // namespace hysco
