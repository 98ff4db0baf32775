// Objective kernels: J(b) = D + alpha S + beta P with gradient and Gauss-Newton coefficients
// (Sec. 2.1 Eq. 1-5, Sec. 2.3.1), the Armijo line search, the GN update, the corrected images
// (Sec. 2.4) and the interpolation cell indices.
//
// Thread mapping ("column march"): thread = (PE column c, segment of kSeg nodes along PE).
// Consecutive threads own consecutive columns, so for pe_dim != 2 every PE step is a coalesced
// row access.  The segment loop is fully unrolled with no serialising branches: field indices are
// clamped into range and absent neighbours are read at the node itself (zero Laplacian
// difference); an interpolation tap outside the image is a predicated-off load that reads 0.  So
// a thread issues all of its field loads, then all of its image gathers.
// Per cell j (nodes j, j+1):
//   bc = (b_j + b_{j+1}) / 2, delta = b_{j+1} - b_j, t+- = j +- bc      (averaging / FD operators)
//   I(t) = I[i] + w (I[i+1] - I[i]), i = floor(t), w = t - i, I = 0 outside 0..m-1
//   T+ = I+(t+)(1 + delta), T- = I-(t-)(1 - delta), r = T+ - T-         (Eq. 1)
//   a = I+'(1 + delta) + I-'(1 - delta), c = I+(t+) + I-(t-);  dr/db_j = a/2 - c, dr/db_{j+1} = a/2 + c
// Per node k the Gauss-Newton Hessian restricted to the column is tridiagonal:
//   d_k = (dr_{k-1}/db_k)^2 + (dr_k/db_k)^2 + psi_{k-1} + psi_k,   e_k = dr_k/db_k * dr_k/db_{k+1} - psi_k
// with psi = beta/2 phi''(delta); H v = vol [e_{k-1} v_{k-1} + d_k v_k + e_k v_{k+1} + alpha (L v)_k],
// and the Jacobi preconditioner is 1 / (vol [d_k + alpha L_kk]).
#include <algorithm>

#include "eval_common.cuh"

namespace hysco {

// ------------------------------------------------------------------------------------------
// J, grad J, the tridiagonal GN coefficients (d, e) and the inverse Jacobi diagonal
// ------------------------------------------------------------------------------------------

// TRIAL = false: evaluation at b (GN iteration `it`, or it = -1 for a single hysco_eval call, or
// it = -2 for a fresh evaluation that a stopped run skips).  In a
// solve, when the previous gamma = 1 trial was accepted the coefficients at this iterate are
// already in place: one thread promotes the stashed terms and every block returns at once (no
// block enters the reduction, so the ticket counter is untouched).
// TRIAL = true: the gamma = 1 Armijo trial, an evaluation at b + q.
// Each thread keeps only the previous cell (rolling window); the in-plane neighbours along the
// column index's fast axis A are the adjacent lanes (warp shuffle; an edge lane loads).
// PROX (the ADMM b-subproblem of Sec. 2.3.2): J gains rho vol/2 ||b - c||^2 (c pitched, rho the
// device state's admm_rho), the gradient rho vol (b - c) and the GN coefficient d the constant rho;
// with the split geometry (in-plane Laplacian weights 0) S is the PE part S3 alone.
template <typename TI, int SEG, bool TRIAL, bool PROX>
__global__ void __launch_bounds__(kBlock)
k_eval(Geo g, const TI* __restrict__ Ip, const TI* __restrict__ Im, const float* __restrict__ b,
       const float* __restrict__ q, const float* __restrict__ cpx, float* __restrict__ grad,
       float* __restrict__ grad_p, float* __restrict__ dco, float* __restrict__ eco,
       float* __restrict__ invd, int it, int ls_max, double c1, float* partials,
       unsigned* counter, DevState* st) {
  if (TRIAL) {
    if (st->stop || st->ls_done) return;
  } else if (it >= 0) {
    if (st->stop) return;
    if (st->coef_fresh) {
      if (blockIdx.x == 0 && blockIdx.y == 0 && threadIdx.x == 0) {
        st->J = st->Jn; st->D = st->Dn; st->S = st->Sn; st->P = st->Pn;
        if (PROX) st->Jacc = st->Jn;
        st->gnorm = st->gnorm_n;
        st->status = st->status_n;
        st->ls_done = 0; st->ls_trials = 0; st->gamma = 0.0; st->gq = 0.0;
        st->pcg_done = 0; st->pcg_iter = 0; st->relres = 0.0;
      }
      return;
    }
  } else if (it < -1 && st->stop) {
    return;   // it = -2: a fresh evaluation unless the run has stopped
  }
  const int inner = g.inner, m = g.m;
  const int lane = threadIdx.x & 31;
  const int ncb = ceil_div(g.ncols, kBlock), nitems = ncb * ceil_div(g.E, SEG);
  const float rho = PROX ? st->admm_rho : 0.f;
  float accD = 0.f, accS = 0.f, accP = 0.f, accG = 0.f, accGQ = 0.f, accR = 0.f;
  // grid-stride over work items (256 columns x SEG nodes); accumulators carry across items
  for (int item = blockIdx.x; item < nitems; item += gridDim.x) {
  int c = (item % ncb) * kBlock + threadIdx.x;
  const bool act = c < g.ncols;
  c = act ? c : g.ncols - 1;
  const int k0 = (item / ncb) * SEG;
  const int ib = col_base(c, inner, g.img_ostride), fb = col_base(c, inner, g.fld_ostride);
  const TI* Ipc = Ip + ib;
  const TI* Imc = Im + ib;
  const ColNbrs nb = col_nbrs(g, c, fb);
  const int pb = col_pbase(g, c);
  const ColNbrs nq = col_nbrs_pitched(g, c, pb);
  const int cA = c % g.nA;
  const bool hasAm = cA > 0, hasAp = cA < g.nA - 1;
  // field value at user offset uo / pitched offset po (b, or b + q in the trial)
  auto fld = [&](int uo, int po) {
    float v = __ldg(b + uo);
    return TRIAL ? fmaf(1.0f, __ldg(q + po), v) : v;
  };

  // column nodes k0-1 .. k0+SEG (clamped to [0, m]); B neighbours of k0 .. k0+SEG-1 by loads,
  // A neighbours from the lanes beside (edge lanes load)
  float bw[SEG + 2], bBm[SEG], bBp[SEG], eAm[SEG], eAp[SEG];
#pragma unroll
  for (int j = 0; j < SEG + 2; ++j) {
    int kk = min(max(k0 - 1 + j, 0), m);
    bw[j] = fld(fb + kk * inner, pb + kk * g.psP);
  }
#pragma unroll
  for (int j = 0; j < SEG; ++j) {
    int kk = min(k0 + j, m);
    int o = kk * inner, op = kk * g.psP;
    bBm[j] = fld(nb.Bm + o, nq.Bm + op);
    bBp[j] = fld(nb.Bp + o, nq.Bp + op);
    eAm[j] = (lane == 0 && hasAm) ? fld(nb.Am + o, nq.Am + op) : 0.f;
    eAp[j] = (lane == 31 && hasAp) ? fld(nb.Ap + o, nq.Ap + op) : 0.f;
  }
  // grad^T q with the gradient at b (trial only), loaded before this thread overwrites it
  if (TRIAL) {
#pragma unroll
    for (int j = 0; j < SEG; ++j) {
      int kk = min(k0 + j, m);
      float gv = grad_p[pb + kk * g.psP], qv = __ldg(q + pb + kk * g.psP);
      accGQ += (act && k0 + j <= m) ? gv * qv : 0.f;
    }
  }
  // the cell left of node k0 (cell k0 - 1)
  float pr, pjr, pdphi, ppsi;
  {
    CellLin cl = cell_lin(Ipc, Imc, inner, m, k0 - 1, bw[0], bw[1], g.half_beta);
    bool cv = k0 >= 1;
    pr = cv ? cl.r : 0.f; pjr = cv ? cl.jr : 0.f;
    pdphi = cv ? cl.dphi : 0.f; ppsi = cv ? cl.psi : 0.f;
  }
#pragma unroll
  for (int j = 0; j < SEG; ++j) {
    const int k = k0 + j;
    // the cell right of node k (cell k)
    CellLin cl = cell_lin(Ipc, Imc, inner, m, k, bw[j + 1], bw[j + 2], g.half_beta);
    const bool cv = k < m;
    const float cr = cv ? cl.r : 0.f, cjl = cv ? cl.jl : 0.f, cjr = cv ? cl.jr : 0.f;
    const float cdphi = cv ? cl.dphi : 0.f, cpsi = cv ? cl.psi : 0.f, cphi = cv ? cl.phi : 0.f;
    const float bk = bw[j + 1], bn = bw[j + 2];
    const float fromL = __shfl_up_sync(0xffffffffu, bk, 1);
    const float fromR = __shfl_down_sync(0xffffffffu, bk, 1);
    const float bAm = hasAm ? (lane > 0 ? fromL : eAm[j]) : bk;
    const float bAp = hasAp ? (lane < 31 ? fromR : eAp[j]) : bk;
    if (act && k <= m) {
      float lap = (bk - bw[j]) + (bk - bn) + g.wA * ((bk - bAm) + (bk - bAp)) +
                  g.wB * ((bk - bBm[j]) + (bk - bBp[j]));
      float dPE = bn - bk, dA = bAp - bk, dB = bBp[j] - bk;
      accS += dPE * dPE + g.wA * dA * dA + g.wB * dB * dB;
      accD += cr * cr;
      accP += cphi;
      const int pi = pb + k * g.psP;   // solver arrays are pitched
      float prx = 0.f;
      if (PROX) {
        prx = bk - __ldg(cpx + pi);
        accR += prx * prx;
      }
      float gsum = pjr * pr + cjl * cr + g.alpha * lap + g.half_beta * (pdphi - cdphi);
      if (PROX) gsum += rho * prx;
      float gk = g.vol * gsum;
      float dk = pjr * pjr + cjl * cjl + ppsi + cpsi;
      if (PROX) dk += rho;
      float ek = cjl * cjr - cpsi;
      float npe = (float)((k > 0) + (k < m));
      float diag = g.vol * (dk + g.alpha * (npe + nb.nin));
      if (grad) grad[fb + k * inner] = gk;
      if (grad_p) grad_p[pi] = gk;
      dco[pi] = dk;
      eco[pi] = ek;
      invd[pi] = diag > 0.f ? __fdividef(1.0f, diag) : 1.0f;
      accG += gk * gk;
    }
    pr = cr; pjr = cjr; pdphi = cdphi; ppsi = cpsi;
  }
  }   // work items
  constexpr int NV = PROX ? 6 : 5;
  float v[NV];
  v[0] = accD; v[1] = accS; v[2] = accP; v[3] = accG; v[4] = accGQ;
  if (PROX) v[NV - 1] = accR;
  double tot[NV];
  if (grid_sum<NV>(v, partials, counter, tot)) {
    double hv = 0.5 * (double)g.vol;
    double D = hv * tot[0], S = hv * tot[1], P = hv * tot[2];
    double J = D + g.alpha_d * S + g.beta_d * P;
    if (PROX) {
      st->prox = hv * tot[NV - 1];
      J += (double)rho * st->prox;
    }
    if (!TRIAL) {
      st->J = J; st->D = D; st->S = S; st->P = P;
      if (PROX) st->Jacc = J;
      st->gnorm = sqrt(tot[3]);
      st->status = isnan(J) ? -4 : (isinf(J) ? 1 : 0);
      st->ls_done = 0; st->ls_trials = 0; st->gamma = 0.0; st->gq = 0.0;
      st->pcg_done = 0; st->pcg_iter = 0; st->relres = 0.0;
      st->coef_fresh = 0;
      if (it >= 0 && !isfinite(J)) { st->stop = 1; st->stop_iter = it; }
    } else {
      double gq = tot[4];
      st->gq = gq;
      st->coef_fresh = 0;
      if (!(gq < 0.0)) {             // not a descent direction: keep the iterate
        st->ls_done = 1; st->gamma = 0.0; st->ls_trials = 0;
      } else {
        st->ls_trials = 1;
        if (J <= st->J + c1 * gq) {  // Armijo with gamma = 1
          st->ls_done = 1; st->gamma = 1.0;
          if (PROX) st->Jacc = J;
          st->coef_fresh = 1;
          st->Jn = J; st->Dn = D; st->Sn = S; st->Pn = P;
          st->gnorm_n = sqrt(tot[3]);
          st->status_n = 0;
        } else if (ls_max <= 1) {
          st->ls_done = 1; st->gamma = 0.0;
        }
      }
    }
  }
}

// ------------------------------------------------------------------------------------------
// Armijo line search: J(b + gamma_t q) for gamma_t = 2^-t, t = t0 .. t0+T-1, in one pass; the
// first accepted trial in order wins, exactly as sequential halving would pick it.  The first
// gamma = 1 trial is a full evaluation (launch_eval_trial); this kernel tries the halvings.
// ------------------------------------------------------------------------------------------

template <typename TI, int SEG, int T, bool PROX>
__global__ void __launch_bounds__(kBlock)
k_linesearch(Geo g, const TI* __restrict__ Ip, const TI* __restrict__ Im,
             const float* __restrict__ b, const float* __restrict__ q,
             const float* __restrict__ cpx, const float* __restrict__ grad, int t0, int ls_max,
             double c1, float* partials, unsigned* counter, DevState* st) {
  if (st->stop || st->ls_done) return;
  const int inner = g.inner, m = g.m;
  const int ncb = ceil_div(g.ncols, kBlock), nitems = ncb * ceil_div(g.E, SEG);
  float aD[T], aS[T], aP[T], aR[T], agq = 0.f;
#pragma unroll
  for (int t = 0; t < T; ++t) { aD[t] = 0.f; aS[t] = 0.f; aP[t] = 0.f; aR[t] = 0.f; }
  // grid-stride over work items (256 columns x SEG nodes); accumulators carry across items
  for (int item = blockIdx.x; item < nitems; item += gridDim.x) {
  int c = (item % ncb) * kBlock + threadIdx.x;
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
    bw[j] = __ldg(b + fb + kk * inner);
    qw[j] = __ldg(q + pb + kk * g.psP);
    if (PROX && j < SEG) cw[j] = __ldg(cpx + pb + kk * g.psP);
  }
#pragma unroll
  for (int j = 0; j < SEG; ++j) {
    int kk = min(k0 + j, m);
    int o = kk * inner, op = kk * g.psP;
    bAp[j] = __ldg(b + nb.Ap + o); qAp[j] = __ldg(q + nq.Ap + op);
    bBp[j] = __ldg(b + nb.Bp + o); qBp[j] = __ldg(q + nq.Bp + op);
  }
  if (t0 == 0) {
#pragma unroll
    for (int j = 0; j < SEG; ++j)
      if (act && k0 + j <= m) agq += __ldg(grad + pb + (k0 + j) * g.psP) * qw[j];
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
  constexpr int NV = (PROX ? 4 : 3) * T + 1;
  float v[NV];
  double tot[NV];
#pragma unroll
  for (int t = 0; t < T; ++t) {
    v[3 * t] = aD[t]; v[3 * t + 1] = aS[t]; v[3 * t + 2] = aP[t];
    if (PROX) v[3 * T + 1 + t] = aR[t];
  }
  v[3 * T] = agq;
  if (grid_sum<NV>(v, partials, counter, tot)) {
    if (t0 == 0) st->gq = tot[3 * T];
    double gq = st->gq, J = st->J, hv = 0.5 * (double)g.vol;
    if (!(gq < 0.0)) { st->ls_done = 1; st->gamma = 0.0; st->ls_trials = 0; return; }
    for (int t = 0; t < T && t0 + t < ls_max; ++t) {
      double gm = ldexp(1.0, -(t0 + t));
      double Jt = hv * tot[3 * t] + g.alpha_d * hv * tot[3 * t + 1] + g.beta_d * hv * tot[3 * t + 2];
      if (PROX) Jt += (double)st->admm_rho * hv * tot[3 * T + 1 + t];
      st->ls_trials = t0 + t + 1;
      if (Jt <= J + c1 * gm * gq) {
        st->ls_done = 1; st->gamma = gm;
        if (PROX) st->Jacc = Jt;
        return;
      }
    }
    if (t0 + T >= ls_max) { st->ls_done = 1; st->gamma = 0.0; }
  }
}

// b += gamma q (b in the caller's layout, q pitched); block 0 records the iteration's statistics
__global__ void __launch_bounds__(kBlock)
k_update(Geo g, float* __restrict__ b, const float* __restrict__ q, int it, double* stats,
         DevState* st) {
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    const double nan = __longlong_as_double(0x7ff8000000000000LL);
    bool stopped_before = st->stop && st->stop_iter < it;
    bool stopped_now = st->stop && st->stop_iter == it;
    if (stats) {
      double* row = stats + it * 10;
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
  const float gam = (float)st->gamma;
  if (gam == 0.0f) return;
  // lanes walk consecutive caller-layout nodes (coalesced b); q's pitched index by one division
  const int T = gridDim.x * blockDim.x;
  for (int i0 = blockIdx.x * blockDim.x + threadIdx.x; i0 < g.nf; i0 += 4 * T) {
    float bv[4], qv[4];
    int idx[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      int i = min(i0 + u * T, g.nf - 1);
      int row = (int)fdiv((unsigned)i, g.divfe2);
      idx[u] = i;
      bv[u] = b[i];
      qv[u] = __ldg(q + row * g.P2 + (i - row * g.fe[2]));
    }
#pragma unroll
    for (int u = 0; u < 4; ++u)
      if (i0 + u * T < g.nf) b[idx[u]] = fmaf(gam, qv[u], bv[u]);
  }
}

// corrected images T+ = I+(t+)(1 + delta), T- = I-(t-)(1 - delta)
template <typename TI>
__global__ void __launch_bounds__(kBlock)
k_correct(Geo g, const TI* __restrict__ Ip, const TI* __restrict__ Im, const float* __restrict__ b,
          float* __restrict__ Tp, float* __restrict__ Tm) {
  const int seg = kSeg;
  int c = blockIdx.x * blockDim.x + threadIdx.x;
  int j0 = blockIdx.y * seg, j1 = min(j0 + seg, g.m);
  if (c >= g.ncols) return;
  const int inner = g.inner, m = g.m;
  int ib = col_base(c, inner, g.img_ostride), fb = col_base(c, inner, g.fld_ostride);
  float bj = j0 < j1 ? __ldg(b + fb + j0 * inner) : 0.f;
  for (int j = j0; j < j1; ++j) {
    float bn = __ldg(b + fb + (j + 1) * inner);
    float tp, tm, wp, wm, vp, sp, vm, sm;
    cell_positions(bj, bn, j, tp, tm);
    int ip = cell_index(tp, m, wp), im = cell_index(tm, m, wm);
    interp(Ip + ib, inner, m, ip, wp, vp, sp);
    interp(Im + ib, inner, m, im, wm, vm, sm);
    float delta = bn - bj;
    Tp[ib + j * inner] = vp * (1.0f + delta);
    Tm[ib + j * inner] = vm * (1.0f - delta);
    bj = bn;
  }
}

__global__ void __launch_bounds__(kBlock)
k_cells(Geo g, const float* __restrict__ b, int* __restrict__ cp, int* __restrict__ cm) {
  const int seg = kSeg;
  int c = blockIdx.x * blockDim.x + threadIdx.x;
  int j0 = blockIdx.y * seg, j1 = min(j0 + seg, g.m);
  if (c >= g.ncols) return;
  int ib = col_base(c, g.inner, g.img_ostride), fb = col_base(c, g.inner, g.fld_ostride);
  for (int j = j0; j < j1; ++j) {
    float tp, tm, wp, wm;
    cell_positions(__ldg(b + fb + j * g.inner), __ldg(b + fb + (j + 1) * g.inner),
                   j, tp, tm);
    cp[ib + j * g.inner] = cell_index(tp, g.m, wp);
    cm[ib + j * g.inner] = cell_index(tm, g.m, wm);
  }
}

__global__ void k_publish_terms(double* terms, const DevState* st) {
  terms[0] = st->J; terms[1] = st->D; terms[2] = st->S; terms[3] = st->P;
}

// ------------------------------------------------------------------------------------------

static dim3 march_grid(const Geo& g, int nodes) {
  return dim3(ceil_div(g.ncols, kBlock), ceil_div(nodes, kSeg));
}

// grid of the grid-stride march kernels (eval, trial, halvings): per_sm blocks per SM (their
// occupancy: 4 for the evaluations at 64 registers, 2 for the 9-trial halving pass at 128), at
// most one per work item.  An early-returning launch then costs one short wave.
static dim3 resident_grid(const Geo& g, int per_sm = 4) {
  static int sms = 0;
  if (sms == 0) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
      sms = 148;
  }
  const int items = ceil_div(g.ncols, kBlock) * ceil_div(g.E, kSeg);
  return dim3(std::min(items, sms * per_sm));
}

#define HYSCO_DISPATCH(dtype, T, ...)                                                  \
  switch (dtype) {                                                                     \
    case 0: { using T = float; __VA_ARGS__; break; }                                   \
    case 1: { using T = __nv_bfloat16; __VA_ARGS__; break; }                           \
    default: { using T = __half; __VA_ARGS__; break; }                                 \
  }

cudaError_t launch_eval(const Geo& g, int dtype, const void* Ip, const void* Im, const float* b,
                        float* grad, float* grad_p, float* dco, float* eco, float* invd, int it,
                        const Work& w, cudaStream_t s, const float* cpx) {
  if (cpx) {
    HYSCO_DISPATCH(dtype, T,
      (k_eval<T, kSeg, false, true><<<resident_grid(g), kBlock, 0, s>>>(
          g, (const T*)Ip, (const T*)Im, b, nullptr, cpx, grad, grad_p, dco, eco, invd, it, 0,
          0.0, w.partials, w.counter, w.st)))
  } else {
    HYSCO_DISPATCH(dtype, T,
      (k_eval<T, kSeg, false, false><<<resident_grid(g), kBlock, 0, s>>>(
          g, (const T*)Ip, (const T*)Im, b, nullptr, nullptr, grad, grad_p, dco, eco, invd, it,
          0, 0.0, w.partials, w.counter, w.st)))
  }
  return cudaGetLastError();
}

cudaError_t launch_eval_trial(const Geo& g, int dtype, const void* Ip, const void* Im,
                              const float* b, const float* q, float* grad_p, float* dco,
                              float* eco, float* invd, int ls_max, double c1, const Work& w,
                              cudaStream_t s, const float* cpx) {
  if (cpx) {
    HYSCO_DISPATCH(dtype, T,
      (k_eval<T, kSeg, true, true><<<resident_grid(g), kBlock, 0, s>>>(
          g, (const T*)Ip, (const T*)Im, b, q, cpx, nullptr, grad_p, dco, eco, invd, 0, ls_max,
          c1, w.partials, w.counter, w.st)))
  } else {
    HYSCO_DISPATCH(dtype, T,
      (k_eval<T, kSeg, true, false><<<resident_grid(g), kBlock, 0, s>>>(
          g, (const T*)Ip, (const T*)Im, b, q, nullptr, nullptr, grad_p, dco, eco, invd, 0,
          ls_max, c1, w.partials, w.counter, w.st)))
  }
  return cudaGetLastError();
}

template <bool PROX>
static void linesearch_impl(const Geo& g, int dtype, const void* Ip, const void* Im,
                            const float* b, const float* q, const float* cpx, const float* grad,
                            int t0, int ls_max, double c1, const Work& w, cudaStream_t s) {
  if (t0 == 0) {
    HYSCO_DISPATCH(dtype, T,
      (k_linesearch<T, kSeg, 1, PROX><<<resident_grid(g), kBlock, 0, s>>>(
          g, (const T*)Ip, (const T*)Im, b, q, cpx, grad, t0, ls_max, c1, w.partials,
          w.counter, w.st)))
  } else {
    HYSCO_DISPATCH(dtype, T,
      (k_linesearch<T, kSeg, kLsBatch, PROX><<<resident_grid(g, 2), kBlock, 0, s>>>(
          g, (const T*)Ip, (const T*)Im, b, q, cpx, grad, t0, ls_max, c1, w.partials,
          w.counter, w.st)))
  }
}

cudaError_t launch_linesearch(const Geo& g, int dtype, const void* Ip, const void* Im,
                              const float* b, const float* q, const float* grad, int t0,
                              int ls_max, double c1, const Work& w, cudaStream_t s,
                              const float* cpx) {
  if (cpx) linesearch_impl<true>(g, dtype, Ip, Im, b, q, cpx, grad, t0, ls_max, c1, w, s);
  else linesearch_impl<false>(g, dtype, Ip, Im, b, q, nullptr, grad, t0, ls_max, c1, w, s);
  return cudaGetLastError();
}

cudaError_t launch_update(const Geo& g, float* b, const float* q, int it, double* stats,
                          const Work& w, cudaStream_t s) {
  int blocks = ceil_div(g.nf, 4 * kBlock);
  if (blocks > 148 * 8) blocks = 148 * 8;
  k_update<<<blocks, kBlock, 0, s>>>(g, b, q, it, stats, w.st);
  return cudaGetLastError();
}

cudaError_t launch_correct(const Geo& g, int dtype, const void* Ip, const void* Im,
                           const float* b, float* Tp, float* Tm, cudaStream_t s) {
  HYSCO_DISPATCH(dtype, T,
    (k_correct<T><<<march_grid(g, g.m), kBlock, 0, s>>>(g, (const T*)Ip, (const T*)Im, b, Tp,
                                                         Tm)))
  return cudaGetLastError();
}

cudaError_t launch_cells(const Geo& g, const float* b, int* cp, int* cm, cudaStream_t s) {
  k_cells<<<march_grid(g, g.m), kBlock, 0, s>>>(g, b, cp, cm);
  return cudaGetLastError();
}

cudaError_t launch_publish_terms(double* terms, const Work& w, cudaStream_t s) {
  k_publish_terms<<<1, 1, 0, s>>>(terms, w.st);
  return cudaGetLastError();
}

}  // namespace hysco
