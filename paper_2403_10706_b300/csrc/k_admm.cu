// ADMM of Sec. 2.3.2 on the device: the b-update's column-parallel CG (BlockPCG), the z-update
// by the real Fourier basis of the periodic in-plane Laplacian, and the multiplier / rho
// bookkeeping of every iteration.
//
// Splitting (Sec. 2.3.2): F(b) = D + alpha S3 + beta P (S3 the PE part of S) and G(z) = alpha
// (S1 + S2) (the in-plane parts), constraint b = z, scaled multiplier u.  The b-update minimises
// F(b) + rho vol/2 ||b - z + u||^2 by Gauss-Newton whose directions come from BlockPCG: that
// subproblem has no in-plane coupling, so its GN Hessian is block diagonal with one tridiagonal
// block per PE column, and every column runs its own Jacobi CG with its own step sizes and stop.
// The z-update solves (alpha H_G + rho I) z = rho (b + u) with H_G the in-plane Laplacian under
// periodic ends, which is block circulant with circulant blocks in every PE plane and so is
// diagonalised by the 2D discrete Fourier transform.  The transform is applied here in its real
// orthonormal form: Q_n holds, for every frequency j of the length-n DFT, the cosine and sine
// columns (one column for j = 0 and, for even n, for j = n/2), all real, Q_n^T Q_n = I, and the
// periodic second difference has eigenvalue 2 - 2 cos(2 pi j / n) on both columns of frequency j.
// Per plane X (nB x nA): z = Q_B [ (Q_B^T X Q_A) .* rho / lambda ] Q_A^T with
// lambda(jB, jA) = rho + alpha (wB mu_B(jB) + wA mu_A(jA)): four small dense products per plane.
#include <algorithm>

#include "hysco_internal.cuh"

namespace hysco {

// ------------------------------------------------------------------------------------------
// BlockPCG: one warp per PE column, lane l holding nodes k = 32 j + l (j < J) in registers.
// ------------------------------------------------------------------------------------------

__device__ __forceinline__ float warp_sum_bfly(float v) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
  return v;
}

// v at node k - 1 and k + 1 of the lane's nodes (0 beyond the column's ends: the caller keeps
// the entries of nodes past m at 0)
template <int J>
__device__ __forceinline__ void neighbours(const float (&v)[J], int lane, float (&vl)[J],
                                           float (&vr)[J]) {
#pragma unroll
  for (int j = 0; j < J; ++j) {
    const float up = __shfl_up_sync(0xffffffffu, v[j], 1);
    const float dn = __shfl_down_sync(0xffffffffu, v[j], 1);
    const float from_prev = __shfl_sync(0xffffffffu, v[j > 0 ? j - 1 : 0], 31);
    const float from_next = __shfl_sync(0xffffffffu, v[j < J - 1 ? j + 1 : J - 1], 0);
    vl[j] = lane > 0 ? up : (j > 0 ? from_prev : 0.f);
    vr[j] = lane < 31 ? dn : (j < J - 1 ? from_next : 0.f);
  }
}

// x = the per-column Jacobi CG solution of H_c x = rhs_sign * rhs (rhs_sign = -1 with the
// gradient as rhs for a GN direction), H_c = vol [tridiag(e_{k-1}, d_k, e_k)
// + alpha L_pe] (d carries rho, L_pe the 1D Neumann second difference along PE), as in Sec. 2.3.1
// per column: x0 = 0, stop after an update when ||r|| / ||r0|| < rtol, or when p^T H p <= 0, or
// after max_it iterations.  Dot products: each lane sums its nodes in j order, then a fixed
// butterfly across the warp (every lane holds the same value, so the column's decisions are
// uniform).  The iterations taken are added to st->blk_iters.
template <int J>
__global__ void __launch_bounds__(kBlock)
k_block_pcg(Geo g, const float* __restrict__ rhs, float rhs_sign, const float* __restrict__ dco,
            const float* __restrict__ eco, const float* __restrict__ invd,
            float* __restrict__ x, int max_it, float rtol, DevState* st) {
  if (st->stop) return;
  const int lane = threadIdx.x & 31;
  const int c = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (c >= g.ncols) return;   // whole warps only
  const int m = g.m;
  const int pb = col_pbase(g, c);
  const float vol = g.vol, alpha = g.alpha;
  float d[J], e[J], em[J], di[J], npe[J], r[J], p[J], xv[J];
  bool ok[J];
#pragma unroll
  for (int j = 0; j < J; ++j) {
    const int k = 32 * j + lane;
    ok[j] = k <= m;
    const int kk = ok[j] ? k : m;
    const int pi = pb + kk * g.psP;
    d[j] = ok[j] ? __ldg(dco + pi) : 0.f;
    e[j] = ok[j] ? __ldg(eco + pi) : 0.f;
    di[j] = ok[j] ? __ldg(invd + pi) : 0.f;
    r[j] = ok[j] ? rhs_sign * __ldg(rhs + pi) : 0.f;
    npe[j] = (float)((k > 0) + (k < m));
    xv[j] = 0.f;
  }
  {
    float er[J];
    neighbours<J>(e, lane, em, er);   // em = e_{k-1}
  }
  float rr0 = 0.f;
#pragma unroll
  for (int j = 0; j < J; ++j) rr0 += r[j] * r[j];
  rr0 = warp_sum_bfly(rr0);
  int it = 0;
  if (rr0 > 0.f) {
    float rz = 0.f;
#pragma unroll
    for (int j = 0; j < J; ++j) {
      p[j] = r[j] * di[j];
      rz += r[j] * p[j];
    }
    rz = warp_sum_bfly(rz);
    for (int i = 0; i < max_it; ++i) {
      float pl[J], pr[J], Hp[J];
      neighbours<J>(p, lane, pl, pr);
      float pHp = 0.f;
#pragma unroll
      for (int j = 0; j < J; ++j) {
        const int k = 32 * j + lane;
        const float lap = npe[j] * p[j] - (k > 0 ? pl[j] : 0.f) - (k < m ? pr[j] : 0.f);
        Hp[j] = ok[j] ? vol * (em[j] * pl[j] + d[j] * p[j] + e[j] * pr[j] + alpha * lap) : 0.f;
        pHp += p[j] * Hp[j];
      }
      pHp = warp_sum_bfly(pHp);
      if (!(pHp > 0.f)) break;
      const float a = rz / pHp;
      float rr = 0.f;
#pragma unroll
      for (int j = 0; j < J; ++j) {
        xv[j] = fmaf(a, p[j], xv[j]);
        r[j] = fmaf(-a, Hp[j], r[j]);
        rr += r[j] * r[j];
      }
      rr = warp_sum_bfly(rr);
      it = i + 1;
      if (sqrtf(rr) / sqrtf(rr0) < rtol) break;
      float zv[J], rzn = 0.f;
#pragma unroll
      for (int j = 0; j < J; ++j) {
        zv[j] = r[j] * di[j];
        rzn += r[j] * zv[j];
      }
      rzn = warp_sum_bfly(rzn);
      const float beta = rzn / rz;
      rz = rzn;
#pragma unroll
      for (int j = 0; j < J; ++j) p[j] = fmaf(beta, p[j], zv[j]);
    }
  }
#pragma unroll
  for (int j = 0; j < J; ++j)
    if (ok[j]) x[pb + (32 * j + lane) * g.psP] = xv[j];
  if (lane == 0 && it > 0) atomicAdd(&st->blk_iters, it);
}

// ------------------------------------------------------------------------------------------
// z-update: dense plane layout [E][nB][nA] for the transforms
// ------------------------------------------------------------------------------------------

// The node-wise ADMM kernels run over (block of kBlock PE columns) x (segment of kAdmmSeg nodes):
// a thread finds its column's bases once and walks the segment.
constexpr int kAdmmSeg = 8;

// T0[k][cB][cA] = b + u at node k of column c = cB nA + cA (b in the caller's layout, u pitched)
__global__ void __launch_bounds__(kBlock)
k_zrhs(Geo g, const float* __restrict__ b, const float* __restrict__ u, float* __restrict__ T0,
       const DevState* st) {
  if (st->stop) return;
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= g.ncols) return;
  const int fb = col_base(c, g.inner, g.fld_ostride), pb = col_pbase(g, c);
  const int k0 = blockIdx.y * kAdmmSeg, k1 = min(k0 + kAdmmSeg, g.E);
  for (int k = k0; k < k1; ++k)
    T0[(long long)k * g.ncols + c] = __ldg(b + fb + k * g.inner) + __ldg(u + pb + k * g.psP);
}

// Batched C_z = A_z B_z (M x N, inner dimension K) over z = blockIdx.z: A(i, l) at
// A.p + z A.sz + i A.si + l A.sj, likewise B(l, j); C(i, j) at
// C + z cz + (i / rp) cp + (i % rp) ci + j cj (rp rows per plane, so that the planes' rows can be
// one tall operand).  A block computes a kGmM x kGmN tile of C over kGmK-deep panels of A and B
// in shared memory, double-buffered: the next panel's copies (cp.async, straight to shared memory)
// are in flight while the current one is multiplied.  Each thread holds a 4 x 8 block of outputs:
// rows 4 ty + a (a < 4), columns 4 tx + b and kGmN / 2 + 4 tx + b (b < 4), so that its operands of
// a depth step are three 16-byte shared loads that consecutive threads take from consecutive
// words (no bank conflicts); 252 threads per 72 x 112 tile keep 18 warps per SM busy on the 3T
// planes' few hundred tiles.  SCALE multiplies entry (i, j) by rho / lambda, lambda =
// rho + alpha (wB muB[i % rp] + wA muA[j]) (rho from the device state).
struct PlaneOperand {
  const float* p;
  long long sz, si, sj;
};
constexpr int kGmM = 72, kGmN = 112, kGmK = 16;
constexpr int kGmTy = kGmM / 4, kGmTx = kGmN / 8, kGmThreads = kGmTy * kGmTx;   // 18 x 14
constexpr int kGmLdA = (kGmM * kGmK + kGmThreads - 1) / kGmThreads;   // copies per thread
constexpr int kGmLdB = (kGmK * kGmN + kGmThreads - 1) / kGmThreads;

template <bool SCALE>
__global__ void __launch_bounds__(kGmThreads, 3)
k_plane_mm(int M, int N, int K, PlaneOperand A, PlaneOperand B, float* __restrict__ C,
           long long cz, int rp, long long cp, long long ci, long long cj,
           const float* __restrict__ muB, const float* __restrict__ muA, float alpha, float wB,
           float wA, const DevState* st) {
  if (st->stop) return;
  __shared__ __align__(16) float As[2][kGmK][kGmM];
  __shared__ __align__(16) float Bs[2][kGmK][kGmN];
  const int z = blockIdx.z, tid = threadIdx.x;
  const int i0 = blockIdx.y * kGmM, j0 = blockIdx.x * kGmN;
  const int tx = tid % kGmTx, ty = tid / kGmTx;
  const float* Ap = A.p + z * A.sz;
  const float* Bp = B.p + z * B.sz;
  // panel element e of A (kGmM x kGmK) and of B (kGmK x kGmN): the unit-stride index fastest
  auto a_pos = [&](int e, int& ri, int& li) {
    if (A.sj == 1) { li = e % kGmK; ri = e / kGmK; } else { ri = e % kGmM; li = e / kGmM; }
  };
  auto b_pos = [&](int e, int& lb, int& jb) {
    if (B.sj == 1) { jb = e % kGmN; lb = e / kGmN; } else { lb = e % kGmK; jb = e / kGmK; }
  };
  // panel at depth l0 into buffer buf, straight to shared memory (cp.async; zeros past the edges)
  auto fetch = [&](int l0, int buf) {
#pragma unroll
    for (int q = 0; q < kGmLdA; ++q) {
      const int e = tid + q * kGmThreads;
      if (e < kGmM * kGmK) {
        int ri, li;
        a_pos(e, ri, li);
        const int ia = i0 + ri, la = l0 + li;
        const bool in = ia < M && la < K;
        cp_async4(&As[buf][li][ri], in ? Ap + (int)(ia * A.si + la * A.sj) : Ap, in);
      }
    }
#pragma unroll
    for (int q = 0; q < kGmLdB; ++q) {
      const int e = tid + q * kGmThreads;
      if (e < kGmK * kGmN) {
        int lb, jb;
        b_pos(e, lb, jb);
        const int lg = l0 + lb, jg = j0 + jb;
        const bool in = lg < K && jg < N;
        cp_async4(&Bs[buf][lb][jb], in ? Bp + (int)(lg * B.si + jg * B.sj) : Bp, in);
      }
    }
    cp_async_commit();
  };
  float acc[4][8];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 8; ++b) acc[a][b] = 0.f;
  const int np = (K + kGmK - 1) / kGmK;
  fetch(0, 0);
  for (int pnl = 0; pnl < np; ++pnl) {
    const int cur = pnl & 1;
    if (pnl + 1 < np) fetch((pnl + 1) * kGmK, cur ^ 1);
    else cp_async_commit();
    cp_async_wait<1>();   // this panel's copies (all but the one just issued) have landed
    __syncthreads();
#pragma unroll
    for (int l = 0; l < kGmK; ++l) {
      const float4 a0 = *reinterpret_cast<const float4*>(&As[cur][l][4 * ty]);
      const float4 b0 = *reinterpret_cast<const float4*>(&Bs[cur][l][4 * tx]);
      const float4 b1 = *reinterpret_cast<const float4*>(&Bs[cur][l][kGmN / 2 + 4 * tx]);
      const float av[4] = {a0.x, a0.y, a0.z, a0.w};
      const float bv[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 8; ++b) acc[a][b] = fmaf(av[a], bv[b], acc[a][b]);
    }
    __syncthreads();   // every thread is done with this buffer before it is refilled
  }
  const float rho = SCALE ? st->admm_rho : 0.f;
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    const int i = i0 + 4 * ty + a;
    if (i >= M) continue;
    const int ip = i / rp, ir = i - ip * rp;
    float* Crow = C + z * cz + ip * cp + ir * ci;
    const float lb = SCALE ? wB * __ldg(muB + ir) : 0.f;
#pragma unroll
    for (int b = 0; b < 8; ++b) {
      const int j = j0 + (b < 4 ? 4 * tx + b : kGmN / 2 + 4 * tx + b - 4);
      if (j >= N) continue;
      float v = acc[a][b];
      if (SCALE) v *= rho / (rho + alpha * (lb + wA * __ldg(muA + j)));
      Crow[j * cj] = v;
    }
  }
}

// ------------------------------------------------------------------------------------------
// multiplier, residuals, rho rule and stop
// ------------------------------------------------------------------------------------------

// Start of an ADMM iteration: u <- s u (s the factor pending from the last rho change), c = z - u,
// b_prev = b (pitched copy); ||b||^2, ||z||^2, ||u||^2 for the relative changes; the GN
// coefficients in the solver arrays are stale (new c and rho): coef_fresh = 0.
__global__ void __launch_bounds__(kBlock)
k_admm_prep(Geo g, const float* __restrict__ b, const float* __restrict__ zc,
            float* __restrict__ u, float* __restrict__ c, float* __restrict__ bprev,
            float* partials, unsigned* counter, DevState* st) {
  if (st->stop) return;
  const float s = st->admm_scale;
  float nb = 0.f, nz = 0.f, nu = 0.f;
  const int cc = blockIdx.x * blockDim.x + threadIdx.x;
  if (cc < g.ncols) {
    const int fb = col_base(cc, g.inner, g.fld_ostride), pb = col_pbase(g, cc);
    const int k0 = blockIdx.y * kAdmmSeg, k1 = min(k0 + kAdmmSeg, g.E);
    for (int k = k0; k < k1; ++k) {
      const int pi = pb + k * g.psP;
      const float bv = __ldg(b + fb + k * g.inner);
      const float zv = zc[pi];
      const float uv = s * u[pi];
      u[pi] = uv;
      c[pi] = zv - uv;
      bprev[pi] = bv;
      nb += bv * bv;
      nz += zv * zv;
      nu += uv * uv;
    }
  }
  float v[3] = {nb, nz, nu};
  double tot[3];
  if (grid_sum<3>(v, partials, counter, tot)) {
    st->nb_prev = tot[0];
    st->nz_prev = tot[1];
    st->nu_prev = tot[2];
    st->admm_scale = 1.f;
    st->coef_fresh = 0;
    st->blk_iters = 0;
  }
}

// ||d|| / ||ref|| from squared norms, with 0/0 = 0 and x/0 = +inf
__device__ __forceinline__ double rel_change(double d2, double ref2) {
  if (ref2 > 0.0) return sqrt(d2) / sqrt(ref2);
  return d2 == 0.0 ? 0.0 : __longlong_as_double(0x7ff0000000000000LL);
}

// End of ADMM iteration `it`: u <- u + b - z; r = ||b - z||, s = rho ||z - z_prev||, the relative
// changes of b, z and u; the statistics row; the rho rule of Boyd et al. (2011, Sec. 3.4.1):
// r > mu s: rho <- tau rho and u <- u / tau, s > mu r: rho <- rho / tau and u <- tau u (the u
// factor is applied by the next k_admm_prep); stop when all three relative changes are < tol.
__global__ void __launch_bounds__(kBlock)
k_admm_post(Geo g, const float* __restrict__ b, const float* __restrict__ z,
            const float* __restrict__ zprev, float* __restrict__ u,
            const float* __restrict__ bprev, int it, float tol, float mu, float tau,
            double* stats, float* partials, unsigned* counter, DevState* st) {
  if (st->stop) return;
  float r2 = 0.f, s2 = 0.f, db2 = 0.f;
  const int cc = blockIdx.x * blockDim.x + threadIdx.x;
  if (cc < g.ncols) {
    const int fb = col_base(cc, g.inner, g.fld_ostride), pb = col_pbase(g, cc);
    const int k0 = blockIdx.y * kAdmmSeg, k1 = min(k0 + kAdmmSeg, g.E);
    for (int k = k0; k < k1; ++k) {
      const int pi = pb + k * g.psP;
      const float bv = __ldg(b + fb + k * g.inner);
      const float zv = z[pi];
      const float dv = bv - zv;
      u[pi] += dv;
      const float dz = zv - zprev[pi], db = bv - bprev[pi];
      r2 += dv * dv;
      s2 += dz * dz;
      db2 += db * db;
    }
  }
  float v[3] = {r2, s2, db2};
  double tot[3];
  if (grid_sum<3>(v, partials, counter, tot)) {
    const double rho = st->admm_rho;
    const double r = sqrt(tot[0]), s = rho * sqrt(tot[1]);
    const double rel_db = rel_change(tot[2], st->nb_prev);
    const double rel_dz = rel_change(tot[1], st->nz_prev);
    const double rel_du = rel_change(tot[0], st->nu_prev);   // u - u_prev = b - z
    if (stats) {
      double* row = stats + (long long)it * kAdmmNStats;
      row[0] = st->J;                                          // J at b (evaluated before)
      row[1] = st->Jacc;                                       // F_c at the b-update's result
      row[2] = rho;
      row[3] = r;
      row[4] = s;
      row[5] = rel_db;
      row[6] = rel_dz;
      row[7] = rel_du;
      row[8] = (double)st->blk_iters;
      row[9] = st->gamma;
    }
    if (r > (double)mu * s) {
      st->admm_rho = (float)(rho * tau);
      st->admm_scale = 1.f / tau;
    } else if (s > (double)mu * r) {
      st->admm_rho = (float)(rho / tau);
      st->admm_scale = tau;
    }
    st->admm_iter = it + 1;
    if (rel_db < tol && rel_dz < tol && rel_du < tol) {
      st->stop = 1;
      st->stop_iter = it;
    }
  }
}

// ADMM start: rho, no pending u factor, no iterations, statistics rows NaN
__global__ void k_admm_init(DevState* st, float rho0, double* stats, int nrows) {
  const double nan = __longlong_as_double(0x7ff8000000000000LL);
  for (int i = threadIdx.x; stats && i < nrows * kAdmmNStats; i += blockDim.x) stats[i] = nan;
  if (threadIdx.x == 0) {
    st->admm_rho = rho0;
    st->admm_scale = 1.f;
    st->admm_iter = 0;
    st->blk_iters = 0;
  }
}

// ------------------------------------------------------------------------------------------

static dim3 node_grid(const Geo& g) {
  return dim3(ceil_div(g.ncols, kBlock), ceil_div(g.E, kAdmmSeg));
}

cudaError_t launch_block_pcg(const Geo& g, const float* rhs, float rhs_sign, const float* dco,
                             const float* eco, const float* invd, float* x, int max_it,
                             double rtol, DevState* st, cudaStream_t s) {
  const int grid = ceil_div(g.ncols, kBlock / 32);
  const float rt = (float)rtol;
#define HYSCO_BPCG(J)                                                                        \
  case J:                                                                                    \
    k_block_pcg<J><<<grid, kBlock, 0, s>>>(g, rhs, rhs_sign, dco, eco, invd, x, max_it, rt, st); \
    break;
  switch (ceil_div(g.E, 32)) {
    HYSCO_BPCG(1) HYSCO_BPCG(2) HYSCO_BPCG(3) HYSCO_BPCG(4)
    HYSCO_BPCG(5) HYSCO_BPCG(6) HYSCO_BPCG(7) HYSCO_BPCG(8)
    default: return cudaErrorInvalidValue;   // the caller limits the column length
  }
#undef HYSCO_BPCG
  return cudaGetLastError();
}

cudaError_t launch_admm_init(DevState* st, float rho0, double* stats, int nrows, cudaStream_t s) {
  k_admm_init<<<1, kBlock, 0, s>>>(st, rho0, stats, nrows);
  return cudaGetLastError();
}

cudaError_t launch_admm_prep(const Geo& g, const float* b, const float* z, float* u, float* c,
                             float* bprev, const Work& w, cudaStream_t s) {
  k_admm_prep<<<node_grid(g), kBlock, 0, s>>>(g, b, z, u, c, bprev,
                                                                    w.partials, w.counter, w.st);
  return cudaGetLastError();
}

cudaError_t launch_admm_zsolve(const Geo& g, const float* b, const float* u, const AdmmBasis& q,
                               float* T0, float* T1, float* z, const DevState* st,
                               cudaStream_t s) {
  const int nA = g.nA, nB = g.nB, E = g.E;
  const long long P = (long long)nA * nB;
  k_zrhs<<<node_grid(g), kBlock, 0, s>>>(g, b, u, T0, st);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  // per-plane products (planes z = PE node k) and the products whose planes' rows form one tall
  // operand (row r = k nB + cB of T, contiguous planes)
  const dim3 plane_grid(ceil_div(nA, kGmN), ceil_div(nB, kGmM), E);
  const int rows = E * nB;
  const dim3 tall_grid(ceil_div(nA, kGmN), ceil_div(rows, kGmM), 1);
  // 1: T1 = Q_B^T T0          (row jB, column cA)
  k_plane_mm<false><<<plane_grid, kGmThreads, 0, s>>>(
      nB, nA, nB, PlaneOperand{q.QB, 0, 1, nB}, PlaneOperand{T0, P, nA, 1}, T1, P, nB, 0, nA, 1,
      nullptr, nullptr, 0.f, 0.f, 0.f, st);
  // 2: T0 = (T1 Q_A) .* rho / lambda
  k_plane_mm<true><<<tall_grid, kGmThreads, 0, s>>>(
      rows, nA, nA, PlaneOperand{T1, 0, nA, 1}, PlaneOperand{q.QA, 0, nA, 1}, T0, 0, nB, P, nA, 1,
      q.muB, q.muA, g.alpha, g.wB, g.wA, st);
  // 3: T1 = Q_B T0
  k_plane_mm<false><<<plane_grid, kGmThreads, 0, s>>>(
      nB, nA, nB, PlaneOperand{q.QB, 0, nB, 1}, PlaneOperand{T0, P, nA, 1}, T1, P, nB, 0, nA, 1,
      nullptr, nullptr, 0.f, 0.f, 0.f, st);
  // 4: z = T1 Q_A^T, written into the pitched field (plane k, row cB, column cA)
  k_plane_mm<false><<<tall_grid, kGmThreads, 0, s>>>(
      rows, nA, nA, PlaneOperand{T1, 0, nA, 1}, PlaneOperand{q.QA, 0, 1, nA}, z, 0, nB, g.psP,
      g.psB, g.psA, nullptr, nullptr, 0.f, 0.f, 0.f, st);
  return cudaGetLastError();
}

cudaError_t launch_admm_post(const Geo& g, const float* b, const float* z, const float* zprev,
                             float* u, const float* bprev, int it, double tol, double mu,
                             double tau, double* stats, const Work& w, cudaStream_t s) {
  k_admm_post<<<node_grid(g), kBlock, 0, s>>>(
      g, b, z, zprev, u, bprev, it, (float)tol, (float)mu, (float)tau, stats, w.partials,
      w.counter, w.st);
  return cudaGetLastError();
}

}  // namespace hysco
