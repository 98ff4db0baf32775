// Gauss-Newton Hessian-vector products and the preconditioned CG steps (Sec. 2.3.1).
//
// The GN Hessian about the last evaluated field is
//   H = vol [T + alpha L],  T = per-column tridiagonal (d_k on the diagonal, e_k between k, k+1),
// with d, e written by the eval kernel and L the 7-point negative Laplacian in PE-voxel units
// (PE weight 1, in-plane weights wA, wB).  Vectors are field-shaped float32.
//
// PCG (Hestenes-Stiefel, x0 = 0) is split in two kernels per iteration i so that every global
// inner product is reduced exactly once, in the kernel that produces it:
//   k_pcg_hp:     p = z + beta p (p = z when i = 0), Hp = H p, partial p.Hp
//                 -> last block: alpha = rho / p.Hp (stop if p.Hp <= 0)
//   k_pcg_update: x += alpha p, r -= alpha Hp, partial r.r; z = M^{-1} r, partial r.z
//                 -> last block: stop if ||r|| / ||r0|| < rtol, else beta = r.z / rho, rho = r.z
// The direction is double-buffered (p_old -> p_new alternate between two arrays), and the in-plane
// neighbours of p needed by H p are recomputed from z and p_old, so no launch reads what it writes.
#include "hysco_internal.cuh"

namespace hysco {

__device__ __forceinline__ float jacobi_diag(const Geo& g, float d, int k, float nin) {
  float npe = (float)((k > 0) + (k < g.m));
  return g.vol * (d + g.alpha * (npe + nin));
}

struct NbrCols {
  long long Am, Ap, Bm, Bp;   // field base offsets of the in-plane neighbours, -1 if absent
  float nin;
};

__device__ __forceinline__ NbrCols nbr_cols(const Geo& g, int c) {
  int cA = c % g.nA, cB = c / g.nA;
  NbrCols n;
  n.Am = cA > 0 ? col_base(c - 1, g.inner, g.fld_ostride) : -1;
  n.Ap = cA < g.nA - 1 ? col_base(c + 1, g.inner, g.fld_ostride) : -1;
  n.Bm = cB > 0 ? col_base(c - g.nA, g.inner, g.fld_ostride) : -1;
  n.Bp = cB < g.nB - 1 ? col_base(c + g.nA, g.inner, g.fld_ostride) : -1;
  n.nin = g.wA * (float)((cA > 0) + (cA < g.nA - 1)) + g.wB * (float)((cB > 0) + (cB < g.nB - 1));
  return n;
}

// value of the PCG direction at field offset i: p = z (first) or z + beta p_old
template <bool PCG>
__device__ __forceinline__ float pval(const float* z, const float* pold, long long i, float beta,
                                      int first) {
  if (!PCG || first) return __ldg(z + i);
  return fmaf(beta, __ldg(pold + i), __ldg(z + i));
}

// Hv (PCG = false: v = z, no reduction) or the fused PCG step (PCG = true: p_new = z + beta p_old).
template <bool PCG>
__global__ void __launch_bounds__(kBlock)
k_hv(Geo g, const float* __restrict__ z, const float* __restrict__ pold, float* __restrict__ pnew,
     float* __restrict__ Hp, const float* __restrict__ dco, const float* __restrict__ eco,
     int first, int seg, double* partials, unsigned* counter, DevState* st) {
  float beta = 0.f;
  if (PCG) {
    if (st->stop || st->pcg_done) return;
    beta = first ? 0.f : (float)st->beta_cg;
  }
  int c = blockIdx.x * blockDim.x + threadIdx.x;
  int k0 = blockIdx.y * seg, k1 = min(k0 + seg, g.E);
  float acc = 0.f;
  if (c < g.ncols) {
    const int inner = g.inner;
    long long fb = col_base(c, inner, g.fld_ostride);
    NbrCols nb = nbr_cols(g, c);
    float p_prev = 0.f, e_prev = 0.f;
    if (k0 > 0) {
      p_prev = pval<PCG>(z, pold, fb + (long long)(k0 - 1) * inner, beta, first);
      e_prev = __ldg(eco + fb + (long long)(k0 - 1) * inner);
    }
    float pk = pval<PCG>(z, pold, fb + (long long)k0 * inner, beta, first);
    for (int k = k0; k < k1; ++k) {
      long long o = (long long)k * inner;
      float pn = k < g.m ? pval<PCG>(z, pold, fb + o + inner, beta, first) : 0.f;
      float dk = __ldg(dco + fb + o), ek = __ldg(eco + fb + o);
      float lap = 0.f, la = 0.f, lb = 0.f;
      if (k > 0) lap += pk - p_prev;
      if (k < g.m) lap += pk - pn;
      if (nb.Am >= 0) la += pk - pval<PCG>(z, pold, nb.Am + o, beta, first);
      if (nb.Ap >= 0) la += pk - pval<PCG>(z, pold, nb.Ap + o, beta, first);
      if (nb.Bm >= 0) lb += pk - pval<PCG>(z, pold, nb.Bm + o, beta, first);
      if (nb.Bp >= 0) lb += pk - pval<PCG>(z, pold, nb.Bp + o, beta, first);
      lap += g.wA * la + g.wB * lb;
      float hv = g.vol * (e_prev * p_prev + dk * pk + ek * pn + g.alpha * lap);
      Hp[fb + o] = hv;
      if (PCG) {
        pnew[fb + o] = pk;
        acc += pk * hv;
      }
      p_prev = pk; pk = pn; e_prev = ek;
    }
  }
  if (!PCG) return;
  double v[1] = {acc}, tot[1];
  if (grid_sum<1>(v, partials, counter, tot)) {
    double pHp = tot[0];
    if (!(pHp > 0.0)) {
      st->pcg_done = 1;
    } else {
      st->alpha_cg = st->rho / pHp;
    }
  }
}

// PCG init with Jacobi: r = -grad, x = 0, z = r / diag; rr0 = r.r, rho = r.z
__global__ void __launch_bounds__(kBlock)
k_pcg_init_jacobi(Geo g, const float* __restrict__ grad, float* __restrict__ x,
                  float* __restrict__ r, float* __restrict__ z, const float* __restrict__ dco,
                  int seg, double* partials, unsigned* counter, DevState* st) {
  if (st->stop) return;
  int c = blockIdx.x * blockDim.x + threadIdx.x;
  int k0 = blockIdx.y * seg, k1 = min(k0 + seg, g.E);
  float arr = 0.f, arz = 0.f;
  if (c < g.ncols) {
    long long fb = col_base(c, g.inner, g.fld_ostride);
    NbrCols nb = nbr_cols(g, c);
    for (int k = k0; k < k1; ++k) {
      long long i = fb + (long long)k * g.inner;
      float rk = -__ldg(grad + i);
      float dg = jacobi_diag(g, __ldg(dco + i), k, nb.nin);
      float zk = dg > 0.f ? rk / dg : rk;
      x[i] = 0.f; r[i] = rk; z[i] = zk;
      arr += rk * rk; arz += rk * zk;
    }
  }
  double v[2] = {arr, arz}, tot[2];
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
                    float* __restrict__ z, const float* __restrict__ dco, int first, double rtol,
                    int seg, double* partials, unsigned* counter, DevState* st) {
  if (st->stop || st->pcg_done) return;
  float a = (float)st->alpha_cg;
  int c = blockIdx.x * blockDim.x + threadIdx.x;
  int k0 = blockIdx.y * seg, k1 = min(k0 + seg, g.E);
  float arr = 0.f, arz = 0.f;
  if (c < g.ncols) {
    long long fb = col_base(c, g.inner, g.fld_ostride);
    NbrCols nb = nbr_cols(g, c);
    for (int k = k0; k < k1; ++k) {
      long long i = fb + (long long)k * g.inner;
      float pk = __ldg(p + i);
      x[i] = first ? a * pk : fmaf(a, pk, x[i]);
      float rk = fmaf(-a, __ldg(Hp + i), r[i]);
      r[i] = rk;
      float dg = jacobi_diag(g, __ldg(dco + i), k, nb.nin);
      float zk = dg > 0.f ? rk / dg : rk;
      z[i] = zk;
      arr += rk * rk; arz += rk * zk;
    }
  }
  double v[2] = {arr, arz}, tot[2];
  if (grid_sum<2>(v, partials, counter, tot)) pcg_finish(st, tot[0], tot[1], rtol);
}

__global__ void __launch_bounds__(kBlock)
k_jacobi_apply(Geo g, const float* __restrict__ r, float* __restrict__ z,
               const float* __restrict__ dco, int seg) {
  int c = blockIdx.x * blockDim.x + threadIdx.x;
  int k0 = blockIdx.y * seg, k1 = min(k0 + seg, g.E);
  if (c >= g.ncols) return;
  long long fb = col_base(c, g.inner, g.fld_ostride);
  NbrCols nb = nbr_cols(g, c);
  for (int k = k0; k < k1; ++k) {
    long long i = fb + (long long)k * g.inner;
    float dg = jacobi_diag(g, __ldg(dco + i), k, nb.nin);
    z[i] = dg > 0.f ? __ldg(r + i) / dg : __ldg(r + i);
  }
}

// ------------------------------------------------------------------------------------------
// per-column block preconditioner: the exact tridiagonal diagonal block of H per PE column,
//   dia_k = vol [d_k + alpha (npe_k + nin)],  off_k = vol [e_k - alpha],
// factored once per GN iteration (LDL^T, l_k = off_k / D_k, D_{k+1} = dia_{k+1} - l_k off_k)
// and applied per PCG iteration by a forward and a backward sweep.
// Tile: CW consecutive columns (lanes) x (kBlock / CW) rows; the tile is staged through shared
// memory with coalesced row accesses and one thread per column runs the sequential sweep.
// ------------------------------------------------------------------------------------------

int column_tile_width(int E) {
  // three E x CW float arrays must fit in shared memory
  if (12LL * E * 32 <= 200 * 1024) return 32;
  if (12LL * E * 16 <= 200 * 1024) return 16;
  return 8;
}

__global__ void __launch_bounds__(kBlock)
k_col_factor(Geo g, const float* __restrict__ dco, const float* __restrict__ eco,
             float* __restrict__ invD, float* __restrict__ lco) {
  extern __shared__ float sm[];
  const int CW = blockDim.x, E = g.E;
  float* dia = sm;            // [E][CW]
  float* off = sm + E * CW;   // [E][CW]
  int tx = threadIdx.x, ty = threadIdx.y;
  int c = blockIdx.x * CW + tx;
  bool act = c < g.ncols;
  long long fb = act ? col_base(c, g.inner, g.fld_ostride) : 0;
  float nin = 0.f;
  if (act) {
    int cA = c % g.nA, cB = c / g.nA;
    nin = g.wA * (float)((cA > 0) + (cA < g.nA - 1)) + g.wB * (float)((cB > 0) + (cB < g.nB - 1));
  }
  for (int k = ty; k < E; k += blockDim.y) {
    float dv = 1.f, ov = 0.f;
    if (act) {
      long long i = fb + (long long)k * g.inner;
      float npe = (float)((k > 0) + (k < g.m));
      dv = g.vol * (__ldg(dco + i) + g.alpha * (npe + nin));
      ov = k < g.m ? g.vol * (__ldg(eco + i) - g.alpha) : 0.f;
    }
    dia[k * CW + tx] = dv;
    off[k * CW + tx] = ov;
  }
  __syncthreads();
  if (ty == 0) {
    float D = dia[tx];
    for (int k = 0; k < E - 1; ++k) {
      float iD = 1.0f / D;
      float ok = off[k * CW + tx];
      float l = ok * iD;
      dia[k * CW + tx] = iD;
      off[k * CW + tx] = l;
      D = fmaf(-l, ok, dia[(k + 1) * CW + tx]);   // D_{k+1} = dia_{k+1} - l_k off_k
    }
    dia[(E - 1) * CW + tx] = 1.0f / D;
    off[(E - 1) * CW + tx] = 0.f;
  }
  __syncthreads();
  if (act)
    for (int k = ty; k < E; k += blockDim.y) {
      long long i = fb + (long long)k * g.inner;
      invD[i] = dia[k * CW + tx];
      lco[i] = off[k * CW + tx];
    }
}

// mode 0: z = M^{-1} r.  mode 1: PCG init (r = -grad, x = 0).  mode 2: PCG update.
template <int MODE>
__global__ void __launch_bounds__(kBlock)
k_col_solve(Geo g, const float* __restrict__ grad, float* __restrict__ x, float* r,
            const float* __restrict__ p, const float* __restrict__ Hp, float* __restrict__ z,
            const float* __restrict__ invD, const float* __restrict__ lco, int first,
            double rtol, double* partials, unsigned* counter, DevState* st) {
  extern __shared__ float sm[];
  if (MODE != 0 && st->stop) return;
  if (MODE == 2 && st->pcg_done) return;
  const int CW = blockDim.x, E = g.E;
  float* R = sm;               // r, then y, then z
  float* L = sm + E * CW;
  float* ID = sm + 2 * E * CW;
  int tx = threadIdx.x, ty = threadIdx.y;
  int c = blockIdx.x * CW + tx;
  bool act = c < g.ncols;
  long long fb = act ? col_base(c, g.inner, g.fld_ostride) : 0;
  float a = MODE == 2 ? (float)st->alpha_cg : 0.f;
  float arr = 0.f, arz = 0.f;
  for (int k = ty; k < E; k += blockDim.y) {
    float rk = 0.f, lk = 0.f, idk = 1.f;
    if (act) {
      long long i = fb + (long long)k * g.inner;
      if (MODE == 0) {
        rk = r[i];
      } else if (MODE == 1) {
        rk = -__ldg(grad + i);
        x[i] = 0.f;
        r[i] = rk;
      } else {
        float pk = __ldg(p + i);
        x[i] = first ? a * pk : fmaf(a, pk, x[i]);
        rk = fmaf(-a, __ldg(Hp + i), r[i]);
        r[i] = rk;
      }
      lk = __ldg(lco + i);
      idk = __ldg(invD + i);
      arr += rk * rk;
    }
    R[k * CW + tx] = rk;
    L[k * CW + tx] = lk;
    ID[k * CW + tx] = idk;
  }
  __syncthreads();
  if (ty == 0) {
    float y = R[tx];
    for (int k = 1; k < E; ++k) {            // forward: y_k = r_k - l_{k-1} y_{k-1}
      y = fmaf(-L[(k - 1) * CW + tx], y, R[k * CW + tx]);
      R[k * CW + tx] = y;
    }
    float zz = y * ID[(E - 1) * CW + tx];    // backward: z_k = y_k / D_k - l_k z_{k+1}
    R[(E - 1) * CW + tx] = zz;
    for (int k = E - 2; k >= 0; --k) {
      zz = fmaf(-L[k * CW + tx], zz, R[k * CW + tx] * ID[k * CW + tx]);
      R[k * CW + tx] = zz;
    }
  }
  __syncthreads();
  if (act)
    for (int k = ty; k < E; k += blockDim.y) {
      long long i = fb + (long long)k * g.inner;
      float zk = R[k * CW + tx];
      z[i] = zk;
      if (MODE != 0) arz += r[i] * zk;
    }
  if (MODE == 0) return;
  double v[2] = {arr, arz}, tot[2];
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

// ------------------------------------------------------------------------------------------

static dim3 field_grid(const Geo& g, int seg) {
  return dim3(ceil_div(g.ncols, kBlock), ceil_div(g.E, seg));
}

cudaError_t launch_hessvec(const Geo& g, const float* v, float* Hv, const float* dco,
                           const float* eco, int seg, cudaStream_t s) {
  k_hv<false><<<field_grid(g, seg), kBlock, 0, s>>>(g, v, nullptr, nullptr, Hv, dco, eco, 0, seg,
                                                    nullptr, nullptr, nullptr);
  return cudaGetLastError();
}

cudaError_t launch_pcg_init_jacobi(const Geo& g, const float* grad, float* x, float* r, float* z,
                                   const float* dco, int seg, const Work& w, cudaStream_t s) {
  k_pcg_init_jacobi<<<field_grid(g, seg), kBlock, 0, s>>>(g, grad, x, r, z, dco, seg, w.partials,
                                                          w.counter, w.st);
  return cudaGetLastError();
}

cudaError_t launch_pcg_hp(const Geo& g, const float* z, const float* pold, float* pnew, float* Hp,
                          const float* dco, const float* eco, int first, int seg, const Work& w,
                          cudaStream_t s) {
  k_hv<true><<<field_grid(g, seg), kBlock, 0, s>>>(g, z, pold, pnew, Hp, dco, eco, first, seg,
                                                   w.partials, w.counter, w.st);
  return cudaGetLastError();
}

cudaError_t launch_pcg_update_jacobi(const Geo& g, float* x, float* r, const float* p,
                                     const float* Hp, float* z, const float* dco, int first,
                                     double rtol, int seg, const Work& w, cudaStream_t s) {
  k_pcg_update_jacobi<<<field_grid(g, seg), kBlock, 0, s>>>(g, x, r, p, Hp, z, dco, first, rtol,
                                                            seg, w.partials, w.counter, w.st);
  return cudaGetLastError();
}

cudaError_t launch_jacobi_apply(const Geo& g, const float* r, float* z, const float* dco, int seg,
                                cudaStream_t s) {
  k_jacobi_apply<<<field_grid(g, seg), kBlock, 0, s>>>(g, r, z, dco, seg);
  return cudaGetLastError();
}

cudaError_t launch_col_factor(const Geo& g, const float* dco, const float* eco, float* invD,
                              float* lco, cudaStream_t s) {
  int CW = column_tile_width(g.E);
  size_t smem = 2ull * g.E * CW * sizeof(float);
  cudaError_t e = cudaFuncSetAttribute(k_col_factor, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  k_col_factor<<<ceil_div(g.ncols, CW), dim3(CW, kBlock / CW), smem, s>>>(g, dco, eco, invD, lco);
  return cudaGetLastError();
}

cudaError_t launch_col_solve(const Geo& g, int mode, const float* grad, float* x, float* r,
                             const float* p, const float* Hp, float* z, const float* invD,
                             const float* lco, int first, double rtol, const Work& w,
                             cudaStream_t s) {
  int CW = column_tile_width(g.E);
  size_t smem = 3ull * g.E * CW * sizeof(float);
  dim3 grid(ceil_div(g.ncols, CW)), block(CW, kBlock / CW);
  cudaError_t e;
#define HYSCO_COLSOLVE(M)                                                                    \
  e = cudaFuncSetAttribute(k_col_solve<M>, cudaFuncAttributeMaxDynamicSharedMemorySize,     \
                           (int)smem);                                                       \
  if (e != cudaSuccess) return e;                                                            \
  k_col_solve<M><<<grid, block, smem, s>>>(g, grad, x, r, p, Hp, z, invD, lco, first, rtol,  \
                                           w.partials, w.counter, w.st);
  if (mode == 0) { HYSCO_COLSOLVE(0) }
  else if (mode == 1) { HYSCO_COLSOLVE(1) }
  else { HYSCO_COLSOLVE(2) }
#undef HYSCO_COLSOLVE
  return cudaGetLastError();
}

}  // namespace hysco
