// Internal declarations shared by the libhysco CUDA translation units.
//
// Geometry: a problem with image dims (d0, d1, d2), PE axis p, m = d_p is seen as `ncols` PE
// columns of m cells (image) and E = m + 1 nodes (field).  Column c has in-plane coordinates
// cA = c % nA (the faster of the two non-PE axes) and cB = c / nA.  Element k of column c sits
// at  (c / inner) * (len * inner) + k * inner + (c % inner)  where inner = product of the dims
// after p and len = m (image) or E (field); `inner` is therefore also the PE stride.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

namespace hysco {

// n / d for 0 <= n < 2^31 by multiply-high (Granlund & Montgomery, "Division by invariant
// integers using multiplication", PLDI 1994): s = ceil(log2 d), mul = floor(2^32 (2^s - d) / d) + 1.
struct FastDiv {
  unsigned d, mul, shift;
};
inline FastDiv make_fastdiv(unsigned d) {
  unsigned s = 0;
  while ((1ull << s) < d) ++s;
  unsigned long long mul = ((1ull << 32) * ((1ull << s) - d)) / d + 1;
  return FastDiv{d, (unsigned)mul, s};
}
__device__ __forceinline__ unsigned fdiv(unsigned n, const FastDiv& f) {
  return (__umulhi(n, f.mul) + n) >> f.shift;
}

struct Geo {
  int m;                 // cells along PE
  int E;                 // nodes along PE (m + 1)
  int ncols;             // PE columns
  int inner;             // PE stride (product of dims after the PE axis)
  int nA, nB;            // in-plane extents, c = cB * nA + cA
  long long img_ostride; // m * inner
  long long fld_ostride; // E * inner
  float wA, wB;          // (h_p / h_A)^2, (h_p / h_B)^2: in-plane Laplacian weights, PE-voxel units
  float vol;             // h0 h1 h2, midpoint quadrature weight
  float alpha;           // smoothness weight
  float half_beta;       // beta / 2 (barrier Hessian / gradient factor)
  double alpha_d, beta_d;
  // flat view of the field: extents fe, C-order strides fs, per-axis Laplacian weight w
  // (w[p] = 1, in-plane (h_p / h_a)^2), the PE axis p, and dividers by fs[0], fs[1]
  int fe[3], fs[3];
  float w[3];
  int p;
  int nf;                // field nodes
  FastDiv div0, div1;
  // Pitched internal layout of the solver's field arrays: the caller's C order with the innermost
  // extent padded to P2 = 4 * ceil(fe[2] / 4), so every row starts 16-byte aligned and a group of 4
  // consecutive nodes never straddles rows.  Padding entries are kept at exactly zero.
  int P2;                // pitch of the innermost axis
  int G4;                // float4 groups per row (P2 / 4)
  int nfp;               // fe[0] * fe[1] * P2
  int ps[3];             // pitched strides (ps[2] = 1)
  int psA, psB, psP;     // pitched strides of the in-plane axes A, B and of the PE axis
  FastDiv divG4, divfe1, divfe2;
  // Column march of the objective kernels: a warp owns 32 consecutive columns (a "tile") and one
  // segment of mseg consecutive nodes of each; nseg segments cover the E nodes.  Chosen at
  // handle creation so that ntile * nseg warps fit in one wave of resident blocks.
  FastDiv divIn, divA;   // dividers by inner and by nA
  int ntile, nseg, mseg;
};

// Device-resident scalar state of a solve (and of single hysco_eval calls).
struct DevState {
  double J, D, S, P, gnorm;   // at the current iterate (last eval)
  double gq;                  // grad^T q
  double rho, rr0, rr, relres, alpha_cg, beta_cg;
  double gamma;               // accepted step of the current GN iteration
  double ot_shift;            // positivity shift of the OT initialisation
  int pcg_iter, pcg_done;
  int ls_done, ls_trials;
  int status;                 // hysco_status of the last numerical evaluation
  int stop, stop_iter;        // solve stopped (J not finite) at GN iteration stop_iter
  int gn_iter;
  // set by the gamma = 1 line-search pass when it accepts: the GN coefficients it wrote (at
  // b + q) are those of the next iterate, whose J, D, S, P, ||grad|| are stashed here
  int coef_fresh, status_n;
  double Jn, Dn, Sn, Pn, gnorm_n;
  float start_scale;          // factor applied to the OT start by the feasible-start rule
  // ADMM (Sec. 2.3.2)
  float admm_rho;             // augmentation weight of the current b-update (prox rho vol/2 ||b-c||^2)
  float admm_scale;           // factor on u pending from the last rho change
  int admm_iter;              // ADMM iterations completed
  int blk_iters;              // BlockPCG iterations summed over columns (this ADMM iteration)
  double prox;                // vol/2 ||b - c||^2 at the last evaluation with the prox term
  double Jacc;                // the prox objective at the iterate the last b-update step kept
  double nb_prev, nz_prev, nu_prev;   // ||b||^2, ||z||^2, ||u||^2 at the iteration's start
};

constexpr int kBlock = 256;   // threads per block of every kernel
constexpr int kMaxTrials = 16;
constexpr int kSeg = 4;       // PE nodes per thread in the short column-march kernels
constexpr int kMinMarch = 4;  // fewest PE nodes per segment of the objective's column march
constexpr int kNpt = 2;       // nodes per thread in the flat stencil kernels
constexpr int kLsBatch = 9;   // Armijo trials per line-search launch after the first (gamma = 1)

__host__ __device__ inline int ceil_div(int a, int b) { return (a + b - 1) / b; }

// offsets fit in 32 bits: the field has fewer than 2^31 nodes (checked at handle creation)
__device__ __forceinline__ int col_base(int c, int inner, long long ostride) {
  int o = c / inner;
  return o * (int)ostride + (c - o * inner);
}

__device__ __forceinline__ float ldf(const float* p) { return __ldg(p); }
__device__ __forceinline__ float ldf(const __nv_bfloat16* p) { return __bfloat162float(__ldg(p)); }
__device__ __forceinline__ float ldf(const __half* p) { return __half2float(__ldg(p)); }

// A load of an array that the launch reads only (RO: the read-only path) or that the same launch
// also writes, before a device-wide barrier (!RO: an ordinary, coherent load).
template <bool RO, typename T>
__device__ __forceinline__ T ld_in(const T* p) {
  if constexpr (RO) return __ldg(p);
  else return *p;
}

// After an accepted gamma = 1 trial the GN coefficients in place are those of the new iterate:
// its stashed J, terms, gradient norm and status become the current ones and the per-step fields
// restart (one thread).  Idempotent: a second call copies the same values.
__device__ __forceinline__ void promote_stash(DevState* st, bool prox) {
  st->J = st->Jn; st->D = st->Dn; st->S = st->Sn; st->P = st->Pn;
  if (prox) st->Jacc = st->Jn;
  st->gnorm = st->gnorm_n;
  st->status = st->status_n;
  st->ls_done = 0; st->ls_trials = 0; st->gamma = 0.0; st->gq = 0.0;
  st->pcg_done = 0; st->pcg_iter = 0; st->relres = 0.0;
}

// Asynchronous 4-byte copies global -> shared (cp.async): the copy lands in shared memory without
// passing through registers, so the compiler cannot move it next to its use.  pred = false fills
// the word with zero and reads nothing.  A thread sees its own copies after cp_async_wait<n>
// (all but its n most recent commit groups complete); other threads after a block barrier too.
__device__ __forceinline__ void cp_async4(float* smem, const float* gmem, bool pred) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(s), "l"(gmem),
               "r"(pred ? 4 : 0)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// ------------------------------------------------------------------------------------------
// deterministic reductions: per-thread and per-block partial sums in single precision (a warp
// shuffle tree, then one warp over the block's warp sums); the last block to finish (atomic
// ticket) adds the per-block partials in double-float (see df32) in a fixed order and
// "finishes".  No double precision on the reduction path: this GPU's FP64 rate is a small
// fraction of its FP32 rate, and FP64 trees dominated the reducing kernels when they had them.
// ------------------------------------------------------------------------------------------

template <int K, typename T>
__device__ __forceinline__ void warp_sum(T (&v)[K]) {
#pragma unroll
  for (int i = 0; i < K; ++i)
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v[i] += __shfl_down_sync(0xffffffffu, v[i], off);
}

__device__ __forceinline__ int linear_tid() {
  return threadIdx.x + blockDim.x * (threadIdx.y + blockDim.y * threadIdx.z);
}
__device__ __forceinline__ int block_threads() { return blockDim.x * blockDim.y * blockDim.z; }

// Sum over the block; the result is valid in thread 0.  blockDim total must be a multiple of 32.
template <int K, typename T>
__device__ __forceinline__ void block_sum(T (&v)[K], T* sh /* >= 32*K */) {
  int tid = linear_tid(), nw = block_threads() >> 5;
  warp_sum<K, T>(v);
  __syncthreads();
  if ((tid & 31) == 0)
#pragma unroll
    for (int i = 0; i < K; ++i) sh[(tid >> 5) * K + i] = v[i];
  __syncthreads();
  if (tid < 32) {
#pragma unroll
    for (int i = 0; i < K; ++i) v[i] = tid < nw ? sh[tid * K + i] : T(0);
    warp_sum<K, T>(v);
  }
}

// Double-float accumulation: an unevaluated sum hi + lo of two floats, added with Knuth's
// TwoSum (error-free transformation of the hi parts), giving close to double-precision sums of
// single-precision partials at single-precision speed.
struct df32 {
  float hi, lo;
};
__device__ __forceinline__ df32 df_add(df32 a, df32 b) {
  float s = a.hi + b.hi;
  if (!isfinite(s)) return df32{s, 0.f};   // +-inf and NaN pass through unchanged
  float bb = s - a.hi;
  float e = (a.hi - (s - bb)) + (b.hi - bb);
  e += a.lo + b.lo;
  float hi = s + e;
  return df32{hi, e - (hi - s)};
}
__device__ __forceinline__ df32 df_shfl_down(df32 v, int off) {
  return df32{__shfl_down_sync(0xffffffffu, v.hi, off), __shfl_down_sync(0xffffffffu, v.lo, off)};
}
// block sum of K double-float values; result valid in thread 0
template <int K>
__device__ __forceinline__ void block_sum_df(df32 (&v)[K], df32* sh /* >= 32*K */) {
  int tid = linear_tid(), nw = block_threads() >> 5;
#pragma unroll
  for (int i = 0; i < K; ++i)
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v[i] = df_add(v[i], df_shfl_down(v[i], off));
  __syncthreads();
  if ((tid & 31) == 0)
#pragma unroll
    for (int i = 0; i < K; ++i) sh[(tid >> 5) * K + i] = v[i];
  __syncthreads();
  if (tid < 32) {
#pragma unroll
    for (int i = 0; i < K; ++i) {
      v[i] = tid < nw ? sh[tid * K + i] : df32{0.f, 0.f};
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) v[i] = df_add(v[i], df_shfl_down(v[i], off));
    }
  }
}

// Grid-wide sum of single-precision per-thread values.  Every thread of every block must call
// it.  Returns true in thread 0 of the last block only, with tot[] holding the grid totals
// (double); the ticket counter is reset there.
template <int K>
__device__ bool grid_sum(float (&v)[K], float* partials, unsigned* counter, double (&tot)[K]) {
  __shared__ float shf[32 * K];
  __shared__ df32 shd[32 * K];
  __shared__ int is_last;
  int tid = linear_tid();
  int nblk = gridDim.x * gridDim.y * gridDim.z;
  int bid = blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z);
  block_sum<K, float>(v, shf);
  if (tid == 0) {
#pragma unroll
    for (int i = 0; i < K; ++i) partials[(long long)bid * K + i] = v[i];
    __threadfence();
    unsigned t = atomicAdd(counter, 1u);
    is_last = (t == (unsigned)(nblk - 1));
  }
  __syncthreads();
  if (!is_last) return false;
  __threadfence();
  // value i is summed by warp i % nwarps: lane l takes blocks l, l + 32, ... in order (sixteen
  // loads in flight, then their sums: one round trip for up to 512 blocks), then a fixed shuffle
  // tree; double-float throughout
  constexpr int NF = 16;
  const int warp = tid >> 5, lane = tid & 31, nwarps = block_threads() >> 5;
  for (int i = warp; i < K; i += nwarps) {
    df32 acc{0.f, 0.f};
    for (int b0 = lane; b0 < nblk; b0 += 32 * NF) {
      float x[NF];
#pragma unroll
      for (int u = 0; u < NF; ++u) {
        const int b = b0 + 32 * u;
        x[u] = b < nblk ? __ldcg(partials + (long long)b * K + i) : 0.f;
      }
#pragma unroll
      for (int u = 0; u < NF; ++u)
        if (b0 + 32 * u < nblk) acc = df_add(acc, df32{x[u], 0.f});
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) acc = df_add(acc, df_shfl_down(acc, off));
    if (lane == 0) shd[i] = acc;
  }
  __syncthreads();
  if (tid == 0) {
#pragma unroll
    for (int i = 0; i < K; ++i) tot[i] = (double)shd[i].hi + (double)shd[i].lo;
    *counter = 0u;
    return true;
  }
  return false;
}

// coordinates of field node n (C order)
__device__ __forceinline__ void field_coords(const Geo& g, int n, int (&i)[3]) {
  unsigned q0 = fdiv((unsigned)n, g.div0);
  unsigned r = (unsigned)n - q0 * (unsigned)g.fs[0];
  unsigned q1 = fdiv(r, g.div1);
  i[0] = (int)q0;
  i[1] = (int)q1;
  i[2] = (int)(r - q1 * (unsigned)g.fs[1]);
}

// pitched index of node k of PE column c
__device__ __forceinline__ int col_pbase(const Geo& g, int c) {
  int cB = c / g.nA;
  return cB * g.psB + (c - cB * g.nA) * g.psA;
}

// position of float4 group t of the pitched field: row (i0, i1) and first innermost index x0
struct GroupPos {
  int row, x0, i0, i1;
};
__device__ __forceinline__ GroupPos group_pos(const Geo& g, int t) {
  GroupPos q;
  q.row = (int)fdiv((unsigned)t, g.divG4);
  q.x0 = 4 * (t - q.row * g.G4);
  q.i0 = (int)fdiv((unsigned)q.row, g.divfe1);
  q.i1 = q.row - q.i0 * g.fe[1];
  return q;
}

__device__ __forceinline__ float f4get(const float4& v, int u) {
  return u == 0 ? v.x : (u == 1 ? v.y : (u == 2 ? v.z : v.w));
}

// H z at the four nodes of group t (pitched layout), with the PCG direction update
// p = z + beta p_old, Hp = H z + beta Hp_old (PCG; p_old, Hp_old given, ignored when first) or
// Hv = H z (plain, into hn).  P is the PE axis.  z, which a persistent kernel writes, is read
// with ordinary loads; d, e with the read-only path (RO), or with ordinary loads when the same
// launch has written them (the persistent GN loop).  Padding lanes produce zeros.  Returns the
// sum over the group of p * Hp (PCG).
template <int P, bool PCG, bool RO = true>
__device__ __forceinline__ float hv_core(const Geo& g, int t, const float* z,
                                         const float* dco, const float* eco, float beta,
                                         bool first,
                                         const float4& po, const float4& ho, float4& pn,
                                         float4& hn) {
  const GroupPos q = group_pos(g, t);
  const int n = 4 * t, fe2 = g.fe[2];
  const int s1 = g.G4, s0 = g.fe[1] * g.G4;          // group strides of axes 1 and 0
  const float4* z4p = reinterpret_cast<const float4*>(z);
  const float4 zc = z4p[t];
  const float4 z1m = q.i1 > 0 ? z4p[t - s1] : zc, z1p = q.i1 < g.fe[1] - 1 ? z4p[t + s1] : zc;
  const float4 z0m = q.i0 > 0 ? z4p[t - s0] : zc, z0p = q.i0 < g.fe[0] - 1 ? z4p[t + s0] : zc;
  const float zl = q.x0 > 0 ? z[n - 1] : 0.f;
  const float zr = q.x0 + 4 < g.P2 ? z[n + 4] : 0.f;
  const float4 d4 = ld_in<RO>(reinterpret_cast<const float4*>(dco) + t);
  const float4 e4 = ld_in<RO>(reinterpret_cast<const float4*>(eco) + t);
  float4 em4 = make_float4(0.f, 0.f, 0.f, 0.f);
  float el = 0.f;
  if (P == 0 && q.i0 > 0) em4 = ld_in<RO>(reinterpret_cast<const float4*>(eco) + t - s0);
  if (P == 1 && q.i1 > 0) em4 = ld_in<RO>(reinterpret_cast<const float4*>(eco) + t - s1);
  if (P == 2 && q.x0 > 0) el = ld_in<RO>(eco + n - 1);
  float outp[4], outh[4], acc = 0.f;
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const int x = q.x0 + u;
    const float zk = f4get(zc, u);
    const float a2m = x > 0 ? (u == 0 ? zl : f4get(zc, u - 1)) : zk;
    const float a2p = x < fe2 - 1 ? (u == 3 ? zr : f4get(zc, u + 1)) : zk;
    const float a1m = f4get(z1m, u), a1p = f4get(z1p, u);
    const float a0m = f4get(z0m, u), a0p = f4get(z0p, u);
    const float lap = g.w[0] * ((zk - a0m) + (zk - a0p)) + g.w[1] * ((zk - a1m) + (zk - a1p)) +
                      g.w[2] * ((zk - a2m) + (zk - a2p));
    float elo = P == 2 ? (u == 0 ? el : f4get(e4, u - 1)) : f4get(em4, u);
    if (P == 2 && x == 0) elo = 0.f;
    const float zlo = P == 0 ? a0m : (P == 1 ? a1m : a2m);
    const float zhi = P == 0 ? a0p : (P == 1 ? a1p : a2p);
    const float w = g.vol * (elo * zlo + f4get(d4, u) * zk + f4get(e4, u) * zhi + g.alpha * lap);
    const bool real = x < fe2;
    if (PCG) {
      float pk = first ? zk : fmaf(beta, f4get(po, u), zk);
      float hk = first ? w : fmaf(beta, f4get(ho, u), w);
      outp[u] = real ? pk : 0.f;
      outh[u] = real ? hk : 0.f;
      acc += outp[u] * outh[u];
    } else {
      outp[u] = 0.f;
      outh[u] = real ? w : 0.f;
    }
  }
  pn = make_float4(outp[0], outp[1], outp[2], outp[3]);
  hn = make_float4(outh[0], outh[1], outh[2], outh[3]);
  return acc;
}

// hv_core with p, Hp in global memory (read with ordinary loads, updated in place)
template <int P, bool PCG>
__device__ __forceinline__ float hv_group(const Geo& g, int t, const float* z, float* p, float* Hp,
                                          const float* __restrict__ dco,
                                          const float* __restrict__ eco, float beta, bool first) {
  float4 po = make_float4(0.f, 0.f, 0.f, 0.f), ho = po, pn, hn;
  if (PCG && !first) {
    po = reinterpret_cast<const float4*>(p)[t];
    ho = reinterpret_cast<const float4*>(Hp)[t];
  }
  const float acc = hv_core<P, PCG>(g, t, z, dco, eco, beta, first, po, ho, pn, hn);
  reinterpret_cast<float4*>(Hp)[t] = hn;
  if (PCG) reinterpret_cast<float4*>(p)[t] = pn;
  return acc;
}

// ------------------------------------------------------------------------------------------
// host-side launchers (one translation unit each)
// ------------------------------------------------------------------------------------------

struct Work {        // device buffers the launchers need
  float* partials;
  unsigned* counter;
  DevState* st;
};

// k_eval.cu
// the column-march decomposition of g (divIn, divA, ntile, nseg, mseg) for `device`
void set_march(Geo& g, int device);
int eval_blocks(const Geo& g);   // blocks of an objective launch (one warp per tile and segment)
// grad: caller layout (nullable); grad_p: pitched solver copy (nullable); dco, eco, invd pitched
// cpx (nullable): the ADMM prox centre c (pitched), see k_eval's PROX; terms (nullable, device):
// a single evaluation (it = -1) also writes J, D, S, P there
cudaError_t launch_eval(const Geo& g, int dtype, const void* Ip, const void* Im, const float* b,
                        float* grad, float* grad_p, float* dco, float* eco, float* invd, int it,
                        const Work& w, cudaStream_t s, const float* cpx = nullptr,
                        double* terms = nullptr);
// The gamma = 1 Armijo trial as a full evaluation at b + q (q pitched): J, grad, d, e, 1/diag at
// b + q overwrite the solver arrays (grad_p is read first for grad^T q), and the Armijo decision
// for gamma = 1 is taken; on acceptance the next launch_eval only promotes the stashed terms.
cudaError_t launch_eval_trial(const Geo& g, int dtype, const void* Ip, const void* Im,
                              const float* b, const float* q, float* grad_p, float* dco,
                              float* eco, float* invd, int ls_max, double c1, const Work& w,
                              cudaStream_t s, const float* cpx = nullptr);
// trials t0 .. t0 + kLsBatch - 1 (J only); the gamma = 1 trial is launch_eval_trial
cudaError_t launch_linesearch(const Geo& g, int dtype, const void* Ip, const void* Im,
                              const float* b, const float* q, const float* grad, int t0,
                              int ls_max, double c1, const Work& w, cudaStream_t s,
                              const float* cpx = nullptr);
cudaError_t launch_update(const Geo& g, float* b, const float* q, int it, double* stats,
                          const Work& w, cudaStream_t s);
// the Armijo halvings (when the gamma = 1 trial left them undecided) and the update in one
// cooperative launch of `grid` kPcgBlock-thread blocks (ls_update_grid: one per SM, 0 when the
// device cannot run it); sync: pcg_sync_words(grid) zeroed words
int ls_update_grid(int device, int dtype);
// eval_next: also the next GN step's evaluation (grad_p, dco, eco, invd as launch_eval's) unless
// an accepted gamma = 1 trial already wrote its coefficients; the next launch_pcg_persistent must
// then promote (its `promote`) and the next launch_eval is not made
cudaError_t launch_ls_update(const Geo& g, int dtype, int grid, const void* Ip, const void* Im,
                             float* b, const float* q, int it, int ls_max, double c1,
                             double* stats, unsigned* sync, DevState* st, cudaStream_t s,
                             int eval_next = 0, float* grad_p = nullptr, float* dco = nullptr,
                             float* eco = nullptr, float* invd = nullptr,
                             unsigned* clear = nullptr, int nclear = 0);
// Tm == nullptr: Tp receives the corrected image 1/2 (T+ + T-)
cudaError_t launch_correct(const Geo& g, int dtype, const void* Ip, const void* Im,
                           const float* b, float* Tp, float* Tm, cudaStream_t s);
// k_adjoint.cu: adjoints of the corrected images and of J's distance term at fixed b
cudaError_t launch_correct_adjoint(const Geo& g, int dtype, const void* Ip, const void* Im,
                                   const float* b, const float* gTp, const float* gTm,
                                   float* dIp, float* dIm, float* db, size_t img_bytes,
                                   cudaStream_t s, float scale = 1.0f);
cudaError_t launch_image_grad(const Geo& g, int dtype, const void* Ip, const void* Im,
                              const float* b, float svol, float* dIp, float* dIm,
                              cudaStream_t s);
// implicit differentiation: sign * v^T dg/d(alpha, beta) into out[2] (device doubles), and
// svol / vol * d(v^T g)/dI+- into dIp, dIm (b, v in the caller's field layout)
cudaError_t launch_theta_dots(const Geo& g, const float* b, const float* v, double sign,
                              double* out, const Work& w, cudaStream_t s);
cudaError_t launch_mixed_image_adjoint(const Geo& g, int dtype, const void* Ip, const void* Im,
                                       const float* b, const float* v, float svol, float* dIp,
                                       float* dIm, cudaStream_t s);
cudaError_t launch_cells(const Geo& g, const float* b, int* cp, int* cm, cudaStream_t s);

// k_pcg.cu
// Hv = H_J v about the last linearisation, v and Hv in the caller's layout (d, e pitched)
cudaError_t launch_hessvec_caller(const Geo& g, const float* v, float* Hv, const float* dco,
                                  const float* eco, cudaStream_t s);
cudaError_t launch_pcg_init_jacobi(const Geo& g, const float* grad, float sign, float* x, float* r,
                                   float* z, const float* invd, const Work& w, cudaStream_t s);
cudaError_t launch_pcg_hp(const Geo& g, const float* z, float* p, float* Hp, const float* dco,
                          const float* eco, int first, const Work& w, cudaStream_t s);
cudaError_t launch_pcg_update_jacobi(const Geo& g, float* x, float* r, const float* p,
                                     const float* Hp, float* z, const float* invd, int first,
                                     double rtol, const Work& w, cudaStream_t s);
// z = r / diag, r and z in the caller's layout
cudaError_t launch_jacobi_apply(const Geo& g, const float* r, float* z, const float* invd,
                                cudaStream_t s);
// caller layout <-> pitched layout of a field-shaped array
cudaError_t launch_to_pitched(const Geo& g, const float* src, float* dst, cudaStream_t s);
cudaError_t launch_from_pitched(const Geo& g, const float* src, float* dst, cudaStream_t s);
cudaError_t launch_col_factor(const Geo& g, const float* dco, const float* eco, float* invD,
                              float* lco, cudaStream_t s);
// mode 0 = apply z = M^{-1} r (r, z in the caller's layout);  1 = PCG init (r = sign * grad,
// x = 0);  2 = PCG update (pitched vectors)
cudaError_t launch_col_solve(const Geo& g, int mode, const float* grad, float* x, float* r,
                             const float* p, const float* Hp, float* z, const float* invD,
                             const float* lco, int first, double rtol, float sign,
                             const Work& w, cudaStream_t s);

// k_admm.cu: ADMM of Sec. 2.3.2 (BlockPCG b-update directions, z-update, multiplier / rho)
constexpr int kAdmmNStats = 10;     // statistics per ADMM iteration
constexpr int kAdmmMaxNodes = 256;  // PE nodes per column that BlockPCG holds in registers
struct AdmmBasis {                  // real orthonormal Fourier bases of the in-plane axes
  const float* QA;                  // nA x nA, row = position, column = basis function
  const float* QB;                  // nB x nB
  const float* muA;                 // 2 - 2 cos(2 pi j / nA) of each column of QA
  const float* muB;
};
cudaError_t launch_block_pcg(const Geo& g, const float* rhs, float rhs_sign, const float* dco,
                             const float* eco, const float* invd, float* x, int max_it,
                             double rtol, DevState* st, cudaStream_t s);
cudaError_t launch_admm_init(DevState* st, float rho0, double* stats, int nrows, cudaStream_t s);
cudaError_t launch_admm_prep(const Geo& g, const float* b, const float* z, float* u, float* c,
                             float* bprev, const Work& w, cudaStream_t s);
// T0, T1: dense scratch of E * nB * nA floats each; z pitched
cudaError_t launch_admm_zsolve(const Geo& g, const float* b, const float* u, const AdmmBasis& q,
                               float* T0, float* T1, float* z, const DevState* st,
                               cudaStream_t s);
// the z-update's four products on the tensor cores (k_zgemm.cu): the plan (null where an in-plane
// axis exceeds 256 nodes or no tensor-map encoder is available; QA, QB the host bases), its
// release, and the launches (z pitched)
struct ZgPlan;
ZgPlan* zg_create(const Geo& g, const std::vector<float>& QA, const std::vector<float>& QB);
void zg_destroy(ZgPlan* p);
cudaError_t launch_zgemm_zsolve(const ZgPlan* p, const Geo& g, const float* b, const float* u,
                                const AdmmBasis& q, float* z, DevState* st, cudaStream_t s);
// the failure self-test: a product launch whose stages never fill runs out of a `spin`-cycle wait
// budget and records HYSCO_ETIMEOUT in st
cudaError_t zg_selftest(const ZgPlan* p, DevState* st, long long spin, cudaStream_t s);
cudaError_t launch_admm_post(const Geo& g, const float* b, const float* z, const float* zprev,
                             float* u, const float* bprev, int it, double tol, double mu,
                             double tau, double* stats, const Work& w, cudaStream_t s);

// k_pcg_persistent.cu: cooperative grid size on `device` (0 if not possible) for a field of n4
// float4 groups, and the slots per thread whose r, p, Hp stay in shared memory; the number of
// 32-bit barrier/reduction words a launch of that grid needs
struct PcgPlan {
  int grid, onchip;
};
PcgPlan pcg_persistent_plan(int device, int pe_axis, int n4);
constexpr int kPcgBlock = 768;        // threads per block of the persistent PCG
constexpr int kWaveMax = 8;           // problems per launch of the batched (wave) PCG
constexpr int kPcgBlocksPerSm = 1;    // its blocks per SM at most
inline size_t pcg_onchip_bytes(int slots) { return (size_t)slots * 3 * kPcgBlock * 16; }   // r, p, Hp
constexpr int kSyncHeader = 32;   // words before the partial-sum slots (the arrival counter's line)
constexpr int kSyncMaxK = 8;      // floats per block and slot (widest fused reduction)
constexpr int kTagWordsPerLaneHost = 16;   // grid_allreduce_unordered's block-range limit / 32
// counter line, two float slots of kSyncMaxK per block, two slots of one tagged 64-bit word per block
__host__ __device__ inline size_t pcg_sync_words(int grid) { return kSyncHeader + 2ull * kSyncMaxK * (size_t)grid + 4ull * (size_t)grid; }
// arguments of one problem's persistent PCG
struct PcgArgs {
  const float* grad;     // right-hand side is rhs_sign * grad
  float rhs_sign;
  float* x;
  float* r;
  float* z;
  float* p0;
  float* p1;
  float* Hp;
  const float* dco;
  const float* eco;
  const float* invd;
  unsigned* sync;        // arrival counter + 2 slots of partial sums; zeroed before every launch
  DevState* st;
  int max_it;
  double rtol;
  int onchip;            // slots per thread whose r, p, Hp are in shared memory
  int promote = 0;       // k_pcg_persistent in a solve's step sequence: first promote a pending
                         // stash (promote_stash), and clear the tail launch's barrier words
                         // (the pcg_sync_words(grid) after this launch's own)
};
constexpr int kWaveSlots = 6;   // on-chip slots per thread a wave plans for (221 KB per block)
// a wave: up to kWaveMax problems, each with its block range and arguments
struct PcgWave {
  int n;
  int blk0[kWaveMax], nblk[kWaveMax];
  Geo g[kWaveMax];
  PcgArgs a[kWaveMax];
};
// co-resident blocks of the wave kernel on `device` (0 if it cannot run); sets its attributes
int pcg_wave_setup(int device);
// one cooperative launch for the problems of w (grid = their block total); sync: the problems'
// sync words, sync_words of them, zeroed first
cudaError_t launch_pcg_wave(const PcgWave& w, int grid, int onchip_max, unsigned* sync,
                            size_t sync_words, cudaStream_t s);
// k_gn.cu: the whole Gauss-Newton loop of a problem (Sec. 2.3.1) in one persistent launch on a
// group of blocks: evaluation, Jacobi PCG, the gamma = 1 trial, Armijo halvings and the update,
// every scalar decision taken identically by every block from the same reduced sums.
struct GnArgs {
  const void* Ip;        // images (the wave's dtype), caller layout
  const void* Im;
  float* b;              // field, caller layout: the start on entry, the result on exit
  float* bscr;           // a second field buffer (>= the field's nodes): the gamma = 1 trial
                         // writes b + q there, and an accepted trial swaps the two buffers
  float* grad_p;         // pitched gradient (the PCG's right-hand side is -grad_p)
  double* stats;         // gn_iters rows of 10 (hysco_solve's statistics) or null
  PcgArgs pcg;           // x = q, the work vectors, d, e, 1/diag, the sync words, the state
  int gn_iters, ls_max;
  double c1;
};
struct GnWave {
  int n;
  int blk0[kWaveMax], nblk[kWaveMax];
  Geo g[kWaveMax];       // each with the column march sized for its block range
  GnArgs a[kWaveMax];
};
// co-resident 768-thread blocks per SM of the GN kernel for images of `dtype` with `onchip`
// slots (0: it cannot run); sets its attributes
int gn_setup(int device, int dtype, int onchip);
// the column march of g for `warps` resident warps (k_eval.cu)
void set_march_warps(Geo& g, int warps);
// one cooperative launch for the problems of w (grid = their block total), images of `dtype`;
// sync: the problems' sync words, sync_words of them, zeroed first
cudaError_t launch_gn_wave(const GnWave& w, int dtype, int grid, int onchip_max, unsigned* sync,
                           size_t sync_words, cudaStream_t s);
// sync: 2 * pcg_sync_words(pl.grid) words (the second half for launch_ls_update), all zeroed
// first unless clear == 0 (in a solve's step sequence after the first step, where the previous
// step's tail launch has cleared this launch's words and this launch clears the tail's)
cudaError_t launch_pcg_persistent(const Geo& g, const PcgPlan& pl, const float* grad,
                                  float rhs_sign, float* x, float* r, float* z, float* p0,
                                  float* p1, float* Hp, const float* dco, const float* eco,
                                  const float* invd, unsigned* sync, int max_it, double rtol,
                                  DevState* st, cudaStream_t s, int promote = 0, int clear = 1);
// k_pcg_batched.cu: the Jacobi PCG of many pairs in one cooperative launch.  Pair i is worked
// on by blocks blk0 .. blk0 + nblk - 1 of the grid; its arrays are those of its handle.
struct BatchPair {
  Geo g;
  const float* grad;          // right-hand side is -grad
  float *x, *r, *z, *p, *Hp;
  const float *dco, *eco, *invd;
  DevState* st;
  int blk0, nblk;
};
int pcg_batched_blocks_per_sm(int device);
cudaError_t launch_barrier_selftest(int grid, int missing, long long budget, unsigned* sync,
                                    int* flag, cudaStream_t s);
cudaError_t launch_pcg_batched(int grid, const BatchPair* pairs, const int* block_pair,
                               int max_it, double rtol, unsigned* sync, cudaStream_t s);

// the one-barrier-per-iteration form of the same PCG (r, w, q alternate between two buffers)
int pcg_fused_grid(int device, int pe_axis);
cudaError_t launch_pcg_fused(const Geo& g, int grid, const float* grad, float rhs_sign, float* x,
                             float* p, float* const rb[2], float* const wb[2], float* const qb[2],
                             const float* dco, const float* eco, const float* invd,
                             unsigned* sync, int max_it, double rtol, DevState* st,
                             cudaStream_t s);

// k_ot.cu
cudaError_t launch_ot_shift(const Geo& g, int dtype, const void* Ip, const void* Im,
                            long long n, double eps, const Work& w, cudaStream_t s);
int ot_tile_width(int E);
cudaError_t launch_ot(const Geo& g, int dtype, const void* Ip, const void* Im, float* b0,
                      int* kp, int* km, const Work& w, cudaStream_t s);
cudaError_t launch_blur(const Geo& g, float* in, float* out, cudaStream_t s);   // in unchanged
// k_ls.cu: least-squares correction; the normal matrix's band lives in kLsBandWide + 1
// image-layout scratch arrays (band + d * bstride), its right-hand side in rhs; wide: one int per
// column (the columns the narrow first pass hands to the wide second pass)
constexpr int kLsBand = 4;
constexpr int kLsBandWide = 16;
cudaError_t launch_ls_correct(const Geo& g, int dtype, const void* Ip, const void* Im,
                              const float* b, float lambda, float* band, long long bstride,
                              float* rhs, float* out, int* nbad, int* wide, cudaStream_t s);

// the GN loop's feasible start: b (caller layout) halved until max |delta| < 1
cudaError_t launch_feasible_start(const Geo& g, float* b, const Work& w, cudaStream_t s);

}  // namespace hysco
