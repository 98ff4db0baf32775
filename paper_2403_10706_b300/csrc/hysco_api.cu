// libhysco C ABI (include/hysco.h): handle, workspace, argument checks and the GN-PCG driver.
//
// The solve is a fixed, data-independent launch sequence: every scalar decision of Sec. 2.3.1
// (PCG step sizes and early stop, the Armijo accept/reject, the stop on a non-finite J) is taken
// on the device by the last block of the kernel that produces the reduction, and later kernels
// read it from the device state and exit immediately when their work is no longer needed.  No
// host synchronisation happens inside a solve.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <vector>

#include "../../include/hysco.h"
#include "hysco_internal.cuh"

using namespace hysco;

struct hysco_ctx {
  Geo g;
  int dtype;
  int64_t dims[3];
  double spacing[3];
  int pe;
  long long nimg, nfld;
  int device;
  // field-shaped workspace
  float *grad, *dco, *eco, *invd, *x, *r, *z, *p0, *p1, *Hp, *invD, *lco, *tmp, *q0, *q1;
  float* partials;
  unsigned* counter;
  DevState* st;
  PcgPlan pplan;      // persistent PCG grid (0: not available on this device), on-chip slots
  int onchip_max;     // the plan's on-chip slots before any hysco_set_pcg_onchip
  int fgrid;          // one-barrier persistent PCG grid (0: not available)
  bool gn_ok;         // the persistent GN loop (pcg_path 4) can run with the plan's grid
  int lsu_grid;       // grid of the halvings-and-update launch (0: separate kernels)
  unsigned* psync;    // their barrier / reduction words
  bool have_lin, have_factor;
  // CUDA graph of the last solve's launch sequence and the arguments it was captured with
  cudaStream_t cap;
  cudaGraphExec_t gexec;
  const void *g_Ip, *g_Im;
  float* g_b;
  double* g_stats;
  hysco_opts g_opts;
  // ADMM workspace (allocated at the first hysco_admm call): z (two buffers, alternating by
  // iteration), u, c = z - u and the b of the iteration's start, pitched; the in-plane bases
  float *az[2], *au, *ac, *abprev;
  float *aQA, *aQB, *amuA, *amuB;
  // the z-update's tensor-core plan (null where it does not apply) and the path in use:
  // 0 tensor cores (tcgen05, TF32 three-term split), 1 FP32 products on the CUDA cores
  ZgPlan* zg;
  int zpath;
  // least-squares correction workspace (allocated at the first hysco_ls_correct call): the
  // normal matrix's band (kLsBandWide image-shaped arrays), its right-hand side, column flags
  float* lsw;
  cudaGraphExec_t agexec;
  const void *ag_Ip, *ag_Im;
  float* ag_b;
  double* ag_stats;
  hysco_admm_opts ag_opts;
  Work work() const { return Work{partials, counter, st}; }
};

namespace {

const char* kVersion = "hysco-b300 0.1 (sm_103a)";

int check_cuda(cudaError_t e) { return e == cudaSuccess ? HYSCO_OK : HYSCO_ECUDA; }

#define HYSCO_TRY(expr)                      \
  do {                                       \
    cudaError_t e_ = (expr);                 \
    if (e_ != cudaSuccess) return HYSCO_ECUDA; \
  } while (0)

bool aligned(const void* p, size_t a) { return ((uintptr_t)p % a) == 0; }

size_t elem_size(int dtype) { return dtype == HYSCO_F32 ? 4 : 2; }

int check_img(const hysco_ctx* h, const void* p) {
  return (p && aligned(p, elem_size(h->dtype))) ? HYSCO_OK : HYSCO_EINVAL;
}
int check_f32(const void* p) { return (p && aligned(p, 4)) ? HYSCO_OK : HYSCO_EINVAL; }

void free_all(hysco_ctx* h) {
  float* bufs[] = {h->grad, h->dco, h->eco, h->invd, h->x, h->r, h->z, h->p0, h->p1, h->Hp,
                   h->invD, h->lco, h->tmp, h->q0, h->q1};
  for (float* b : bufs)
    if (b) cudaFree(b);
  if (h->partials) cudaFree(h->partials);
  if (h->counter) cudaFree(h->counter);
  if (h->psync) cudaFree(h->psync);
  if (h->gexec) cudaGraphExecDestroy(h->gexec);
  if (h->lsw) cudaFree(h->lsw);
  float* abufs[] = {h->az[0], h->az[1], h->au, h->ac, h->abprev, h->aQA, h->aQB, h->amuA, h->amuB};
  for (float* b : abufs)
    if (b) cudaFree(b);
  if (h->agexec) cudaGraphExecDestroy(h->agexec);
  zg_destroy(h->zg);
  if (h->cap) cudaStreamDestroy(h->cap);
  if (h->st) cudaFree(h->st);
}

int reset_state(hysco_ctx* h, cudaStream_t s) {
  return check_cuda(cudaMemsetAsync(h->st, 0, sizeof(DevState), s));
}

// How a Jacobi or column PCG runs: separate kernels per phase, one persistent kernel with two
// barriers per iteration, or one persistent kernel with one barrier per iteration; in a solve,
// kGnLoop runs the whole GN loop (PCG included) in one persistent kernel.
enum PcgMode { kPcgSeparate = 0, kPcgPersistent = 1, kPcgFused = 2, kGnLoop = 3 };

// pcg_path (hysco_opts) -> mode; HYSCO_EINVAL when the requested kernel cannot run here
int pcg_mode(const hysco_ctx* h, int precond, int path, PcgMode* mode) {
  const bool jac = precond == HYSCO_PC_JACOBI;
  switch (path) {
    case 0:   // measured fastest on B300 at 3T and 7T sizes: the two-barrier persistent kernel
      *mode = jac && h->pplan.grid > 0 ? kPcgPersistent : kPcgSeparate;
      return HYSCO_OK;
    case 1: *mode = kPcgSeparate; return HYSCO_OK;
    case 2: *mode = kPcgPersistent; return jac && h->pplan.grid > 0 ? HYSCO_OK : HYSCO_EINVAL;
    case 3: *mode = kPcgFused; return jac && h->fgrid > 0 ? HYSCO_OK : HYSCO_EINVAL;
    case 4: *mode = kGnLoop; return jac && h->gn_ok ? HYSCO_OK : HYSCO_EINVAL;
    default: return HYSCO_EINVAL;
  }
}

// PCG for H q = sign * g about the handle's linearisation (Sec. 2.3.1); q is written to x.
// promote (persistent mode): the launch first promotes a pending gamma = 1 stash and clears the
// step's tail launch's barrier words; clear: zero the sync words first (see launch_pcg_persistent)
int run_pcg(hysco_ctx* h, const float* g, float sign, float* x, int precond, int max_it,
            double rtol, PcgMode mode, cudaStream_t s, int promote = 0, int clear = 1) {
  const Geo& geo = h->g;
  Work w = h->work();
  if (mode == kPcgFused) {
    float* const rb[2] = {h->r, h->z};
    float* const wb[2] = {h->Hp, h->p1};
    float* const qb[2] = {h->q0, h->q1};
    HYSCO_TRY(launch_pcg_fused(geo, h->fgrid, g, sign, x, h->p0, rb, wb, qb, h->dco, h->eco,
                               h->invd, h->psync, max_it, rtol, h->st, s));
    return HYSCO_OK;
  }
  if (mode == kPcgPersistent) {
    HYSCO_TRY(launch_pcg_persistent(geo, h->pplan, g, sign, x, h->r, h->z, h->p0, h->p1, h->Hp,
                                    h->dco, h->eco, h->invd, h->psync, max_it, rtol,
                                    h->st, s, promote, clear));
    return HYSCO_OK;
  }
  if (precond == HYSCO_PC_JACOBI) {
    HYSCO_TRY(launch_pcg_init_jacobi(geo, g, sign, x, h->r, h->z, h->invd, w, s));
  } else {
    if (!h->have_factor) HYSCO_TRY(launch_col_factor(geo, h->dco, h->eco, h->invD, h->lco, s));
    h->have_factor = true;
    HYSCO_TRY(launch_col_solve(geo, 1, g, x, h->r, nullptr, nullptr, h->z, h->invD, h->lco, 0,
                               rtol, sign, w, s));
  }
  for (int i = 0; i < max_it; ++i) {
    HYSCO_TRY(launch_pcg_hp(geo, h->z, h->p0, h->Hp, h->dco, h->eco, i == 0, w, s));
    if (precond == HYSCO_PC_JACOBI)
      HYSCO_TRY(launch_pcg_update_jacobi(geo, x, h->r, h->p0, h->Hp, h->z, h->invd, i == 0, rtol,
                                         w, s));
    else
      HYSCO_TRY(launch_col_solve(geo, 2, nullptr, x, h->r, h->p0, h->Hp, h->z, h->invD, h->lco,
                                 i == 0, rtol, 1.0f, w, s));
  }
  return HYSCO_OK;
}

}  // namespace

extern "C" {

const char* hysco_version(void) { return kVersion; }

void hysco_default_opts(hysco_opts* o) {
  if (!o) return;
  o->gn_iters = 10;
  o->pcg_max_iters = 10;
  o->ls_max_iters = 10;
  o->precond = HYSCO_PC_JACOBI;
  o->init = 1;
  o->ot_blur = 1;
  o->pcg_rtol = 0.1;
  o->armijo_c1 = 1e-4;
  o->ot_eps = 1e-3;
  o->pcg_path = 0;
  o->no_graph = 0;
}

const char* hysco_strerror(int status) {
  switch (status) {
    case HYSCO_OK: return "success";
    case HYSCO_INFEASIBLE: return "barrier infeasible: |d_v b| >= 1 somewhere, J = +inf";
    case HYSCO_EINVAL: return "invalid argument";
    case HYSCO_ECUDA: return "CUDA runtime error";
    case HYSCO_ENOMEM: return "device memory allocation failed";
    case HYSCO_ENONFINITE: return "non-finite (NaN) objective";
    case HYSCO_ENOTREADY: return "no Gauss-Newton linearisation yet: call hysco_eval first";
    case HYSCO_ETIMEOUT: return "a device-wide barrier of the persistent PCG kernel timed out";
    default: return "unknown status";
  }
}

int hysco_create(const int64_t dims[3], const double spacing[3], int pe_dim, double alpha,
                 double beta, int img_dtype, hysco_t* out) {
  if (!out) return HYSCO_EINVAL;
  *out = nullptr;
  if (!dims || !spacing || pe_dim < 0 || pe_dim > 2) return HYSCO_EINVAL;
  if (img_dtype < HYSCO_F32 || img_dtype > HYSCO_F16) return HYSCO_EINVAL;
  if (!(alpha >= 0.0) || !(beta >= 0.0) || !std::isfinite(alpha) || !std::isfinite(beta))
    return HYSCO_EINVAL;
  for (int a = 0; a < 3; ++a) {
    if (dims[a] < 1) return HYSCO_EINVAL;
    if (!(spacing[a] > 0.0) || !std::isfinite(spacing[a])) return HYSCO_EINVAL;
  }
  if (dims[pe_dim] < 2) return HYSCO_EINVAL;
  long long nimg = dims[0] * dims[1] * dims[2];
  long long m = dims[pe_dim];
  long long nfld = nimg / m * (m + 1);
  if (nfld >= (1LL << 31)) return HYSCO_EINVAL;

  hysco_ctx* h = new (std::nothrow) hysco_ctx();
  if (!h) return HYSCO_ENOMEM;
  std::memcpy(h->dims, dims, sizeof(h->dims));
  std::memcpy(h->spacing, spacing, sizeof(h->spacing));
  h->pe = pe_dim;
  h->dtype = img_dtype;
  h->nimg = nimg;
  h->nfld = nfld;
  cudaGetDevice(&h->device);

  Geo& g = h->g;
  g.m = (int)m;
  g.E = (int)m + 1;
  g.ncols = (int)(nimg / m);
  long long inner = 1;
  for (int a = pe_dim + 1; a < 3; ++a) inner *= dims[a];
  g.inner = (int)inner;
  int q[2], k = 0;
  for (int a = 0; a < 3; ++a)
    if (a != pe_dim) q[k++] = a;
  // column index c = cB * nA + cA with A the faster (later) non-PE axis
  g.nA = (int)dims[q[1]];
  g.nB = (int)dims[q[0]];
  g.img_ostride = m * inner;
  g.fld_ostride = (m + 1) * inner;
  double hp = spacing[pe_dim];
  g.wA = (float)((hp / spacing[q[1]]) * (hp / spacing[q[1]]));
  g.wB = (float)((hp / spacing[q[0]]) * (hp / spacing[q[0]]));
  g.vol = (float)(spacing[0] * spacing[1] * spacing[2]);
  g.alpha = (float)alpha;
  g.half_beta = (float)(0.5 * beta);
  g.alpha_d = alpha;
  g.beta_d = beta;
  for (int a = 0; a < 3; ++a) g.fe[a] = (int)(dims[a] + (a == pe_dim ? 1 : 0));
  g.fs[2] = 1;
  g.fs[1] = g.fe[2];
  g.fs[0] = g.fe[1] * g.fe[2];
  for (int a = 0; a < 3; ++a)
    g.w[a] = a == pe_dim ? 1.0f : (float)((hp / spacing[a]) * (hp / spacing[a]));
  g.p = pe_dim;
  g.nf = (int)nfld;
  g.div0 = make_fastdiv((unsigned)g.fs[0]);
  g.div1 = make_fastdiv((unsigned)g.fs[1]);
  g.P2 = (g.fe[2] + 3) / 4 * 4;
  g.G4 = g.P2 / 4;
  g.ps[2] = 1;
  g.ps[1] = g.P2;
  g.ps[0] = g.fe[1] * g.P2;
  g.psA = g.ps[q[1]];
  g.psB = g.ps[q[0]];
  g.psP = g.ps[pe_dim];
  g.divG4 = make_fastdiv((unsigned)g.G4);
  g.divfe1 = make_fastdiv((unsigned)g.fe[1]);
  g.divfe2 = make_fastdiv((unsigned)g.fe[2]);
  set_march(g, h->device);
  long long nfp = (long long)g.fe[0] * g.fe[1] * g.P2;
  if (nfp >= (1LL << 31)) {
    delete h;
    return HYSCO_EINVAL;
  }
  g.nfp = (int)nfp;

  // solver arrays use the pitched layout (>= nfld entries); zeroed once so that every padding
  // entry starts, and stays, at zero
  size_t fbytes = (size_t)(nfp > nfld ? nfp : nfld) * sizeof(float);
  float** bufs[] = {&h->grad, &h->dco, &h->eco, &h->invd, &h->x, &h->r, &h->z, &h->p0, &h->p1,
                    &h->Hp, &h->invD, &h->lco, &h->tmp, &h->q0, &h->q1};
  for (float** b : bufs) {
    if (cudaMalloc((void**)b, fbytes) != cudaSuccess || cudaMemset(*b, 0, fbytes) != cudaSuccess) {
      free_all(h);
      delete h;
      return HYSCO_ENOMEM;
    }
  }
  // partials: the largest grid of any reducing kernel times its reduction width
  long long march_blocks = (long long)ceil_div(g.ncols, kBlock) * ceil_div(g.E, kSeg);
  long long flat_blocks = (long long)ceil_div(g.nf, kBlock) + 1;
  long long nparts = march_blocks * (4 * kLsBatch + 1) + flat_blocks * 2 + 148 * 8 * 2 +
                     (long long)eval_blocks(g) * 8 +
                     (long long)g.ncols * 2 + 64;
  if (cudaMalloc((void**)&h->partials, nparts * sizeof(float)) != cudaSuccess ||
      cudaMalloc((void**)&h->counter, 64 * sizeof(unsigned)) != cudaSuccess ||
      cudaMalloc((void**)&h->st, sizeof(DevState)) != cudaSuccess) {
    free_all(h);
    delete h;
    return HYSCO_ENOMEM;
  }
  h->pplan = pcg_persistent_plan(h->device, pe_dim, (int)(nfp >> 2));
  h->onchip_max = h->pplan.onchip;
  h->fgrid = pcg_fused_grid(h->device, pe_dim);
  h->gn_ok = h->pplan.grid > 0 && gn_setup(h->device, h->dtype, h->onchip_max) >= 1;
  h->lsu_grid = std::min(ls_update_grid(h->device, h->dtype), h->pplan.grid);
  const int sync_grid = h->pplan.grid > h->fgrid ? h->pplan.grid : h->fgrid;
  if (sync_grid > 0 &&
      cudaMalloc((void**)&h->psync, 2 * pcg_sync_words(sync_grid) * sizeof(unsigned)) !=
          cudaSuccess) {
    free_all(h);
    delete h;
    return HYSCO_ENOMEM;
  }
  if (cudaStreamCreateWithFlags(&h->cap, cudaStreamNonBlocking) != cudaSuccess) {
    free_all(h);
    delete h;
    return HYSCO_ECUDA;
  }
  if (cudaMemset(h->counter, 0, 64 * sizeof(unsigned)) != cudaSuccess ||
      cudaMemset(h->st, 0, sizeof(DevState)) != cudaSuccess) {
    free_all(h);
    delete h;
    return HYSCO_ECUDA;
  }
  *out = h;
  return HYSCO_OK;
}

void hysco_destroy(hysco_t h) {
  if (!h) return;
  free_all(h);
  delete h;
}

int hysco_field_dims(hysco_t h, int64_t out[3]) {
  if (!h || !out) return HYSCO_EINVAL;
  for (int a = 0; a < 3; ++a) out[a] = h->dims[a] + (a == h->pe ? 1 : 0);
  return HYSCO_OK;
}

static int init_ot_impl(hysco_t h, const void* Ip, const void* Im, float* b_out, int blur,
                        double eps, int* kp, int* km, cudaStream_t s) {
  Work w = h->work();
  HYSCO_TRY(launch_ot_shift(h->g, h->dtype, Ip, Im, h->nimg, eps, w, s));
  float* dst = blur ? h->tmp : b_out;
  HYSCO_TRY(launch_ot(h->g, h->dtype, Ip, Im, dst, kp, km, w, s));
  if (blur) HYSCO_TRY(launch_blur(h->g, h->tmp, b_out, s));
  return HYSCO_OK;
}

int hysco_init_ot(hysco_t h, const void* Ip, const void* Im, float* b_out, int blur, double eps,
                  hysco_stream_t stream) {
  if (!h || check_img(h, Ip) || check_img(h, Im) || check_f32(b_out)) return HYSCO_EINVAL;
  if (!(eps >= 0.0) || !std::isfinite(eps)) return HYSCO_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  if (int rc = reset_state(h, s)) return rc;
  return init_ot_impl(h, Ip, Im, b_out, blur, eps, nullptr, nullptr, s);
}

int hysco_ot_indices(hysco_t h, const void* Ip, const void* Im, double eps, int32_t* kidx_p,
                     int32_t* kidx_m, hysco_stream_t stream) {
  if (!h || check_img(h, Ip) || check_img(h, Im) || check_f32(kidx_p) || check_f32(kidx_m))
    return HYSCO_EINVAL;
  if (!(eps >= 0.0) || !std::isfinite(eps)) return HYSCO_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  if (int rc = reset_state(h, s)) return rc;
  return init_ot_impl(h, Ip, Im, h->tmp, 0, eps, kidx_p, kidx_m, s);
}

int hysco_eval(hysco_t h, const void* Ip, const void* Im, const float* b, double* terms_dev,
               float* grad, hysco_stream_t stream) {
  if (!h || check_img(h, Ip) || check_img(h, Im) || check_f32(b)) return HYSCO_EINVAL;
  if (!terms_dev || !aligned(terms_dev, 8)) return HYSCO_EINVAL;
  if (grad && !aligned(grad, 4)) return HYSCO_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  // one launch: the evaluation's last block writes J, D, S, P and the state itself
  Work w = h->work();
  HYSCO_TRY(launch_eval(h->g, h->dtype, Ip, Im, b, grad, nullptr, h->dco, h->eco, h->invd, -1, w,
                        s, nullptr, terms_dev));
  h->have_lin = true;
  h->have_factor = false;
  return HYSCO_OK;
}

int hysco_hessvec(hysco_t h, const float* v, float* Hv, hysco_stream_t stream) {
  if (!h || check_f32(v) || check_f32(Hv)) return HYSCO_EINVAL;
  if (!h->have_lin) return HYSCO_ENOTREADY;
  cudaStream_t s = (cudaStream_t)stream;
  HYSCO_TRY(launch_hessvec_caller(h->g, v, Hv, h->dco, h->eco, s));
  return HYSCO_OK;
}

int hysco_precond(hysco_t h, const float* r, float* z, int kind, hysco_stream_t stream) {
  if (!h || check_f32(r) || check_f32(z)) return HYSCO_EINVAL;
  if (kind != HYSCO_PC_JACOBI && kind != HYSCO_PC_COLUMN) return HYSCO_EINVAL;
  if (kind == HYSCO_PC_COLUMN && h->g.m > 1024) return HYSCO_EINVAL;
  if (!h->have_lin) return HYSCO_ENOTREADY;
  cudaStream_t s = (cudaStream_t)stream;
  // both apply in the caller's layout (the factors and 1/diag stay pitched)
  if (kind == HYSCO_PC_JACOBI) {
    HYSCO_TRY(launch_jacobi_apply(h->g, r, z, h->invd, s));
  } else {
    if (!h->have_factor) {
      HYSCO_TRY(launch_col_factor(h->g, h->dco, h->eco, h->invD, h->lco, s));
      h->have_factor = true;
    }
    HYSCO_TRY(launch_col_solve(h->g, 0, nullptr, nullptr, const_cast<float*>(r), nullptr,
                               nullptr, z, h->invD, h->lco, 0, 0.0, 1.0f, h->work(), s));
  }
  return HYSCO_OK;
}

int hysco_pcg(hysco_t h, const float* rhs, float* q, int precond, int max_iters, double rtol,
              int pcg_path, hysco_stream_t stream) {
  if (!h || check_f32(rhs) || check_f32(q)) return HYSCO_EINVAL;
  if (precond != HYSCO_PC_JACOBI && precond != HYSCO_PC_COLUMN) return HYSCO_EINVAL;
  if (precond == HYSCO_PC_COLUMN && h->g.m > 1024) return HYSCO_EINVAL;
  if (max_iters < 1 || max_iters > 64 || !(rtol >= 0.0)) return HYSCO_EINVAL;
  PcgMode mode;
  if (pcg_mode(h, precond, pcg_path, &mode)) return HYSCO_EINVAL;
  if (mode == kGnLoop) mode = kPcgPersistent;   // the GN loop's PCG is the persistent kernel's
  if (!h->have_lin) return HYSCO_ENOTREADY;
  cudaStream_t s = (cudaStream_t)stream;
  if (int rc = reset_state(h, s)) return rc;
  HYSCO_TRY(launch_to_pitched(h->g, rhs, h->tmp, s));
  if (int rc = run_pcg(h, h->tmp, 1.0f, h->x, precond, max_iters, rtol, mode, s)) return rc;
  HYSCO_TRY(launch_from_pitched(h->g, h->x, q, s));
  return HYSCO_OK;
}

int hysco_correct(hysco_t h, const void* Ip, const void* Im, const float* b, float* Tp,
                  float* Tm, hysco_stream_t stream) {
  if (!h || check_img(h, Ip) || check_img(h, Im) || check_f32(b) || check_f32(Tp) ||
      check_f32(Tm))
    return HYSCO_EINVAL;
  HYSCO_TRY(launch_correct(h->g, h->dtype, Ip, Im, b, Tp, Tm, (cudaStream_t)stream));
  return HYSCO_OK;
}

int hysco_correct_mean(hysco_t h, const void* Ip, const void* Im, const float* b, float* T,
                       hysco_stream_t stream) {
  if (!h || check_img(h, Ip) || check_img(h, Im) || check_f32(b) || check_f32(T))
    return HYSCO_EINVAL;
  HYSCO_TRY(launch_correct(h->g, h->dtype, Ip, Im, b, T, nullptr, (cudaStream_t)stream));
  return HYSCO_OK;
}

int hysco_correct_mean_adjoint(hysco_t h, const void* Ip, const void* Im, const float* b,
                               const float* gT, float* dIp, float* dIm, float* db,
                               hysco_stream_t stream) {
  if (!h || check_img(h, Ip) || check_img(h, Im) || check_f32(b) || check_f32(gT))
    return HYSCO_EINVAL;
  if ((dIp && !aligned(dIp, 4)) || (dIm && !aligned(dIm, 4)) || (db && !aligned(db, 4)))
    return HYSCO_EINVAL;
  // T = 1/2 (T+ + T-): the adjoint of hysco_correct with both upstream sensitivities gT / 2
  HYSCO_TRY(launch_correct_adjoint(h->g, h->dtype, Ip, Im, b, gT, gT, dIp, dIm, db,
                                   (size_t)h->nimg * sizeof(float), (cudaStream_t)stream, 0.5f));
  return HYSCO_OK;
}

int hysco_correct_adjoint(hysco_t h, const void* Ip, const void* Im, const float* b,
                          const float* gTp, const float* gTm, float* dIp, float* dIm, float* db,
                          hysco_stream_t stream) {
  if (!h || check_img(h, Ip) || check_img(h, Im) || check_f32(b)) return HYSCO_EINVAL;
  if ((gTp && !aligned(gTp, 4)) || (gTm && !aligned(gTm, 4)) || (dIp && !aligned(dIp, 4)) ||
      (dIm && !aligned(dIm, 4)) || (db && !aligned(db, 4)))
    return HYSCO_EINVAL;
  HYSCO_TRY(launch_correct_adjoint(h->g, h->dtype, Ip, Im, b, gTp, gTm, dIp, dIm, db,
                                   (size_t)h->nimg * sizeof(float), (cudaStream_t)stream));
  return HYSCO_OK;
}

int hysco_implicit_parts(hysco_t h, const void* Ip, const void* Im, const float* b,
                         const float* v, float* dIp, float* dIm, double* dtheta,
                         hysco_stream_t stream) {
  if (!h || check_img(h, Ip) || check_img(h, Im) || check_f32(b) || check_f32(v)) return HYSCO_EINVAL;
  if ((dIp && !aligned(dIp, 4)) || (dIm && !aligned(dIm, 4)) || (dtheta && !aligned(dtheta, 8)))
    return HYSCO_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  HYSCO_TRY(launch_mixed_image_adjoint(h->g, h->dtype, Ip, Im, b, v, -h->g.vol, dIp, dIm, s));
  if (dtheta) {
    HYSCO_TRY(launch_theta_dots(h->g, b, v, -1.0, dtheta, h->work(), s));
  }
  return HYSCO_OK;
}

int hysco_solve_adjoint(hysco_t h, const void* Ip, const void* Im, const float* b,
                        const float* dLdb, int max_iters, double rtol, float* v_out, float* dIp,
                        float* dIm, double* dtheta, hysco_stream_t stream) {
  if (!h || check_img(h, Ip) || check_img(h, Im) || check_f32(b) || check_f32(dLdb))
    return HYSCO_EINVAL;
  if (max_iters < 1 || max_iters > 1000 || !(rtol >= 0.0)) return HYSCO_EINVAL;
  if (v_out && !aligned(v_out, 4)) return HYSCO_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  PcgMode mode;
  if (pcg_mode(h, HYSCO_PC_JACOBI, 0, &mode)) return HYSCO_EINVAL;
  // the GN linearisation at b, then v = H^{-1} dL/db
  if (int rc = reset_state(h, s)) return rc;
  HYSCO_TRY(launch_eval(h->g, h->dtype, Ip, Im, b, nullptr, h->grad, h->dco, h->eco, h->invd, -1,
                        h->work(), s));
  h->have_lin = true;
  h->have_factor = false;
  HYSCO_TRY(launch_to_pitched(h->g, dLdb, h->tmp, s));
  if (int rc = run_pcg(h, h->tmp, 1.0f, h->x, HYSCO_PC_JACOBI, max_iters, rtol, mode, s)) return rc;
  float* v = v_out ? v_out : h->tmp;   // the caller's layout (tmp is free once the PCG has run)
  HYSCO_TRY(launch_from_pitched(h->g, h->x, v, s));
  return hysco_implicit_parts(h, Ip, Im, b, v, dIp, dIm, dtheta, stream);
}

int hysco_image_grad(hysco_t h, const void* Ip, const void* Im, const float* b, double gJ,
                     float* dIp, float* dIm, hysco_stream_t stream) {
  if (!h || check_img(h, Ip) || check_img(h, Im) || check_f32(b) || !std::isfinite(gJ))
    return HYSCO_EINVAL;
  if ((dIp && !aligned(dIp, 4)) || (dIm && !aligned(dIm, 4))) return HYSCO_EINVAL;
  const float svol = (float)(gJ * (double)h->g.vol);
  HYSCO_TRY(launch_image_grad(h->g, h->dtype, Ip, Im, b, svol, dIp, dIm, (cudaStream_t)stream));
  return HYSCO_OK;
}

int hysco_ls_correct(hysco_t h, const void* Ip, const void* Im, const float* b, double lambda,
                     float* out, int32_t* nbad, hysco_stream_t stream) {
  if (!h || check_img(h, Ip) || check_img(h, Im) || check_f32(b) || check_f32(out)) return HYSCO_EINVAL;
  if (!(lambda > 0.0) || !std::isfinite(lambda) || (nbad && !aligned(nbad, 4))) return HYSCO_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  const size_t nimg = (size_t)h->nimg;
  if (!h->lsw &&
      cudaMalloc((void**)&h->lsw, ((kLsBandWide + 1) * nimg + (size_t)h->g.ncols) * sizeof(float)) !=
          cudaSuccess) {
    h->lsw = nullptr;
    return HYSCO_ENOMEM;
  }
  float* band = h->lsw;
  float* rhs = h->lsw + kLsBandWide * nimg;
  int* wide = reinterpret_cast<int*>(h->lsw + (kLsBandWide + 1) * nimg);
  int* bad = reinterpret_cast<int*>(h->counter + 48);
  HYSCO_TRY(cudaMemsetAsync(bad, 0, sizeof(int), s));
  HYSCO_TRY(launch_ls_correct(h->g, h->dtype, Ip, Im, b, (float)lambda, band, (long long)nimg, rhs,
                              out, bad, wide, s));
  if (nbad) HYSCO_TRY(cudaMemcpyAsync(nbad, bad, sizeof(int), cudaMemcpyDeviceToDevice, s));
  return HYSCO_OK;
}

int hysco_cell_indices(hysco_t h, const float* b, int32_t* cell_p, int32_t* cell_m,
                       hysco_stream_t stream) {
  if (!h || check_f32(b) || check_f32(cell_p) || check_f32(cell_m)) return HYSCO_EINVAL;
  HYSCO_TRY(launch_cells(h->g, b, cell_p, cell_m, (cudaStream_t)stream));
  return HYSCO_OK;
}

}  // extern "C"

namespace {

// The solve's launch sequence (fixed for given arguments; every data-dependent decision is taken
// on the device).
int enqueue_solve(hysco_t h, const void* Ip, const void* Im, float* b_inout, const hysco_opts* o,
                  double* stats, PcgMode mode, cudaStream_t s) {
  const Geo& g = h->g;
  Work w = h->work();
  if (int rc = reset_state(h, s)) return rc;
  if (o->init) {
    if (int rc = init_ot_impl(h, Ip, Im, b_inout, o->ot_blur, o->ot_eps, nullptr, nullptr, s))
      return rc;
    HYSCO_TRY(launch_feasible_start(g, b_inout, w, s));
  }
  if (mode == kGnLoop) {   // the whole GN loop in one persistent launch on the PCG plan's grid
    if (o->gn_iters == 0) return HYSCO_OK;
    GnWave wv{};
    wv.n = 1;
    wv.blk0[0] = 0;
    wv.nblk[0] = h->pplan.grid;
    wv.g[0] = g;
    set_march_warps(wv.g[0], h->pplan.grid * (kPcgBlock / 32));
    wv.a[0] = GnArgs{Ip, Im, b_inout, h->p1, h->grad, stats,
                     PcgArgs{h->grad, -1.0f, h->x, h->r, h->z, h->p0, h->p1, h->Hp, h->dco,
                             h->eco, h->invd, h->psync, h->st, o->pcg_max_iters, o->pcg_rtol,
                             h->pplan.onchip},
                     o->gn_iters, o->ls_max_iters, o->armijo_c1};
    HYSCO_TRY(launch_gn_wave(wv, h->dtype, h->pplan.grid, h->pplan.onchip, h->psync,
                             pcg_sync_words(h->pplan.grid), s));
    return HYSCO_OK;
  }
  // with the persistent PCG, each step ends in one launch: the halvings (if needed), the update
  // and the next step's evaluation (unless the accepted gamma = 1 trial made it unnecessary, the
  // next PCG then promoting the trial's stash)
  const bool tail = mode == kPcgPersistent && h->lsu_grid > 0;
  for (int it = 0; it < o->gn_iters; ++it) {
    if (!tail || it == 0)
      HYSCO_TRY(launch_eval(g, h->dtype, Ip, Im, b_inout, nullptr, h->grad, h->dco, h->eco,
                            h->invd, it, w, s));
    h->have_factor = false;
    if (int rc = run_pcg(h, h->grad, -1.0f, h->x, o->precond, o->pcg_max_iters, o->pcg_rtol,
                         mode, s, tail ? 1 : 0, !tail || it == 0))
      return rc;
    // gamma = 1 as a full evaluation at b + q (its coefficients serve the next GN step when
    // accepted), then the remaining halvings in batches of kLsBatch, J only
    HYSCO_TRY(launch_eval_trial(g, h->dtype, Ip, Im, b_inout, h->x, h->grad, h->dco, h->eco,
                                h->invd, o->ls_max_iters, o->armijo_c1, w, s));
    if (tail) {
      HYSCO_TRY(launch_ls_update(g, h->dtype, h->lsu_grid, Ip, Im, b_inout, h->x, it,
                                 o->ls_max_iters, o->armijo_c1, stats,
                                 h->psync + pcg_sync_words(h->pplan.grid), h->st, s,
                                 it + 1 < o->gn_iters, h->grad, h->dco, h->eco, h->invd,
                                 h->psync, (int)pcg_sync_words(h->pplan.grid)));
      continue;
    }
    for (int t0 = 1; t0 < o->ls_max_iters; t0 += kLsBatch)
      HYSCO_TRY(launch_linesearch(g, h->dtype, Ip, Im, b_inout, h->x, h->grad, t0,
                                  o->ls_max_iters, o->armijo_c1, w, s));
    HYSCO_TRY(launch_update(g, b_inout, h->x, it, stats, w, s));
  }
  return HYSCO_OK;
}

bool same_opts(const hysco_opts& a, const hysco_opts& b) { return std::memcmp(&a, &b, sizeof a) == 0; }

// option values every solve accepts (the handle-dependent checks follow in the callers)
int check_opts(const hysco_opts* o) {
  if (!o) return HYSCO_EINVAL;
  if (o->gn_iters < 0 || o->pcg_max_iters < 1 || o->pcg_max_iters > 64 || o->ls_max_iters < 1 ||
      o->ls_max_iters > kMaxTrials)
    return HYSCO_EINVAL;
  if (o->precond != HYSCO_PC_JACOBI && o->precond != HYSCO_PC_COLUMN) return HYSCO_EINVAL;
  if (!(o->pcg_rtol >= 0.0) || !(o->armijo_c1 >= 0.0) || !(o->ot_eps >= 0.0)) return HYSCO_EINVAL;
  if (o->no_graph < 0 || o->no_graph > 1) return HYSCO_EINVAL;
  return HYSCO_OK;
}

}  // namespace

extern "C" {

int hysco_solve(hysco_t h, const void* Ip, const void* Im, float* b_inout, const hysco_opts* o,
                double* stats, hysco_stream_t stream) {
  if (!h || check_opts(o) || check_img(h, Ip) || check_img(h, Im) || check_f32(b_inout))
    return HYSCO_EINVAL;
  if (stats && !aligned(stats, 8)) return HYSCO_EINVAL;
  if (o->precond == HYSCO_PC_COLUMN && h->g.m > 1024) return HYSCO_EINVAL;
  PcgMode mode;
  if (pcg_mode(h, o->precond, o->pcg_path, &mode)) return HYSCO_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  // the stored linearisation belongs to the iterate before the last update: invalidate it
  h->have_lin = false;
  if (o->no_graph) {
    int rc = enqueue_solve(h, Ip, Im, b_inout, o, stats, mode, s);
    h->have_factor = false;
    return rc;
  }
  const bool cached = h->gexec && h->g_Ip == Ip && h->g_Im == Im && h->g_b == b_inout &&
                      h->g_stats == stats && same_opts(h->g_opts, *o);
  if (!cached) {
    if (h->gexec) cudaGraphExecDestroy(h->gexec);
    h->gexec = nullptr;
    cudaGraph_t graph = nullptr;
    bool ok = cudaStreamBeginCapture(h->cap, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
    int rc = ok ? enqueue_solve(h, Ip, Im, b_inout, o, stats, mode, h->cap) : HYSCO_ECUDA;
    cudaError_t ec = cudaStreamEndCapture(h->cap, &graph);
    ok = ok && rc == HYSCO_OK && ec == cudaSuccess && graph != nullptr;
    if (ok) ok = cudaGraphInstantiate(&h->gexec, graph, 0) == cudaSuccess;
    if (graph) cudaGraphDestroy(graph);
    h->have_factor = false;
    if (!ok) {
      // capture unavailable: launch directly (same kernels)
      h->gexec = nullptr;
      cudaGetLastError();
      int rc2 = enqueue_solve(h, Ip, Im, b_inout, o, stats, mode, s);
      h->have_factor = false;
      return rc2;
    }
    h->g_Ip = Ip;
    h->g_Im = Im;
    h->g_b = b_inout;
    h->g_stats = stats;
    h->g_opts = *o;
  }
  HYSCO_TRY(cudaGraphLaunch(h->gexec, s));
  return HYSCO_OK;
}

int hysco_pcg_plan(hysco_t h, int32_t out[4]) {
  if (!h || !out) return HYSCO_EINVAL;
  const long long T = (long long)h->pplan.grid * kPcgBlock;
  out[0] = h->pplan.grid;
  out[1] = h->pplan.onchip;
  out[2] = T > 0 ? (int32_t)(((long long)(h->g.nfp >> 2) + T - 1) / T) : 0;
  out[3] = kPcgBlock;
  return HYSCO_OK;
}

int hysco_set_pcg_onchip(hysco_t h, int onchip) {
  if (!h || onchip < -1 || onchip > h->onchip_max) return HYSCO_EINVAL;
  h->pplan.onchip = onchip < 0 ? h->onchip_max : onchip;
  if (h->gexec) cudaGraphExecDestroy(h->gexec);   // the cached graph used the old plan
  h->gexec = nullptr;
  return HYSCO_OK;
}

int hysco_last_status(hysco_t h, hysco_stream_t stream) {
  if (!h) return HYSCO_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  if (cudaStreamSynchronize(s) != cudaSuccess) return HYSCO_ECUDA;
  DevState st;
  if (cudaMemcpy(&st, h->st, sizeof(DevState), cudaMemcpyDeviceToHost) != cudaSuccess)
    return HYSCO_ECUDA;
  return st.status;
}

}  // extern "C"

// ------------------------------------------------------------------------------------------
// ADMM (Sec. 2.3.2): see include/hysco.h and k_admm.cu
// ------------------------------------------------------------------------------------------

namespace {

// real orthonormal Fourier basis of length n (row = position x, column = basis function) and the
// eigenvalue 2 - 2 cos(2 pi j / n) of the periodic second difference on each column: the
// constant, then cos / sin pairs of frequencies j = 1 .. (n - 1) / 2, then (-1)^x for even n
void real_fourier_basis(int n, std::vector<float>& Q, std::vector<float>& mu) {
  const double pi = 3.14159265358979323846;
  Q.assign((size_t)n * n, 0.f);
  mu.assign(n, 0.f);
  const double c0 = 1.0 / std::sqrt((double)n), c1 = std::sqrt(2.0 / n);
  for (int x = 0; x < n; ++x) Q[(size_t)x * n] = (float)c0;
  int col = 1;
  for (int j = 1; 2 * j < n; ++j, col += 2) {
    for (int x = 0; x < n; ++x) {
      const double t = 2.0 * pi * (double)((long long)j * x % n) / n;
      Q[(size_t)x * n + col] = (float)(c1 * std::cos(t));
      Q[(size_t)x * n + col + 1] = (float)(c1 * std::sin(t));
    }
    mu[col] = mu[col + 1] = (float)(2.0 - 2.0 * std::cos(2.0 * pi * j / n));
  }
  if (n % 2 == 0) {
    for (int x = 0; x < n; ++x) Q[(size_t)x * n + col] = (float)((x % 2 ? -1.0 : 1.0) * c0);
    mu[col] = 4.f;
  }
}

// allocates what is still missing (a failed earlier call leaves no leak: every buffer lives in
// the handle and is freed with it); the bases are uploaded once
int admm_setup(hysco_ctx* h) {
  if (h->amuB) return HYSCO_OK;
  const size_t fbytes = (size_t)std::max<long long>(h->g.nfp, h->nfld) * sizeof(float);
  float** bufs[] = {&h->az[0], &h->az[1], &h->au, &h->ac, &h->abprev};
  for (float** b : bufs) {
    if (*b) continue;
    if (cudaMalloc((void**)b, fbytes) != cudaSuccess) {
      *b = nullptr;
      cudaGetLastError();
      return HYSCO_ENOMEM;
    }
    if (cudaMemset(*b, 0, fbytes) != cudaSuccess) return HYSCO_ECUDA;
  }
  std::vector<float> QA, QB, muA, muB;
  real_fourier_basis(h->g.nA, QA, muA);
  real_fourier_basis(h->g.nB, QB, muB);
  if (!h->zg) {
    h->zg = zg_create(h->g, QA, QB);
    h->zpath = h->zg ? 0 : 1;
  }
  struct { float** d; const std::vector<float>* v; } up[] = {
      {&h->aQA, &QA}, {&h->aQB, &QB}, {&h->amuA, &muA}, {&h->amuB, &muB}};
  for (auto& u : up) {
    if (*u.d) continue;
    float* d = nullptr;
    if (cudaMalloc((void**)&d, u.v->size() * sizeof(float)) != cudaSuccess) {
      cudaGetLastError();
      return HYSCO_ENOMEM;
    }
    if (cudaMemcpy(d, u.v->data(), u.v->size() * sizeof(float), cudaMemcpyHostToDevice) !=
        cudaSuccess) {
      cudaFree(d);
      return HYSCO_ECUDA;
    }
    *u.d = d;   // set only once uploaded: amuB marks a complete setup
  }
  return HYSCO_OK;
}

// the z-update by the handle's path (admm_setup has run)
cudaError_t zsolve(hysco_ctx* h, const float* b, const float* u, float* z, cudaStream_t s) {
  const AdmmBasis basis{h->aQA, h->aQB, h->amuA, h->amuB};
  if (h->zpath == 0 && h->zg) return launch_zgemm_zsolve(h->zg, h->g, b, u, basis, z, h->st, s);
  return launch_admm_zsolve(h->g, b, u, basis, h->tmp, h->q0, z, h->st, s);
}

int check_admm_opts(const hysco_ctx* h, const hysco_admm_opts* o) {
  if (!o) return HYSCO_EINVAL;
  if (o->admm_iters < 0 || o->admm_iters > 100000 || o->gn_iters < 1 || o->gn_iters > 100 ||
      o->pcg_max_iters < 1 || o->pcg_max_iters > 64 || o->ls_max_iters < 1 ||
      o->ls_max_iters > kMaxTrials)
    return HYSCO_EINVAL;
  if (!(o->pcg_rtol >= 0.0) || !(o->armijo_c1 >= 0.0) || !(o->ot_eps >= 0.0) ||
      !(o->tol >= 0.0) || !(o->mu >= 1.0) || !(o->tau > 1.0) || !std::isfinite(o->rho0) ||
      !std::isfinite(o->mu) || !std::isfinite(o->tau))
    return HYSCO_EINVAL;
  if (o->init < 0 || o->init > 1 || o->no_graph < 0 || o->no_graph > 1) return HYSCO_EINVAL;
  if (h->g.E > kAdmmMaxNodes) return HYSCO_EINVAL;
  return HYSCO_OK;
}

int enqueue_admm(hysco_ctx* h, const void* Ip, const void* Im, float* b, const hysco_admm_opts* o,
                 double* stats, cudaStream_t s) {
  const Geo& g = h->g;
  Geo gs = g;   // the b-subproblem's geometry: no in-plane smoothness (S3 alone)
  gs.wA = 0.f;
  gs.wB = 0.f;
  for (int a = 0; a < 3; ++a)
    if (a != g.p) gs.w[a] = 0.f;
  Work w = h->work();
  if (int rc = reset_state(h, s)) return rc;
  if (o->init) {
    if (int rc = init_ot_impl(h, Ip, Im, b, o->ot_blur, o->ot_eps, nullptr, nullptr, s)) return rc;
    HYSCO_TRY(launch_feasible_start(g, b, w, s));
  }
  const float rho0 = o->rho0 > 0.0 ? (float)o->rho0 : g.alpha;
  HYSCO_TRY(launch_admm_init(h->st, rho0, stats, o->admm_iters, s));
  HYSCO_TRY(launch_to_pitched(g, b, h->az[0], s));
  HYSCO_TRY(cudaMemsetAsync(h->au, 0, (size_t)g.nfp * sizeof(float), s));
  for (int k = 0; k < o->admm_iters; ++k) {
    float* zc = h->az[k & 1];
    float* zn = h->az[(k + 1) & 1];
    HYSCO_TRY(launch_admm_prep(g, b, zc, h->au, h->ac, h->abprev, w, s));
    for (int i = 0; i < o->gn_iters; ++i) {
      HYSCO_TRY(launch_eval(gs, h->dtype, Ip, Im, b, nullptr, h->grad, h->dco, h->eco, h->invd,
                            i, w, s, h->ac));
      HYSCO_TRY(launch_block_pcg(gs, h->grad, -1.0f, h->dco, h->eco, h->invd, h->x,
                                 o->pcg_max_iters, o->pcg_rtol, h->st, s));
      HYSCO_TRY(launch_eval_trial(gs, h->dtype, Ip, Im, b, h->x, h->grad, h->dco, h->eco,
                                  h->invd, o->ls_max_iters, o->armijo_c1, w, s, h->ac));
      for (int t0 = 1; t0 < o->ls_max_iters; t0 += kLsBatch)
        HYSCO_TRY(launch_linesearch(gs, h->dtype, Ip, Im, b, h->x, h->grad, t0, o->ls_max_iters,
                                    o->armijo_c1, w, s, h->ac));
      HYSCO_TRY(launch_update(gs, b, h->x, i, nullptr, w, s));
    }
    // J(b) for the statistics (a fresh full evaluation unless the run has stopped)
    HYSCO_TRY(launch_eval(g, h->dtype, Ip, Im, b, nullptr, h->grad, h->dco, h->eco, h->invd, -2,
                          w, s));
    HYSCO_TRY(zsolve(h, b, h->au, zn, s));
    HYSCO_TRY(launch_admm_post(g, b, zn, zc, h->au, h->abprev, k, o->tol, o->mu, o->tau, stats,
                               w, s));
  }
  return HYSCO_OK;
}

bool same_admm_opts(const hysco_admm_opts& a, const hysco_admm_opts& b) {
  return std::memcmp(&a, &b, sizeof a) == 0;
}

}  // namespace

extern "C" {

void hysco_default_admm_opts(hysco_admm_opts* o) {
  if (!o) return;
  std::memset(o, 0, sizeof *o);
  o->admm_iters = 20;
  o->gn_iters = 2;
  o->pcg_max_iters = 10;
  o->ls_max_iters = 10;
  o->init = 1;
  o->ot_blur = 1;
  o->no_graph = 0;
  o->pcg_rtol = 0.1;
  o->armijo_c1 = 1e-4;
  o->ot_eps = 1e-3;
  o->rho0 = 0.0;
  o->tol = 1e-3;
  o->mu = 10.0;
  o->tau = 2.0;
}

int hysco_block_pcg(hysco_t h, const void* Ip, const void* Im, const float* b, double rho,
                    const float* rhs, float* q, int max_iters, double rtol, int32_t* iters,
                    hysco_stream_t stream) {
  if (!h || check_img(h, Ip) || check_img(h, Im) || check_f32(b) || check_f32(rhs) ||
      check_f32(q))
    return HYSCO_EINVAL;
  if (iters && !aligned(iters, 4)) return HYSCO_EINVAL;
  if (!(rho >= 0.0) || !std::isfinite(rho) || max_iters < 1 || max_iters > 1000 ||
      !(rtol >= 0.0) || h->g.E > kAdmmMaxNodes)
    return HYSCO_EINVAL;
  if (int rc = admm_setup(h)) return rc;
  const Geo& g = h->g;
  Geo gs = g;   // the b-subproblem's geometry: no in-plane smoothness
  gs.wA = 0.f;
  gs.wB = 0.f;
  for (int a = 0; a < 3; ++a)
    if (a != g.p) gs.w[a] = 0.f;
  cudaStream_t s = (cudaStream_t)stream;
  Work w = h->work();
  h->have_lin = false;
  h->have_factor = false;
  if (int rc = reset_state(h, s)) return rc;
  HYSCO_TRY(launch_admm_init(h->st, (float)rho, nullptr, 0, s));
  // the linearisation at b with the prox centre c = b (the coefficients do not depend on c)
  HYSCO_TRY(launch_to_pitched(g, b, h->ac, s));
  HYSCO_TRY(launch_eval(gs, h->dtype, Ip, Im, b, nullptr, h->grad, h->dco, h->eco, h->invd, -1, w,
                        s, h->ac));
  HYSCO_TRY(launch_to_pitched(g, rhs, h->tmp, s));
  HYSCO_TRY(launch_block_pcg(gs, h->tmp, 1.0f, h->dco, h->eco, h->invd, h->x, max_iters, rtol,
                             h->st, s));
  HYSCO_TRY(launch_from_pitched(g, h->x, q, s));
  if (iters)
    HYSCO_TRY(cudaMemcpyAsync(iters, &h->st->blk_iters, sizeof(int32_t), cudaMemcpyDeviceToDevice,
                              s));
  return HYSCO_OK;
}

int hysco_admm_zsolve(hysco_t h, const float* v, double rho, float* z, hysco_stream_t stream) {
  if (!h || check_f32(v) || check_f32(z) || !(rho > 0.0) || !std::isfinite(rho))
    return HYSCO_EINVAL;
  if (int rc = admm_setup(h)) return rc;
  const Geo& g = h->g;
  cudaStream_t s = (cudaStream_t)stream;
  if (int rc = reset_state(h, s)) return rc;
  HYSCO_TRY(launch_admm_init(h->st, (float)rho, nullptr, 0, s));
  HYSCO_TRY(cudaMemsetAsync(h->ac, 0, (size_t)g.nfp * sizeof(float), s));   // u = 0
  HYSCO_TRY(zsolve(h, v, h->ac, h->az[0], s));
  HYSCO_TRY(launch_from_pitched(g, h->az[0], z, s));
  return HYSCO_OK;
}

int hysco_set_zsolve_path(hysco_t h, int path) {
  if (!h || path < 0 || path > 1) return HYSCO_EINVAL;
  if (int rc = admm_setup(h)) return rc;
  if (path == 0 && !h->zg) return HYSCO_EINVAL;
  if (path != h->zpath && h->agexec) {   // the cached ADMM graph used the other path
    cudaGraphExecDestroy(h->agexec);
    h->agexec = nullptr;
  }
  h->zpath = path;
  return HYSCO_OK;
}

int hysco_selftest_zsolve(hysco_t h, int64_t spin_cycles, hysco_stream_t stream) {
  if (!h || spin_cycles < 1 || spin_cycles > 4000000000LL) return HYSCO_EINVAL;
  if (int rc = admm_setup(h)) return rc;
  if (!h->zg) return HYSCO_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  if (int rc = reset_state(h, s)) return rc;
  HYSCO_TRY(zg_selftest(h->zg, h->st, (long long)spin_cycles, s));
  DevState st;
  HYSCO_TRY(cudaMemcpyAsync(&st, h->st, sizeof(DevState), cudaMemcpyDeviceToHost, s));
  HYSCO_TRY(cudaStreamSynchronize(s));
  if (int rc = reset_state(h, s)) return rc;
  HYSCO_TRY(cudaStreamSynchronize(s));
  return (st.status == HYSCO_ETIMEOUT && st.stop) ? HYSCO_ETIMEOUT : HYSCO_OK;
}

int hysco_zsolve_path(hysco_t h) {
  if (!h) return HYSCO_EINVAL;
  if (int rc = admm_setup(h)) return rc;
  return h->zpath;
}

int hysco_admm(hysco_t h, const void* Ip, const void* Im, float* b_inout,
               const hysco_admm_opts* o, double* stats, hysco_stream_t stream) {
  if (!h || check_admm_opts(h, o) || check_img(h, Ip) || check_img(h, Im) || check_f32(b_inout))
    return HYSCO_EINVAL;
  if (stats && !aligned(stats, 8)) return HYSCO_EINVAL;
  if (int rc = admm_setup(h)) return rc;
  cudaStream_t s = (cudaStream_t)stream;
  h->have_lin = false;
  h->have_factor = false;
  if (o->no_graph) return enqueue_admm(h, Ip, Im, b_inout, o, stats, s);
  const bool cached = h->agexec && h->ag_Ip == Ip && h->ag_Im == Im && h->ag_b == b_inout &&
                      h->ag_stats == stats && same_admm_opts(h->ag_opts, *o);
  if (!cached) {
    if (h->agexec) cudaGraphExecDestroy(h->agexec);
    h->agexec = nullptr;
    cudaGraph_t graph = nullptr;
    bool ok = cudaStreamBeginCapture(h->cap, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
    int rc = ok ? enqueue_admm(h, Ip, Im, b_inout, o, stats, h->cap) : HYSCO_ECUDA;
    cudaError_t ec = cudaStreamEndCapture(h->cap, &graph);
    ok = ok && rc == HYSCO_OK && ec == cudaSuccess && graph != nullptr;
    if (ok) ok = cudaGraphInstantiate(&h->agexec, graph, 0) == cudaSuccess;
    if (graph) cudaGraphDestroy(graph);
    if (!ok) {
      h->agexec = nullptr;
      cudaGetLastError();
      return enqueue_admm(h, Ip, Im, b_inout, o, stats, s);
    }
    h->ag_Ip = Ip;
    h->ag_Im = Im;
    h->ag_b = b_inout;
    h->ag_stats = stats;
    h->ag_opts = *o;
  }
  HYSCO_TRY(cudaGraphLaunch(h->agexec, s));
  return HYSCO_OK;
}

}  // extern "C"

// ------------------------------------------------------------------------------------------
// Batched solve: many handles (volume pairs of any sizes and PE axes) advance through the
// Gauss-Newton loop together.  Per GN iteration the per-pair kernels (evaluation, gamma = 1 trial,
// halvings, update) of different pairs run on concurrent branches, and the PCG of all pairs is
// one cooperative launch of k_pcg_batched.  The fixed launch sequence is captured once in a CUDA
// graph and replayed.  The schedule -- how many branches, and how the PCG grid's blocks are
// shared among the pairs -- is picked by hysco_batch_tune by timing.
// ------------------------------------------------------------------------------------------

struct hysco_batch_ctx {
  int n = 0;
  int device = 0;
  std::vector<hysco_ctx*> hs;
  int grid = 0;                       // k_pcg_batched grid (co-resident blocks)
  BatchPair* d_pairs = nullptr;
  int* d_block_pair = nullptr;
  unsigned* sync = nullptr;
  int branches = 4;                   // schedule: concurrent branches of per-pair kernels
  int policy = 0;                     // schedule: 0 blocks by field size, 1 the same with >= 2 each,
                                      // 2 each pair's own persistent PCG in turn, 3 waves
  // policy 3: the pairs in waves whose PCGs share one cooperative launch (each pair on its own
  // block range with its vectors on chip); a wave runs its whole GN loop before the next
  int wgrid = 0;                      // co-resident blocks of the wave kernel
  std::vector<std::vector<int>> waves;          // pair indices of each wave
  std::vector<std::vector<int>> wave_nblk;      // their block shares
  std::vector<int> wave_onchip;                 // largest on-chip slot count in each wave
  unsigned* wsync = nullptr;                    // sync words of the running wave
  size_t wsync_words = 0;
  cudaStream_t cap = nullptr;
  std::vector<cudaStream_t> side;
  cudaEvent_t fork = nullptr;
  std::vector<cudaEvent_t> join;
  cudaGraphExec_t gexec = nullptr;
  std::vector<const void*> gIp, gIm;
  std::vector<float*> gb;
  std::vector<double*> gst;
  hysco_opts gopts{};
};

namespace {

constexpr int kMaxBranches = 8;
constexpr int kMaxPolicy = 8;
constexpr double kWavePack[3] = {1.0, 1.25, 1.5};   // policies 3, 4, 5 and 6, 7, 8

void batch_free(hysco_batch_ctx* B) {
  if (B->gexec) cudaGraphExecDestroy(B->gexec);
  if (B->wsync) cudaFree(B->wsync);
  if (B->d_pairs) cudaFree(B->d_pairs);
  if (B->d_block_pair) cudaFree(B->d_block_pair);
  if (B->sync) cudaFree(B->sync);
  for (cudaStream_t st : B->side) cudaStreamDestroy(st);
  if (B->cap) cudaStreamDestroy(B->cap);
  if (B->fork) cudaEventDestroy(B->fork);
  for (cudaEvent_t e : B->join) cudaEventDestroy(e);
}

// blocks of the PCG grid per pair: proportional to the pitched field size (largest remainders),
// at least `lo` each
bool batch_shares(const hysco_batch_ctx* B, int lo, std::vector<int>& out) {
  const int n = B->n, G = B->grid;
  if ((long long)n * lo > G) return false;
  double tot = 0.0;
  for (const hysco_ctx* h : B->hs) tot += (double)h->g.nfp;
  std::vector<double> want(n);
  std::vector<int> idx(n);
  int used = 0;
  out.assign(n, lo);
  used = n * lo;
  const int rest = G - used;
  std::vector<double> frac(n);
  int given = 0;
  for (int i = 0; i < n; ++i) {
    want[i] = rest * (double)B->hs[i]->g.nfp / tot;
    int k = (int)want[i];
    out[i] += k;
    given += k;
    frac[i] = want[i] - k;
    idx[i] = i;
  }
  // largest remainders, ties to the lower index
  for (int r = 0; r < rest - given; ++r) {
    int best = -1;
    for (int i = 0; i < n; ++i)
      if (best < 0 || frac[i] > frac[best]) best = i;
    out[best] += 1;
    frac[best] = -1.0;
  }
  return true;
}

// policy 3: pairs sorted by field size, largest first, placed first-fit into waves; a pair needs
// enough blocks to keep its r, p, Hp on chip (kWaveSlots slots per thread) and a wave holds at
// most wgrid blocks and kWaveMax pairs.  A wave's spare blocks go to its pairs in proportion to
// their sizes (fewer groups per block: a shorter stencil phase).
// by_dtype: a wave holds pairs of one image type only (the GN-loop kernel is compiled per type)
int batch_waves(hysco_batch_ctx* B, double pack, bool by_dtype) {
  if (B->wgrid <= 0) return HYSCO_EINVAL;
  const int n = B->n;
  // float4 groups a block takes: kWaveSlots on chip per thread, times `pack` (> 1: the slots past
  // kWaveSlots keep r, p, Hp in global memory, so that more pairs share a wave)
  const long long per_block = (long long)(kPcgBlock * kWaveSlots * pack);
  std::vector<long long> n4(n);
  std::vector<int> need(n), order(n);
  for (int i = 0; i < n; ++i) {
    n4[i] = B->hs[i]->g.nfp / 4;
    need[i] = (int)std::min<long long>((n4[i] + per_block - 1) / per_block, B->wgrid);
    order[i] = i;
  }
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return n4[a] > n4[b]; });
  std::vector<std::vector<int>> waves;
  std::vector<int> used;
  for (int i : order) {
    size_t w = 0;
    while (w < waves.size() &&
           (used[w] + need[i] > B->wgrid || (int)waves[w].size() >= kWaveMax ||
            (by_dtype && B->hs[waves[w][0]]->dtype != B->hs[i]->dtype)))
      ++w;
    if (w == waves.size()) {
      waves.emplace_back();
      used.push_back(0);
    }
    waves[w].push_back(i);
    used[w] += need[i];
  }
  B->waves = waves;
  B->wave_nblk.assign(waves.size(), {});
  B->wave_onchip.assign(waves.size(), 0);
  size_t words = 0;
  for (size_t w = 0; w < waves.size(); ++w) {
    long long tot = 0;
    for (int i : waves[w]) tot += n4[i];
    const int spare = B->wgrid - used[w];
    std::vector<int>& nb = B->wave_nblk[w];
    size_t ww = 0;
    for (int i : waves[w]) {
      const int k = need[i] + (int)((long long)spare * n4[i] / tot);
      nb.push_back(k);
      const long long G = (n4[i] + (long long)k * kPcgBlock - 1) / ((long long)k * kPcgBlock);
      B->wave_onchip[w] = std::max(B->wave_onchip[w], (int)std::min<long long>(G, kWaveSlots));
      ww += pcg_sync_words(k);
    }
    words = std::max(words, ww);
  }
  if (words > B->wsync_words) {
    if (B->wsync) cudaFree(B->wsync);
    B->wsync = nullptr;
    B->wsync_words = 0;
    if (cudaMalloc((void**)&B->wsync, words * sizeof(unsigned)) != cudaSuccess)
      return HYSCO_ENOMEM;
    B->wsync_words = words;
  }
  return HYSCO_OK;
}

int batch_layout(hysco_batch_ctx* B, int policy) {
  if (policy == 2) {   // per-pair persistent PCG: every pair needs its cooperative plan
    for (const hysco_ctx* h : B->hs)
      if (h->pplan.grid <= 0) return HYSCO_EINVAL;
    B->policy = policy;
    return HYSCO_OK;
  }
  if (policy >= 3 && policy <= 5) {
    if (int rc = batch_waves(B, kWavePack[policy - 3], false)) return rc;
    B->policy = policy;
    return HYSCO_OK;
  }
  if (policy >= 6 && policy <= 8) {   // whole GN loops per wave: the kernel must fit each wave
    if (int rc = batch_waves(B, kWavePack[policy - 6], true)) return rc;
    for (size_t w = 0; w < B->waves.size(); ++w)
      if (gn_setup(B->device, B->hs[B->waves[w][0]]->dtype, B->wave_onchip[w]) < 1)
        return HYSCO_EINVAL;
    B->policy = policy;
    return HYSCO_OK;
  }
  std::vector<int> share;
  if (!batch_shares(B, policy == 1 ? 2 : 1, share)) return HYSCO_EINVAL;
  std::vector<BatchPair> pairs(B->n);
  std::vector<int> block_pair(B->grid);
  int b0 = 0;
  for (int i = 0; i < B->n; ++i) {
    hysco_ctx* h = B->hs[i];
    pairs[i] = BatchPair{h->g, h->grad, h->x, h->r, h->z, h->p0, h->Hp, h->dco, h->eco, h->invd,
                         h->st, b0, share[i]};
    for (int k = 0; k < share[i]; ++k) block_pair[b0 + k] = i;
    b0 += share[i];
  }
  if (cudaMemcpy(B->d_pairs, pairs.data(), sizeof(BatchPair) * B->n, cudaMemcpyHostToDevice) !=
          cudaSuccess ||
      cudaMemcpy(B->d_block_pair, block_pair.data(), sizeof(int) * B->grid,
                 cudaMemcpyHostToDevice) != cudaSuccess)
    return HYSCO_ECUDA;
  B->policy = policy;
  return HYSCO_OK;
}

// fork: branches wait for everything enqueued on s so far; join: s waits for every branch
cudaError_t batch_fork(hysco_batch_ctx* B, cudaStream_t s) {
  cudaError_t e = cudaEventRecord(B->fork, s);
  for (int k = 0; k < B->branches && e == cudaSuccess; ++k) e = cudaStreamWaitEvent(B->side[k], B->fork, 0);
  return e;
}
cudaError_t batch_join(hysco_batch_ctx* B, cudaStream_t s) {
  cudaError_t e = cudaSuccess;
  for (int k = 0; k < B->branches && e == cudaSuccess; ++k) {
    e = cudaEventRecord(B->join[k], B->side[k]);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(s, B->join[k], 0);
  }
  return e;
}

// policy 3: wave after wave, each wave's pairs through their whole GN loop together, their per-
// pair kernels on concurrent branches and their PCGs in one cooperative launch per GN step
int enqueue_waves(hysco_batch_ctx* B, const void* const* Ip, const void* const* Im,
                  float* const* b, const hysco_opts* o, double* const* stats, cudaStream_t s) {
  for (size_t w = 0; w < B->waves.size(); ++w) {
    const std::vector<int>& pw = B->waves[w];
    auto branch = [&](int j) { return B->side[j % B->branches]; };
    HYSCO_TRY(batch_fork(B, s));
    for (size_t j = 0; j < pw.size(); ++j) {
      const int i = pw[j];
      hysco_ctx* h = B->hs[i];
      if (int rc = reset_state(h, branch(j))) return rc;
      if (o->init) {
        if (int rc = init_ot_impl(h, Ip[i], Im[i], b[i], o->ot_blur, o->ot_eps, nullptr, nullptr,
                                  branch(j)))
          return rc;
        HYSCO_TRY(launch_feasible_start(h->g, b[i], h->work(), branch(j)));
      }
    }
    // the wave's PCG arguments (fixed for the whole loop)
    PcgWave wv{};
    wv.n = (int)pw.size();
    int blk = 0;
    size_t off = 0;
    for (size_t j = 0; j < pw.size(); ++j) {
      hysco_ctx* h = B->hs[pw[j]];
      const int nb = B->wave_nblk[w][j];
      const long long n4 = h->g.nfp / 4;
      const int G = (int)std::min<long long>((n4 + (long long)nb * kPcgBlock - 1) /
                                                 ((long long)nb * kPcgBlock), kWaveSlots);
      wv.blk0[j] = blk;
      wv.nblk[j] = nb;
      wv.g[j] = h->g;
      wv.a[j] = PcgArgs{h->grad, -1.0f, h->x, h->r, h->z, h->p0, h->p1, h->Hp, h->dco, h->eco,
                        h->invd, B->wsync + off, h->st, o->pcg_max_iters, o->pcg_rtol, G};
      blk += nb;
      off += pcg_sync_words(nb);
    }
    for (int it = 0; it < o->gn_iters; ++it) {
      for (size_t j = 0; j < pw.size(); ++j) {
        hysco_ctx* h = B->hs[pw[j]];
        const int i = pw[j];
        HYSCO_TRY(launch_eval(h->g, h->dtype, Ip[i], Im[i], b[i], nullptr, h->grad, h->dco,
                              h->eco, h->invd, it, h->work(), branch(j)));
      }
      HYSCO_TRY(batch_join(B, s));
      HYSCO_TRY(launch_pcg_wave(wv, blk, B->wave_onchip[w], B->wsync, off, s));
      HYSCO_TRY(batch_fork(B, s));
      for (size_t j = 0; j < pw.size(); ++j) {
        const int i = pw[j];
        hysco_ctx* h = B->hs[i];
        const Geo& g = h->g;
        Work wk = h->work();
        cudaStream_t bs = branch(j);
        HYSCO_TRY(launch_eval_trial(g, h->dtype, Ip[i], Im[i], b[i], h->x, h->grad, h->dco,
                                    h->eco, h->invd, o->ls_max_iters, o->armijo_c1, wk, bs));
        for (int t0 = 1; t0 < o->ls_max_iters; t0 += kLsBatch)
          HYSCO_TRY(launch_linesearch(g, h->dtype, Ip[i], Im[i], b[i], h->x, h->grad, t0,
                                      o->ls_max_iters, o->armijo_c1, wk, bs));
        HYSCO_TRY(launch_update(g, b[i], h->x, it, stats ? stats[i] : nullptr, wk, bs));
      }
    }
    HYSCO_TRY(batch_join(B, s));
  }
  return HYSCO_OK;
}

// policies 6-8: wave after wave, each wave's pairs started (OT) on concurrent branches, then
// their whole GN loops in one persistent cooperative launch, each pair on its own block range
int enqueue_gn_waves(hysco_batch_ctx* B, const void* const* Ip, const void* const* Im,
                     float* const* b, const hysco_opts* o, double* const* stats, cudaStream_t s) {
  for (size_t w = 0; w < B->waves.size(); ++w) {
    const std::vector<int>& pw = B->waves[w];
    auto branch = [&](int j) { return B->side[j % B->branches]; };
    HYSCO_TRY(batch_fork(B, s));
    for (size_t j = 0; j < pw.size(); ++j) {
      const int i = pw[j];
      hysco_ctx* h = B->hs[i];
      if (int rc = reset_state(h, branch(j))) return rc;
      if (o->init) {
        if (int rc = init_ot_impl(h, Ip[i], Im[i], b[i], o->ot_blur, o->ot_eps, nullptr, nullptr,
                                  branch(j)))
          return rc;
        HYSCO_TRY(launch_feasible_start(h->g, b[i], h->work(), branch(j)));
      }
    }
    HYSCO_TRY(batch_join(B, s));
    if (o->gn_iters == 0) continue;
    GnWave wv{};
    wv.n = (int)pw.size();
    int blk = 0;
    size_t off = 0;
    for (size_t j = 0; j < pw.size(); ++j) {
      const int i = pw[j];
      hysco_ctx* h = B->hs[i];
      const int nb = B->wave_nblk[w][j];
      const long long n4 = h->g.nfp / 4;
      const int G = (int)std::min<long long>((n4 + (long long)nb * kPcgBlock - 1) /
                                                 ((long long)nb * kPcgBlock), kWaveSlots);
      wv.blk0[j] = blk;
      wv.nblk[j] = nb;
      wv.g[j] = h->g;
      set_march_warps(wv.g[j], nb * (kPcgBlock / 32));
      wv.a[j] = GnArgs{Ip[i], Im[i], b[i], h->p1, h->grad, stats ? stats[i] : nullptr,
                       PcgArgs{h->grad, -1.0f, h->x, h->r, h->z, h->p0, h->p1, h->Hp, h->dco,
                               h->eco, h->invd, B->wsync + off, h->st, o->pcg_max_iters,
                               o->pcg_rtol, G},
                       o->gn_iters, o->ls_max_iters, o->armijo_c1};
      blk += nb;
      off += pcg_sync_words(nb);
    }
    HYSCO_TRY(launch_gn_wave(wv, B->hs[pw[0]]->dtype, blk, B->wave_onchip[w], B->wsync, off, s));
  }
  return HYSCO_OK;
}

int enqueue_batch(hysco_batch_ctx* B, const void* const* Ip, const void* const* Im,
                  float* const* b, const hysco_opts* o, double* const* stats, cudaStream_t s) {
  if (B->policy >= 6) return enqueue_gn_waves(B, Ip, Im, b, o, stats, s);
  if (B->policy >= 3) return enqueue_waves(B, Ip, Im, b, o, stats, s);
  auto branch = [&](int i) { return B->side[i % B->branches]; };
  HYSCO_TRY(batch_fork(B, s));
  for (int i = 0; i < B->n; ++i) {
    hysco_ctx* h = B->hs[i];
    if (int rc = reset_state(h, branch(i))) return rc;
    if (o->init) {
      if (int rc = init_ot_impl(h, Ip[i], Im[i], b[i], o->ot_blur, o->ot_eps, nullptr, nullptr,
                                branch(i)))
        return rc;
      HYSCO_TRY(launch_feasible_start(h->g, b[i], h->work(), branch(i)));
    }
  }
  for (int it = 0; it < o->gn_iters; ++it) {
    for (int i = 0; i < B->n; ++i) {
      hysco_ctx* h = B->hs[i];
      HYSCO_TRY(launch_eval(h->g, h->dtype, Ip[i], Im[i], b[i], nullptr, h->grad, h->dco, h->eco,
                            h->invd, it, h->work(), branch(i)));
    }
    HYSCO_TRY(batch_join(B, s));
    if (B->policy == 2) {
      // one pair at a time, each with its vectors on chip (a stopped pair's launch returns at once)
      for (int i = 0; i < B->n; ++i)
        if (int rc = run_pcg(B->hs[i], B->hs[i]->grad, -1.0f, B->hs[i]->x, HYSCO_PC_JACOBI,
                             o->pcg_max_iters, o->pcg_rtol, kPcgPersistent, s))
          return rc;
    } else {
      HYSCO_TRY(launch_pcg_batched(B->grid, B->d_pairs, B->d_block_pair, o->pcg_max_iters,
                                   o->pcg_rtol, B->sync, s));
    }
    HYSCO_TRY(batch_fork(B, s));
    for (int i = 0; i < B->n; ++i) {
      hysco_ctx* h = B->hs[i];
      const Geo& g = h->g;
      Work w = h->work();
      cudaStream_t bs = branch(i);
      HYSCO_TRY(launch_eval_trial(g, h->dtype, Ip[i], Im[i], b[i], h->x, h->grad, h->dco, h->eco,
                                  h->invd, o->ls_max_iters, o->armijo_c1, w, bs));
      for (int t0 = 1; t0 < o->ls_max_iters; t0 += kLsBatch)
        HYSCO_TRY(launch_linesearch(g, h->dtype, Ip[i], Im[i], b[i], h->x, h->grad, t0,
                                    o->ls_max_iters, o->armijo_c1, w, bs));
      HYSCO_TRY(launch_update(g, b[i], h->x, it, stats ? stats[i] : nullptr, w, bs));
    }
  }
  HYSCO_TRY(batch_join(B, s));
  return HYSCO_OK;
}

int batch_check(hysco_batch_ctx* B, const void* const* Ip, const void* const* Im,
                float* const* b, const hysco_opts* o, double* const* stats) {
  if (!B || !Ip || !Im || !b || check_opts(o) || o->precond != HYSCO_PC_JACOBI)
    return HYSCO_EINVAL;
  for (int i = 0; i < B->n; ++i) {
    hysco_ctx* h = B->hs[i];
    if (check_img(h, Ip[i]) || check_img(h, Im[i]) || check_f32(b[i])) return HYSCO_EINVAL;
    if (stats && stats[i] && !aligned(stats[i], 8)) return HYSCO_EINVAL;
  }
  return HYSCO_OK;
}

// capture the batch's launch sequence into a graph (exec out); false if capture is unavailable
bool batch_capture(hysco_batch_ctx* B, const void* const* Ip, const void* const* Im,
                   float* const* b, const hysco_opts* o, double* const* stats,
                   cudaGraphExec_t* out) {
  cudaGraph_t graph = nullptr;
  bool ok = cudaStreamBeginCapture(B->cap, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
  int rc = ok ? enqueue_batch(B, Ip, Im, b, o, stats, B->cap) : HYSCO_ECUDA;
  cudaError_t ec = cudaStreamEndCapture(B->cap, &graph);
  ok = ok && rc == HYSCO_OK && ec == cudaSuccess && graph != nullptr;
  if (ok) ok = cudaGraphInstantiate(out, graph, 0) == cudaSuccess;
  if (graph) cudaGraphDestroy(graph);
  if (!ok) cudaGetLastError();
  return ok;
}

}  // namespace

extern "C" {

int hysco_batch_create(int n, const hysco_t* handles, hysco_batch_t* out) {
  if (!out || !handles || n < 1) return HYSCO_EINVAL;
  *out = nullptr;
  for (int i = 0; i < n; ++i) {
    if (!handles[i]) return HYSCO_EINVAL;
    for (int j = 0; j < i; ++j)
      if (handles[j] == handles[i]) return HYSCO_EINVAL;   // a pair's workspace is used once
    if (handles[i]->device != handles[0]->device) return HYSCO_EINVAL;
  }
  int sms = 0;
  const int per_sm = pcg_batched_blocks_per_sm(handles[0]->device);
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, handles[0]->device) !=
      cudaSuccess)
    return HYSCO_ECUDA;
  if (per_sm < 1 || n > sms * per_sm) return HYSCO_EINVAL;
  const int grid = std::min(sms * per_sm, 32 * kTagWordsPerLaneHost);
  if (n > grid) return HYSCO_EINVAL;
  auto* B = new (std::nothrow) hysco_batch_ctx;
  if (!B) return HYSCO_ENOMEM;
  B->n = n;
  B->device = handles[0]->device;
  B->hs.assign(handles, handles + n);
  B->grid = grid;
  B->wgrid = pcg_wave_setup(B->device);
  bool ok = cudaMalloc((void**)&B->d_pairs, sizeof(BatchPair) * n) == cudaSuccess &&
            cudaMalloc((void**)&B->d_block_pair, sizeof(int) * B->grid) == cudaSuccess &&
            cudaMalloc((void**)&B->sync, pcg_sync_words(B->grid) * sizeof(unsigned)) ==
                cudaSuccess &&
            cudaStreamCreateWithFlags(&B->cap, cudaStreamNonBlocking) == cudaSuccess &&
            cudaEventCreateWithFlags(&B->fork, cudaEventDisableTiming) == cudaSuccess;
  for (int k = 0; ok && k < kMaxBranches; ++k) {
    cudaStream_t st = nullptr;
    cudaEvent_t ev = nullptr;
    ok = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) == cudaSuccess &&
         cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) == cudaSuccess;
    if (st) B->side.push_back(st);
    if (ev) B->join.push_back(ev);
  }
  B->branches = n < 4 ? n : 4;
  int rc = ok ? batch_layout(B, 0) : HYSCO_ENOMEM;
  if (rc != HYSCO_OK) {
    batch_free(B);
    delete B;
    return rc;
  }
  *out = B;
  return HYSCO_OK;
}

void hysco_batch_destroy(hysco_batch_t B) {
  if (!B) return;
  batch_free(B);
  delete B;
}

int hysco_batch_schedule(hysco_batch_t B, int32_t out[3]) {
  if (!B || !out) return HYSCO_EINVAL;
  out[0] = B->branches;
  out[1] = B->policy;
  out[2] = B->grid;
  return HYSCO_OK;
}

int hysco_batch_set_schedule(hysco_batch_t B, int branches, int policy) {
  if (!B || branches < 1 || branches > kMaxBranches || branches > B->n || policy < 0 ||
      policy > kMaxPolicy)
    return HYSCO_EINVAL;
  const int old = B->policy;
  if (int rc = batch_layout(B, policy)) {
    batch_layout(B, old);
    return rc;
  }
  B->branches = branches;
  if (B->gexec) cudaGraphExecDestroy(B->gexec);   // the cached graph used the old schedule
  B->gexec = nullptr;
  return HYSCO_OK;
}

int hysco_batch_solve(hysco_batch_t B, const void* const* Ip, const void* const* Im,
                      float* const* b, const hysco_opts* o, double* const* stats,
                      hysco_stream_t stream) {
  if (int rc = batch_check(B, Ip, Im, b, o, stats)) return rc;
  cudaStream_t s = (cudaStream_t)stream;
  for (hysco_ctx* h : B->hs) h->have_lin = false;
  std::vector<double*> st(B->n, nullptr);
  if (stats)
    for (int i = 0; i < B->n; ++i) st[i] = stats[i];
  const bool cached = B->gexec && same_opts(B->gopts, *o) &&
                      std::equal(B->gIp.begin(), B->gIp.end(), Ip) &&
                      std::equal(B->gIm.begin(), B->gIm.end(), Im) &&
                      std::equal(B->gb.begin(), B->gb.end(), b) && B->gst == st;
  if (!o->no_graph && !cached) {
    if (B->gexec) cudaGraphExecDestroy(B->gexec);
    B->gexec = nullptr;
    if (batch_capture(B, Ip, Im, b, o, stats, &B->gexec)) {
      B->gIp.assign(Ip, Ip + B->n);
      B->gIm.assign(Im, Im + B->n);
      B->gb.assign(b, b + B->n);
      B->gst = st;
      B->gopts = *o;
    }
  }
  if (!o->no_graph && B->gexec) {
    HYSCO_TRY(cudaGraphLaunch(B->gexec, s));
    return HYSCO_OK;
  }
  return enqueue_batch(B, Ip, Im, b, o, stats, s);
}

int hysco_batch_tune(hysco_batch_t B, const void* const* Ip, const void* const* Im,
                     const hysco_opts* o, hysco_stream_t stream) {
  if (!B || !Ip || !Im || check_opts(o) || o->precond != HYSCO_PC_JACOBI) return HYSCO_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  // scratch fields: the trial solves must not touch the caller's fields
  std::vector<float*> scratch(B->n, nullptr);
  int rc = HYSCO_OK;
  for (int i = 0; i < B->n && rc == HYSCO_OK; ++i)
    if (cudaMalloc((void**)&scratch[i], (size_t)B->hs[i]->nfld * sizeof(float)) != cudaSuccess)
      rc = HYSCO_ENOMEM;
  if (rc == HYSCO_OK) rc = batch_check(B, Ip, Im, scratch.data(), o, nullptr);
  hysco_opts t = *o;
  t.init = 1;   // the trial solves start from the OT initialisation
  t.gn_iters = o->gn_iters < 2 ? o->gn_iters : 2;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (rc == HYSCO_OK && (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess))
    rc = HYSCO_ECUDA;
  float best = 1e30f;
  int best_br = B->branches, best_pol = B->policy;
  for (int pol = 0; pol <= kMaxPolicy && rc == HYSCO_OK; ++pol) {
    if (batch_layout(B, pol) != HYSCO_OK) continue;   // policy not feasible for this batch
    for (int br = 1; br <= kMaxBranches && br <= B->n && rc == HYSCO_OK; br *= 2) {
      B->branches = br;
      cudaGraphExec_t ge = nullptr;
      if (!batch_capture(B, Ip, Im, scratch.data(), &t, nullptr, &ge)) { rc = HYSCO_ECUDA; break; }
      float ms = 0.f;
      bool ok = cudaGraphLaunch(ge, s) == cudaSuccess && cudaEventRecord(e0, s) == cudaSuccess &&
                cudaGraphLaunch(ge, s) == cudaSuccess && cudaGraphLaunch(ge, s) == cudaSuccess &&
                cudaEventRecord(e1, s) == cudaSuccess && cudaEventSynchronize(e1) == cudaSuccess &&
                cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess;
      cudaGraphExecDestroy(ge);
      if (!ok) { rc = HYSCO_ECUDA; break; }
      if (ms < best) { best = ms; best_br = br; best_pol = pol; }
    }
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  for (float* p : scratch)
    if (p) cudaFree(p);
  B->branches = best_br;
  if (int rl = batch_layout(B, best_pol)) rc = rc == HYSCO_OK ? rl : rc;
  if (B->gexec) cudaGraphExecDestroy(B->gexec);   // the cached graph used the old schedule
  B->gexec = nullptr;
  for (hysco_ctx* h : B->hs) h->have_lin = false;
  return rc;
}

int hysco_selftest_barrier(int grid, int missing_block, int64_t spin_cycles,
                           hysco_stream_t stream) {
  if (grid < 1 || grid > 64 || missing_block < -1 || missing_block >= grid || spin_cycles < 1 ||
      spin_cycles > 4000000000LL)
    return HYSCO_EINVAL;
  int dev = 0, coop = 0, per_sm = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return HYSCO_ECUDA;
  per_sm = pcg_batched_blocks_per_sm(dev);
  if (!coop || grid > sms * per_sm) return HYSCO_EINVAL;   // every block must be co-resident
  unsigned* sync = nullptr;
  int* flag = nullptr;
  cudaStream_t s = (cudaStream_t)stream;
  int rc = HYSCO_ECUDA, host_flag = 0;
  if (cudaMalloc((void**)&sync, pcg_sync_words(grid) * sizeof(unsigned)) == cudaSuccess &&
      cudaMalloc((void**)&flag, sizeof(int)) == cudaSuccess &&
      launch_barrier_selftest(grid, missing_block, (long long)spin_cycles, sync, flag, s) ==
          cudaSuccess &&
      cudaMemcpyAsync(&host_flag, flag, sizeof(int), cudaMemcpyDeviceToHost, s) == cudaSuccess &&
      cudaStreamSynchronize(s) == cudaSuccess)
    rc = host_flag == 1 ? HYSCO_ETIMEOUT : (host_flag == 0 ? HYSCO_OK : HYSCO_ENONFINITE);
  if (sync) cudaFree(sync);
  if (flag) cudaFree(flag);
  return rc;
}

}  // extern "C"
