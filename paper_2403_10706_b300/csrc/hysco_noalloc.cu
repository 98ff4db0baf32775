// hysco_eval_static: the objective J (and optionally its gradient) for callers that must not
// allocate device memory.  The handle-based hysco_eval needs a handle whose workspace comes from
// cudaMalloc; this entry point takes the geometry by value and keeps its only scratch -- the
// per-block partial sums of the grid reduction and the ticket counter of the block that finishes
// it -- in the file-scope device array below, which every GPU that loads the library holds until
// the process exits.
//
// Host code must not pass the array's name to a kernel: on the host that name is a stand-in, not
// a device address.  The first call in each CUDA context (the device's primary context, with that
// device current) looks up the array's device address with cudaGetSymbolAddress and remembers it
// under the context's unique id; every call then passes that address to the kernel.  A context
// that is destroyed and re-created (cudaDeviceReset) gets a new id, and so a fresh lookup.
#include <cuda.h>

#include <cmath>
#include <mutex>

#include "../../include/hysco.h"
#include "eval_common.cuh"

namespace hysco {
namespace {

constexpr int kStaticMaxBlocks = 32768;   // largest reduction grid served (384 KiB of partials)
constexpr int kStaticTerms = 3;           // D, S and P
constexpr size_t kCounterBytes = 256;     // ticket counter, padded to keep the partials aligned
constexpr size_t kStaticScratchBytes =
    kCounterBytes + sizeof(float) * (size_t)kStaticMaxBlocks * kStaticTerms;

static __device__ __align__(256) unsigned char g_eval_scratch[kStaticScratchBytes];

constexpr int kMaxContexts = 64;
struct ScratchEntry {
  unsigned long long ctx_id;
  void* addr;
};
std::mutex g_setup_mutex;
ScratchEntry g_scratch[kMaxContexts] = {};
int g_nscratch = 0;
using CtxGetCurrent = CUresult (*)(CUcontext*);
using CtxGetId = CUresult (*)(CUcontext, unsigned long long*);
CtxGetCurrent g_ctx_current = nullptr;
CtxGetId g_ctx_id = nullptr;

// unique id of the calling thread's current context (the driver entry points are looked up once)
cudaError_t current_context_id(unsigned long long* id) {
  if (!g_ctx_current || !g_ctx_id) {
    void* f0 = nullptr;
    void* f1 = nullptr;
    cudaDriverEntryPointQueryResult q0, q1;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f0, 12000, cudaEnableDefault, &q0) !=
            cudaSuccess ||
        cudaGetDriverEntryPointByVersion("cuCtxGetId", &f1, 12000, cudaEnableDefault, &q1) !=
            cudaSuccess ||
        q0 != cudaDriverEntryPointSuccess || q1 != cudaDriverEntryPointSuccess)
      return cudaErrorNotSupported;
    g_ctx_current = reinterpret_cast<CtxGetCurrent>(f0);
    g_ctx_id = reinterpret_cast<CtxGetId>(f1);
  }
  CUcontext ctx = nullptr;
  if (g_ctx_current(&ctx) != CUDA_SUCCESS || !ctx) return cudaErrorDeviceUninitialized;
  return g_ctx_id(ctx, id) == CUDA_SUCCESS ? cudaSuccess : cudaErrorDeviceUninitialized;
}

// device address of g_eval_scratch in the current context (looked up once per context)
cudaError_t scratch_address(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  e = cudaSetDevice(dev);   // makes the device's primary context current, initialised
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  unsigned long long id = 0;
  e = current_context_id(&id);
  if (e != cudaSuccess) return e;
  for (int i = 0; i < g_nscratch; ++i)
    if (g_scratch[i].ctx_id == id) {
      *out = g_scratch[i].addr;
      return cudaSuccess;
    }
  void* p = nullptr;
  e = cudaGetSymbolAddress(&p, g_eval_scratch);
  if (e != cudaSuccess) return e;
  ScratchEntry ent{id, p};
  if (g_nscratch < kMaxContexts) g_scratch[g_nscratch++] = ent;
  else g_scratch[id % kMaxContexts] = ent;   // many re-created contexts: reuse a slot
  *out = p;
  return cudaSuccess;
}

// Same per-cell and per-node arithmetic as the handle-based eval kernel; no Gauss-Newton
// coefficients are written and the last block stores J, D, S, P straight into `terms`.
template <typename TI, int SEG>
__global__ void __launch_bounds__(kBlock)
k_eval_static(Geo g, const TI* __restrict__ Ip, const TI* __restrict__ Im,
              const float* __restrict__ b, float* __restrict__ grad, double* terms,
              unsigned char* scratch) {
  unsigned* counter = reinterpret_cast<unsigned*>(scratch);
  float* partials = reinterpret_cast<float*>(scratch + kCounterBytes);
  const int inner = g.inner, m = g.m;
  int c = blockIdx.x * blockDim.x + threadIdx.x;
  const bool act = c < g.ncols;
  c = act ? c : g.ncols - 1;
  const int k0 = blockIdx.y * SEG;
  const int ib = col_base(c, inner, g.img_ostride), fb = col_base(c, inner, g.fld_ostride);
  const TI* Ipc = Ip + ib;
  const TI* Imc = Im + ib;
  const ColNbrs nb = col_nbrs(g, c, fb);
  float bw[SEG + 2], bAm[SEG], bAp[SEG], bBm[SEG], bBp[SEG];
#pragma unroll
  for (int j = 0; j < SEG + 2; ++j) bw[j] = __ldg(b + fb + min(max(k0 - 1 + j, 0), m) * inner);
#pragma unroll
  for (int j = 0; j < SEG; ++j) {
    int o = min(k0 + j, m) * inner;
    bAm[j] = __ldg(b + nb.Am + o); bAp[j] = __ldg(b + nb.Ap + o);
    bBm[j] = __ldg(b + nb.Bm + o); bBp[j] = __ldg(b + nb.Bp + o);
  }
  float cr[SEG + 1], cjl[SEG + 1], cjr[SEG + 1], cdphi[SEG + 1], cphi[SEG + 1];
#pragma unroll
  for (int j = 0; j <= SEG; ++j) {
    int jc = k0 - 1 + j;
    bool cv = jc >= 0 && jc < m;
    CellLin q = cell_lin(Ipc, Imc, inner, m, jc, bw[j], bw[j + 1], g.half_beta);
    cr[j] = cv ? q.r : 0.f;
    cjl[j] = cv ? q.jl : 0.f;
    cjr[j] = cv ? q.jr : 0.f;
    cdphi[j] = cv ? q.dphi : 0.f;
    cphi[j] = cv ? q.phi : 0.f;
  }
  float accD = 0.f, accS = 0.f, accP = 0.f;
#pragma unroll
  for (int j = 0; j < SEG; ++j) {
    int k = k0 + j;
    if (!act || k > m) continue;
    float bk = bw[j + 1], bn = bw[j + 2];
    float lap = (bk - bw[j]) + (bk - bn) + g.wA * ((bk - bAm[j]) + (bk - bAp[j])) +
                g.wB * ((bk - bBm[j]) + (bk - bBp[j]));
    float dPE = bn - bk, dA = bAp[j] - bk, dB = bBp[j] - bk;
    accS += dPE * dPE + g.wA * dA * dA + g.wB * dB * dB;
    accD += cr[j + 1] * cr[j + 1];
    accP += cphi[j + 1];
    float gk = g.vol * (cjr[j] * cr[j] + cjl[j + 1] * cr[j + 1] + g.alpha * lap +
                        g.half_beta * (cdphi[j] - cdphi[j + 1]));
    if (grad) grad[fb + k * inner] = gk;
  }
  float v[kStaticTerms] = {accD, accS, accP};
  double tot[kStaticTerms];
  if (grid_sum<kStaticTerms>(v, partials, counter, tot)) {
    double hv = 0.5 * (double)g.vol;
    double D = hv * tot[0], S = hv * tot[1], P = hv * tot[2];
    terms[0] = D + g.alpha_d * S + g.beta_d * P;
    terms[1] = D;
    terms[2] = S;
    terms[3] = P;
  }
}

int make_geo(const int64_t dims[3], const double spacing[3], int pe_dim, double alpha,
             double beta, Geo* out) {
  if (!dims || !spacing || pe_dim < 0 || pe_dim > 2) return HYSCO_EINVAL;
  if (!(alpha >= 0.0) || !(beta >= 0.0) || !std::isfinite(alpha) || !std::isfinite(beta))
    return HYSCO_EINVAL;
  for (int a = 0; a < 3; ++a) {
    if (dims[a] < 1) return HYSCO_EINVAL;
    if (!(spacing[a] > 0.0) || !std::isfinite(spacing[a])) return HYSCO_EINVAL;
  }
  if (dims[pe_dim] < 2) return HYSCO_EINVAL;
  long long nimg = dims[0] * dims[1] * dims[2];
  long long m = dims[pe_dim];
  if (nimg / m * (m + 1) >= (1LL << 31)) return HYSCO_EINVAL;
  Geo g{};
  g.m = (int)m;
  g.E = (int)m + 1;
  g.ncols = (int)(nimg / m);
  long long inner = 1;
  for (int a = pe_dim + 1; a < 3; ++a) inner *= dims[a];
  g.inner = (int)inner;
  int q[2], k = 0;
  for (int a = 0; a < 3; ++a)
    if (a != pe_dim) q[k++] = a;
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
  *out = g;
  return HYSCO_OK;
}

}  // namespace
}  // namespace hysco

extern "C" int hysco_eval_static(const int64_t dims[3], const double spacing[3], int pe_dim,
                                 double alpha, double beta, int img_dtype, const void* Ip,
                                 const void* Im, const float* b, double* terms_dev, float* grad,
                                 hysco_stream_t stream) {
  using namespace hysco;
  Geo g;
  if (int rc = make_geo(dims, spacing, pe_dim, alpha, beta, &g)) return rc;
  if (img_dtype < HYSCO_F32 || img_dtype > HYSCO_F16) return HYSCO_EINVAL;
  size_t esz = img_dtype == HYSCO_F32 ? 4 : 2;
  if (!Ip || !Im || ((uintptr_t)Ip % esz) || ((uintptr_t)Im % esz)) return HYSCO_EINVAL;
  if (!b || ((uintptr_t)b % 4) || (grad && ((uintptr_t)grad % 4))) return HYSCO_EINVAL;
  if (!terms_dev || ((uintptr_t)terms_dev % 8)) return HYSCO_EINVAL;
  dim3 grid(ceil_div(g.ncols, kBlock), ceil_div(g.E, kSeg));
  if ((long long)grid.x * grid.y > kStaticMaxBlocks) return HYSCO_EINVAL;
  void* scratch = nullptr;
  if (scratch_address(&scratch) != cudaSuccess) return HYSCO_ECUDA;
  cudaStream_t s = (cudaStream_t)stream;
  // the ticket counter must start at zero; the previous call's partials are simply overwritten
  if (cudaMemsetAsync(scratch, 0, sizeof(unsigned), s) != cudaSuccess) return HYSCO_ECUDA;
  unsigned char* sc = static_cast<unsigned char*>(scratch);
  switch (img_dtype) {
    case HYSCO_F32:
      k_eval_static<float, kSeg><<<grid, kBlock, 0, s>>>(g, (const float*)Ip, (const float*)Im, b,
                                                         grad, terms_dev, sc);
      break;
    case HYSCO_BF16:
      k_eval_static<__nv_bfloat16, kSeg><<<grid, kBlock, 0, s>>>(
          g, (const __nv_bfloat16*)Ip, (const __nv_bfloat16*)Im, b, grad, terms_dev, sc);
      break;
    default:
      k_eval_static<__half, kSeg><<<grid, kBlock, 0, s>>>(g, (const __half*)Ip, (const __half*)Im,
                                                          b, grad, terms_dev, sc);
      break;
  }
  return cudaGetLastError() == cudaSuccess ? HYSCO_OK : HYSCO_ECUDA;
}
