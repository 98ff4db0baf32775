/*
 * hysco.h -- C ABI of libhysco, the B300 (sm_103a) implementation of the hot path of the
 * reversed-gradient-polarity field-map estimation of PyHySCO (Julian & Ruthotto,
 * arXiv 2403.10706): the objective J(b) = D(b) + alpha S(b) + beta P(b), its gradient, the
 * Gauss-Newton Hessian-vector product, the Jacobi and per-column block preconditioners, the 1D
 * optimal-transport initialiser and the GN-PCG solve.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - Images are C-contiguous d0 x d1 x d2 arrays (last index fastest) in DEVICE memory, element
 *    type fixed at hysco_create (float32, bfloat16 or float16).  The phase-encoding (PE) axis is
 *    pe_dim (0-based; the paper's command line counts from 1).  m = dims[pe_dim].
 *  - The field map b lives on the e_p-staggered grid (Sec. 2.1, discretisation paragraph): its
 *    dims are the image dims with dims[pe_dim] replaced by m + 1 (see hysco_field_dims).  It is
 *    float32 in device memory and expressed in PE-voxel units (b in mm = spacing[pe_dim] * b).
 *    The objective is the paper's physical J (spacing in mm, midpoint quadrature).
 *  - Every pointer argument is caller-owned device memory unless stated otherwise, must be
 *    4-byte aligned (2-byte for 16-bit images), and must not alias another argument.  The handle
 *    owns only its own device workspace (allocated in hysco_create, freed in hysco_destroy).
 *  - Work is enqueued on `stream` (a cudaStream_t; NULL = legacy default stream) and is
 *    asynchronous: argument errors are returned before anything is enqueued; numerical outcomes
 *    (barrier infeasibility, non-finite values) are recorded on the device and returned by
 *    hysco_last_status, which synchronises the stream.
 *  - A handle is not thread-safe and its calls must not overlap on different streams; distinct
 *    handles are independent.
 *  - Return value: hysco_status (0 = success, < 0 = error, > 0 = non-error condition).
 */
#ifndef HYSCO_H
#define HYSCO_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct hysco_ctx* hysco_t;
typedef struct CUstream_st* hysco_stream_t;   /* identical to cudaStream_t */

typedef enum {
  HYSCO_OK = 0,
  HYSCO_INFEASIBLE = 1,   /* some |d_v b| >= 1: the barrier of Eq. 3 makes J = +inf */
  HYSCO_EINVAL = -1,      /* bad argument (dims, pe_dim, spacing, weights, pointer, option) */
  HYSCO_ECUDA = -2,       /* a CUDA runtime call failed */
  HYSCO_ENOMEM = -3,      /* device workspace allocation failed */
  HYSCO_ENONFINITE = -4,  /* NaN met in J (non-finite input) */
  HYSCO_ENOTREADY = -5,   /* hysco_hessvec / hysco_precond before any hysco_eval */
  HYSCO_ETIMEOUT = -6     /* a device-wide barrier of the persistent PCG kernel timed out */
} hysco_status;

typedef enum { HYSCO_F32 = 0, HYSCO_BF16 = 1, HYSCO_F16 = 2 } hysco_dtype;
typedef enum { HYSCO_PC_JACOBI = 0, HYSCO_PC_COLUMN = 1 } hysco_precond_kind;

/* Options of the GN-PCG solve (Sec. 2.3.1).  hysco_default_opts fills the paper's values. */
typedef struct {
  int32_t gn_iters;       /* fixed number of Gauss-Newton iterations (default 10) */
  int32_t pcg_max_iters;  /* PCG iterations per GN step, <= 64 (paper: 10) */
  int32_t ls_max_iters;   /* Armijo trials gamma = 1, 1/2, ..., <= 16 (default 10) */
  int32_t precond;        /* hysco_precond_kind (paper default: Jacobi) */
  int32_t init;           /* 1 = OT initialisation (Sec. 2.2), 0 = start from b_inout */
  int32_t ot_blur;        /* 1 = 3x3x3 Gaussian blur, sigma 1 voxel, after OT (Sec. 2.4) */
  double pcg_rtol;        /* stop PCG when ||r|| / ||r0|| < pcg_rtol (paper: 0.1) */
  double armijo_c1;       /* sufficient-decrease constant (default 1e-4) */
  double ot_eps;          /* OT positivity shift factor (default 1e-3) */
  int32_t pcg_path;       /* Jacobi PCG: 0 = the fastest form the device supports (default: 2,
                             else 1); 1 = separate kernels per phase; 2 = one persistent
                             cooperative kernel per GN step with two device-wide barriers per PCG
                             iteration, or HYSCO_EINVAL; 3 = one persistent kernel with one
                             barrier per iteration (the direction product p.Hp taken from its
                             bilinear expansion in H z, see k_pcg_persistent.cu), or HYSCO_EINVAL.
                             1 and 2 have the same arithmetic; 3 gives the same iterates in exact
                             arithmetic; 4 = hysco_solve only: the whole GN loop (evaluation,
                             PCG as in 2, the gamma = 1 trial, halvings, update) in one persistent
                             cooperative launch, every scalar decision on the device (hysco_pcg
                             takes it as 2), or HYSCO_EINVAL.  4 gives the iterates of 2 up to the
                             rounding of J's sums.  The column preconditioner always uses 1. */
  int32_t no_graph;       /* 0 (default): the solve's fixed launch sequence is captured once in a
                             CUDA graph per (images, field, stats, options) and replayed; 1: launch
                             the kernels directly every call.  Same kernels either way. */
} hysco_opts;

/* Per-GN-iteration record written by hysco_solve when `stats` is non-NULL (device memory,
 * gn_iters x HYSCO_NSTATS doubles): J, D, S, P at the iterate, ||grad J||, grad^T q, accepted
 * step gamma (0 = rejected), PCG iterations, final PCG relative residual, line-search trials. */
enum { HYSCO_NSTATS = 10 };

void hysco_default_opts(hysco_opts* opts);
const char* hysco_strerror(int status);
/* Library version string (static storage). */
const char* hysco_version(void);

/* Create a handle for one problem geometry (Sec. 2.1, Eq. 4):
 *   dims[3]     image dims (each >= 1, dims[pe_dim] >= 2, total < 2^31 voxels),
 *   spacing[3]  voxel sizes in mm (> 0),
 *   pe_dim      phase-encoding axis 0..2,
 *   alpha, beta smoothness and barrier weights (>= 0; the paper uses 300 and 1e-4),
 *   img_dtype   hysco_dtype of the images passed to every later call.
 * Allocates the device workspace on the current device.  *out is NULL on failure. */
int hysco_create(const int64_t dims[3], const double spacing[3], int pe_dim, double alpha,
                 double beta, int img_dtype, hysco_t* out);
void hysco_destroy(hysco_t h);
/* Field dims (image dims with the PE extent + 1). */
int hysco_field_dims(hysco_t h, int64_t out[3]);

/* 1D optimal-transport initial field (Sec. 2.2): per PE column, shift both images to positive
 * measures (s = max(0, -min) + eps * max|I| over both images), form the normalised cumulative
 * sums C+- at the m + 1 nodes, invert them with the linear spline, and set
 *   b0_k = 1/4 [ (C+^{-1}(C-(k)) - k) - (C-^{-1}(C+(k)) - k) ]
 * (half the displacement of T- minus half that of T+, T+- = C_half^{-1} o C+-).  Columns with
 * no mass get 0.  blur != 0 applies the separable 3x3x3 Gaussian (sigma 1 voxel, replicate
 * boundary) of Sec. 2.4.  b_out: field-shaped float32. */
int hysco_init_ot(hysco_t h, const void* Ip, const void* Im, float* b_out, int blur, double eps,
                  hysco_stream_t stream);

/* Objective at b (Eq. 1-5): terms_dev[0..3] = J, D, S, P (device doubles).  grad (nullable,
 * field-shaped) receives grad J = vol [Jr^T r + alpha h^2 L b + beta/2 D^T phi'(delta)].  Also
 * stores the per-node Gauss-Newton coefficients at b in the handle, used by hysco_hessvec and
 * hysco_precond until the next hysco_eval / hysco_solve on this handle. */
int hysco_eval(hysco_t h, const void* Ip, const void* Im, const float* b, double* terms_dev,
               float* grad, hysco_stream_t stream);

/* Hv = H_J v with the Gauss-Newton Hessian of Sec. 2.3.1 about the field of the last
 * hysco_eval: H_J = vol [Jr^T Jr + alpha h^2 L + beta/2 D^T diag(phi''(delta)) D].
 * v, Hv: field-shaped float32. */
int hysco_hessvec(hysco_t h, const float* v, float* Hv, hysco_stream_t stream);

/* z = M^{-1} r about the field of the last hysco_eval: kind = HYSCO_PC_JACOBI divides by the
 * diagonal of H_J (Sec. 2.3.1); HYSCO_PC_COLUMN solves with the exact tridiagonal diagonal
 * block of H_J belonging to each PE column (the block-diagonal preconditioner mentioned at the
 * end of Sec. 2.3.1).  HYSCO_PC_COLUMN requires m <= 1024. */
int hysco_precond(hysco_t h, const float* r, float* z, int kind, hysco_stream_t stream);

/* The PCG step of Sec. 2.3.1 on its own: q ~= H_J^{-1} rhs about the field of the last
 * hysco_eval, x0 = 0, at most max_iters (<= 64) iterations, stop when ||r|| / ||r0|| < rtol or
 * p^T H p <= 0; preconditioner `precond` (hysco_precond_kind); pcg_path as in hysco_opts.  In a
 * Gauss-Newton step rhs = -grad J.  rhs, q: field-shaped float32, distinct.
 * hysco_last_status afterwards also reports a persistent-kernel barrier timeout. */
int hysco_pcg(hysco_t h, const float* rhs, float* q, int precond, int max_iters, double rtol,
              int pcg_path, hysco_stream_t stream);

/* Corrected images at b (Eq. 1, the Jacobian-modulation correction of Sec. 2.4):
 * Tp = I+(x + b v)(1 + d_v b), Tm = I-(x - b v)(1 - d_v b), image-shaped float32. */
int hysco_correct(hysco_t h, const void* Ip, const void* Im, const float* b, float* Tp,
                  float* Tm, hysco_stream_t stream);

/* Adjoint (vector-Jacobian product) of hysco_correct at b, for differentiation (Eq. 1 at fixed
 * b).  Given the sensitivities gTp, gTm of a scalar loss to Tp and Tm (image-shaped float32,
 * device; either may be NULL, meaning zero) it writes
 *   dIp = (dTp/dIp)^T gTp,  dIm = (dTm/dIm)^T gTm        image-shaped float32 (sensitivity to
 *                                                        the stored image values, whatever the
 *                                                        handle's image dtype)
 *   db  = (dTp/db)^T gTp + (dTm/db)^T gTm                 field-shaped float32
 * Each output may be NULL (not computed).  Per cell, Tp depends on I+ at the two voxels around
 * t+ with weights (1 - w, w) times (1 + d_v b), and on b through t+ (slope of I+) and d_v b; Tm
 * likewise with t-, 1 - d_v b.  Cells and weights are recomputed from b, not stored.
 * Deterministic (no atomics).  Outputs must not alias the inputs; they are overwritten. */
int hysco_correct_adjoint(hysco_t h, const void* Ip, const void* Im, const float* b,
                          const float* gTp, const float* gTm, float* dIp, float* dIm, float* db,
                          hysco_stream_t stream);

/* The corrected image of Sec. 2.4 ("Image Correction"): the average of the two corrected images
 * of Eq. 1, T = 1/2 (Tp + Tm), image-shaped float32 -- the image PyHySCO returns. */
int hysco_correct_mean(hysco_t h, const void* Ip, const void* Im, const float* b, float* T,
                       hysco_stream_t stream);

/* Adjoint of hysco_correct_mean at b: for the sensitivity gT of a scalar loss to T (image-shaped
 * float32, device, not NULL) it writes dIp, dIm and db as hysco_correct_adjoint does for
 * gTp = gTm = gT / 2 (each output nullable; same layout, determinism and aliasing rules). */
int hysco_correct_mean_adjoint(hysco_t h, const void* Ip, const void* Im, const float* b,
                               const float* gT, float* dIp, float* dIm, float* db,
                               hysco_stream_t stream);

/* Implicit differentiation through a solve (the Gauss-Newton system of Sec. 2.3.1 at a solution):
 * at a stationary point b of J the gradient g(b; theta) = 0 defines b as a function of every input
 * theta, and for a loss L(b), with H the Gauss-Newton Hessian at b standing in for J's Hessian,
 *   dL/dtheta = -(dg/dtheta)^T v,   H v = dL/db.
 * hysco_implicit_parts takes v (field-shaped float32, caller's layout) and writes
 *   dIp = -d(v^T g)/dI+, dIm = -d(v^T g)/dI-   image-shaped float32 (nullable; only the distance
 *                                              term of Eq. 2 depends on the images)
 *   dtheta[0] = -v^T dg/dalpha = -v^T grad S, dtheta[1] = -v^T dg/dbeta = -v^T grad P
 *                                              (2 doubles, device, nullable).
 * hysco_solve_adjoint computes the Gauss-Newton linearisation at b (as hysco_eval does, replacing
 * the handle's), solves H v = dLdb by Jacobi PCG (x0 = 0, at most max_iters <= 1000 iterations,
 * relative residual rtol), writes v to v_out when non-NULL, then the parts as above.  The total
 * derivative of a loss of the solved field adds these to the loss's direct dependence on the
 * images.  Outputs must not alias the inputs. */
int hysco_implicit_parts(hysco_t h, const void* Ip, const void* Im, const float* b,
                         const float* v, float* dIp, float* dIm, double* dtheta,
                         hysco_stream_t stream);
int hysco_solve_adjoint(hysco_t h, const void* Ip, const void* Im, const float* b,
                        const float* dLdb, int max_iters, double rtol, float* v_out, float* dIp,
                        float* dIm, double* dtheta, hysco_stream_t stream);

/* Gradient of gJ * J with respect to the two images at fixed b.  Only the distance term of Eq. 2
 * depends on them: dIp = gJ vol (dTp/dIp)^T r, dIm = -gJ vol (dTm/dIm)^T r with the residual
 * r = Tp - Tm recomputed.  (With respect to b it is gJ times the gradient of hysco_eval; with
 * respect to alpha and beta it is gJ S and gJ P.)  Outputs image-shaped float32, either may be
 * NULL; they must not alias the inputs. */
int hysco_image_grad(hysco_t h, const void* Ip, const void* Im, const float* b, double gJ,
                     float* dIp, float* dIm, hysco_stream_t stream);

/* Least-squares corrected image at b (Sec. 2.4 "Image Correction", the alternative to hysco_correct):
 * per PE column, the true image I minimising |P+ I - Ip|^2 + |P- I - Im|^2 + lambda |I|^2, where the
 * push-forward matrix P+- spreads the mass of true cell j uniformly over its mapped interval
 * [j - 1/2 +- b_j, j + 1/2 +- b_{j+1}] (cell-index coordinates, b in PE voxels) and distorted cell i
 * collects the part inside [i - 1/2, i + 1/2].  lambda > 0 (1e-6 is negligible at single precision)
 * sets cells whose mass leaves the column in both images to 0.  out: image-shaped float32.  A column
 * whose field has |d_v b| >= 1 somewhere, or whose normal matrix is wider than a band of half-width
 * 16 (compression |d_v b| above about 0.94 over many cells), is set to 0 and counted in *nbad
 * (device int32, nullable).  The first call allocates the handle's least-squares workspace (17
 * image-shaped arrays): HYSCO_ENOMEM if that fails. */
int hysco_ls_correct(hysco_t h, const void* Ip, const void* Im, const float* b, double lambda,
                     float* out, int32_t* nbad, hysco_stream_t stream);

/* Full solve (Sec. 2.2 + 2.3.1): optional OT init (opts->init), then opts->gn_iters Gauss-Newton
 * iterations b <- b + gamma q with H_J q ~= -grad J from at most pcg_max_iters PCG iterations
 * (x0 = 0, stop at relative residual < pcg_rtol) and gamma the first of 1, 1/2, 1/4, ... that
 * satisfies the Armijo condition J(b + gamma q) <= J(b) + c1 gamma grad^T q (none, or
 * grad^T q >= 0: the iterate is kept).  The iteration count is fixed; the loop stops early only
 * when J(b) is not finite (hysco_last_status then reports it).  b_inout: field-shaped float32,
 * read when opts->init == 0, always written.  stats: nullable, see HYSCO_NSTATS. */
int hysco_solve(hysco_t h, const void* Ip, const void* Im, float* b_inout,
                const hysco_opts* opts, double* stats, hysco_stream_t stream);

/* Self-test of failure detection in the persistent kernels' device-wide barrier (the one that
 * separates their phases): launches a cooperative grid of `grid` (<= 64) blocks of which block
 * `missing_block` never arrives (-1: all arrive); the others wait at most `spin_cycles` clock
 * cycles, then give up.  Returns HYSCO_ETIMEOUT when the waits ran out, HYSCO_OK when the barrier
 * completed with the correct grid-wide sum, HYSCO_ENONFINITE for a wrong sum, HYSCO_EINVAL for
 * bad arguments.  Synchronises `stream`; the CUDA context stays usable either way. */
int hysco_selftest_barrier(int grid, int missing_block, int64_t spin_cycles,
                           hysco_stream_t stream);

/* ---- ADMM (Sec. 2.3.2) -----------------------------------------------------------------------
 * The alternative optimiser of Sec. 2.3.2: the objective is split into F(b) = D + alpha S3 +
 * beta P (S3 the smoothness along PE) and G(z) = alpha (S1 + S2) (the in-plane smoothness) with
 * the constraint b = z; with the scaled multiplier u every iteration
 *   b <- argmin F(b) + rho vol/2 ||b - z + u||^2   by gn_iters Gauss-Newton steps whose
 *        directions come from BlockPCG (the Jacobi CG of Sec. 2.3.1 run on every PE column
 *        independently, with the column's own step sizes and stop) and Armijo backtracking on
 *        that subproblem's objective;
 *   z <- argmin G(z) + rho vol/2 ||b - z + u||^2   solved directly per PE plane with periodic
 *        in-plane ends (the 2D Fourier transform diagonalises it);
 *   u <- u + b - z;
 * then rho is balanced (Boyd et al. 2011, Sec. 3.4.1): r = ||b - z||, s = rho ||z - z_prev||,
 * rho <- tau rho (u <- u / tau) when r > mu s, rho <- rho / tau (u <- tau u) when s > mu r; the
 * run stops after the iteration in which the relative changes of b, z and u are all below tol.
 * (Readings where the paper is silent: the augmentation weight rho h^3 is rho times the cell
 * volume; rho starts at alpha unless rho0 > 0; the relative change of a vector that was zero is
 * infinite.) */
typedef struct {
  int32_t admm_iters;     /* maximum ADMM iterations (default 20) */
  int32_t gn_iters;       /* Gauss-Newton steps per b-update (default 2) */
  int32_t pcg_max_iters;  /* BlockPCG iterations per column and GN step, <= 64 (default 10) */
  int32_t ls_max_iters;   /* Armijo trials per GN step, <= 16 (default 10) */
  int32_t init;           /* 1 = OT initialisation with the feasible-start rule, 0 = from b_inout */
  int32_t ot_blur;        /* as in hysco_opts */
  int32_t no_graph;       /* as in hysco_opts */
  int32_t pad_;
  double pcg_rtol;        /* per-column relative residual stop (default 0.1) */
  double armijo_c1;       /* default 1e-4 */
  double ot_eps;          /* default 1e-3 */
  double rho0;            /* initial rho; <= 0: alpha (default 0) */
  double tol;             /* stop tolerance on the relative changes (default 1e-3) */
  double mu, tau;         /* rho rule (defaults 10 and 2) */
} hysco_admm_opts;

void hysco_default_admm_opts(hysco_admm_opts* opts);

#define HYSCO_ADMM_NSTATS 10   /* per iteration: J(b), the b-subproblem's objective
                                  F(b) + rho vol/2 ||b - z + u||^2 at the new b, rho, r, s,
                                  relative changes of b, z and u, BlockPCG iterations summed over
                                  columns and GN steps, the last GN step's gamma */

/* Runs ADMM on the pair (images as in hysco_solve) from b_inout (or OT) and writes the final b
 * into b_inout.  stats: NULL or an admm_iters x HYSCO_ADMM_NSTATS device array of doubles (rows
 * after the stop NaN).  The PE extent must be at most 255 cells (BlockPCG keeps a column's 256
 * nodes in one warp's registers), else HYSCO_EINVAL.  Stream-ordered; hysco_last_status reports
 * HYSCO_INFEASIBLE / HYSCO_ENONFINITE when a b-update met a non-finite objective (the run stops
 * there).  Uses the handle's workspace plus five field-sized arrays allocated at the first call. */
int hysco_admm(hysco_t h, const void* Ip, const void* Im, float* b_inout,
               const hysco_admm_opts* opts, double* stats, hysco_stream_t stream);

/* The ADMM b-update's direction solver alone (BlockPCG, Sec. 2.3.2): linearises the b-subproblem
 * F(b) + rho vol/2 ||b - c||^2 at b (its GN Hessian does not depend on c) and solves
 * H_col q = rhs on every PE column independently by Jacobi CG with the column's own step sizes
 * and stop (||r|| / ||r0|| < rtol after an update, p^T H p <= 0, or max_iters <= 1000).  b, rhs,
 * q: field-shaped float32 (device); iters: NULL or one device int32 receiving the iterations
 * summed over columns.  PE extent at most 255 cells, rho >= 0, else HYSCO_EINVAL. */
int hysco_block_pcg(hysco_t h, const void* Ip, const void* Im, const float* b, double rho,
                    const float* rhs, float* q, int max_iters, double rtol, int32_t* iters,
                    hysco_stream_t stream);

/* The ADMM z-update alone (Sec. 2.3.2): z = argmin alpha (S1 + S2)(z) + rho vol/2 ||v - z||^2
 * with periodic in-plane ends, i.e. z = rho (alpha H_G + rho I)^{-1} v, per PE plane through the
 * real Fourier bases of the in-plane axes.  v, z: field-shaped float32 (device); rho > 0. */
int hysco_admm_zsolve(hysco_t h, const float* v, double rho, float* z, hysco_stream_t stream);

/* The z-update's arithmetic path (Sec. 2.3.2), for testing and tuning: 0 = its four per-plane
 * basis products on the tensor cores (tcgen05 kind::tf32 with each operand split into a TF32 pair
 * hi + lo and three products per pair, FP32 accumulation: single-precision accuracy), the default
 * wherever both in-plane axes have at most 256 nodes; 1 = the same products in FP32 on the CUDA
 * cores.  hysco_set_zsolve_path returns HYSCO_EINVAL for an unknown path or for path 0 where it
 * does not apply, and drops the cached ADMM graph when the path changes; hysco_zsolve_path returns
 * the path in use (or a negative status).  Both allocate the ADMM workspace if needed. */
int hysco_set_zsolve_path(hysco_t h, int path);
int hysco_zsolve_path(hysco_t h);

/* Self-test of failure detection in the tensor-core z-update (path 0): one launch of its first
 * product whose copies are never issued, so that the stage barriers never fill and every wait on
 * them gives up after `spin_cycles` (1 .. 4e9) clock cycles.  Returns HYSCO_ETIMEOUT when the
 * launch recorded the timeout (nothing left in flight, its tensor memory freed), HYSCO_OK if it
 * did not, HYSCO_EINVAL for bad arguments or where path 0 does not apply.  Synchronises `stream`
 * and clears the handle's device state afterwards; the handle and the context stay usable. */
int hysco_selftest_zsolve(hysco_t h, int64_t spin_cycles, hysco_stream_t stream);

/* ---- batched solve (many volume pairs of uneven sizes) -------------------------------------
 * A batch groups n distinct handles (same device; any dims, spacings, PE axes and image dtypes)
 * whose solves advance through the Gauss-Newton loop together (Sec. 2.3.1 per pair, unchanged):
 * per GN iteration the per-pair evaluation, Armijo and update kernels of different pairs run on
 * concurrent branches, and the Jacobi PCG of all pairs is either one cooperative launch whose grid
 * is shared among the pairs (the device-wide barriers are paid once for the batch), each pair's
 * own persistent PCG in turn (its vectors on chip, see hysco_pcg_plan), or waves: the pairs are
 * packed, largest first, into waves whose PCG vectors fit the device together (on chip, or with up
 * to 1.25 or 1.5 times as many vector slots per thread as shared memory holds, the excess in
 * global memory); a wave's pairs go through their whole GN loop together and their PCGs share one
 * cooperative launch per GN step, each pair on its own block range with barriers among those
 * blocks only.  The fixed launch
 * sequence is captured in a CUDA graph (cached per argument set) unless opts->no_graph.  The batch
 * holds no reference count: destroy it before any of its handles. */
typedef struct hysco_batch_ctx* hysco_batch_t;

/* n >= 1 distinct handles, at most one per block of the batched PCG grid (296 or more on a B300);
 * HYSCO_EINVAL otherwise. */
int hysco_batch_create(int n, const hysco_t* handles, hysco_batch_t* out);
void hysco_batch_destroy(hysco_batch_t batch);

/* Solve every pair i: images Ip[i], Im[i] (its handle's dtype and dims), field b[i] in/out, stats
 * optional (NULL, or n pointers each NULL or a gn_iters x HYSCO_NSTATS device array as in
 * hysco_solve).  Same options for all pairs; precond must be HYSCO_PC_JACOBI (pcg_path is ignored).
 * Each pair's numerical status: hysco_last_status on its handle. */
int hysco_batch_solve(hysco_batch_t batch, const void* const* Ip, const void* const* Im,
                      float* const* b, const hysco_opts* opts, double* const* stats,
                      hysco_stream_t stream);

/* Autotuner: times short trial solves (OT + at most 2 GN iterations into scratch fields, the
 * caller's fields untouched) of each candidate schedule -- 1, 2, 4 or 8 concurrent branches for
 * the per-pair kernels; the shared PCG launch with blocks by field size and at least 1 or at least
 * 2 blocks per pair, the per-pair persistent PCG, waves of PCG launches, or waves of whole GN
 * loops, each wave packing at 1, 1.25 or 1.5 -- and keeps the fastest.  Synchronises
 * `stream`. */
int hysco_batch_tune(hysco_batch_t batch, const void* const* Ip, const void* const* Im,
                     const hysco_opts* opts, hysco_stream_t stream);

/* The schedule in use: out[0] branches, out[1] PCG policy (0: shared launch, blocks by field size;
 * 1: the same with >= 2 blocks per pair; 2: each pair's persistent PCG in turn; 3, 4, 5: waves
 * packed to 1, 1.25 and 1.5 times the on-chip vector capacity, one PCG launch per wave and GN
 * step; 6, 7, 8: the same waves, each wave's whole GN loops in one persistent launch as in
 * pcg_path 4, waves of one image type), out[2] blocks of the shared PCG launch's grid. */
int hysco_batch_schedule(hysco_batch_t batch, int32_t out[3]);

/* Sets the schedule: branches 1 .. min(8, n), PCG policy 0 .. 8 as in hysco_batch_schedule.
 * HYSCO_EINVAL when out of range or infeasible for this batch (then unchanged).  Drops the cached
 * graph. */
int hysco_batch_set_schedule(hysco_batch_t batch, int branches, int policy);

/* The persistent PCG's launch plan (pcg_path 0 / 2): out[0] cooperative grid (0 when the device
 * cannot run it), out[1] slots per thread whose r, p and H p stay in shared memory for the whole
 * launch, out[2] slots per thread in all (float4 groups of the pitched field over grid * out[3]
 * threads), out[3] threads per block.  Slots past out[1] keep those vectors in global memory;
 * the arithmetic, and so the result, is the same either way. */
int hysco_pcg_plan(hysco_t h, int32_t out[4]);

/* Limits the on-chip slots of the persistent PCG to `onchip` (0 .. the plan's maximum; -1
 * restores the maximum), for testing and tuning.  HYSCO_EINVAL outside that range.  Drops the
 * cached solve graph. */
int hysco_set_pcg_onchip(hysco_t h, int onchip);

/* Synchronises `stream` and returns the numerical status of the last hysco_eval / hysco_solve /
 * hysco_init_ot on this handle: HYSCO_OK, HYSCO_INFEASIBLE, HYSCO_ENONFINITE or HYSCO_ETIMEOUT
 * (or HYSCO_ECUDA when the stream reports an error). */
int hysco_last_status(hysco_t h, hysco_stream_t stream);

/* Diagnostics: the same kernels with extra outputs.
 * hysco_cell_indices: interpolation cell indices floor(t+-) of every cell at b (image-shaped
 * int32; positions outside [-2, m + 1] are reported clamped to that range).
 * hysco_ot_indices: the merge indices k* = min{k : C(k+1) >= r} of the two inverse-CDF
 * lookups C-^{-1}(C+(k)) and C+^{-1}(C-(k)) of hysco_init_ot (field-shaped int32). */
int hysco_cell_indices(hysco_t h, const float* b, int32_t* cell_p, int32_t* cell_m,
                       hysco_stream_t stream);
int hysco_ot_indices(hysco_t h, const void* Ip, const void* Im, double eps, int32_t* kidx_p,
                     int32_t* kidx_m, hysco_stream_t stream);

/* Allocation-free objective: J, D, S, P (terms_dev, 4 device doubles) and, when grad is
 * non-NULL, the gradient, for callers that cannot allocate device memory -- for example code
 * running under a memory manager that owns the whole device budget, or latency-critical callers
 * for which cudaMalloc's implicit synchronisation is unacceptable.  The paper has no counterpart:
 * this is a library convenience around the same per-cell arithmetic as hysco_eval.
 * Takes the geometry of hysco_create by value and needs no handle.  Its only scratch (the
 * per-block partial sums of the reduction and a ticket counter, 384 KiB plus 256 bytes) lives in a
 * static device array that every GPU loading this library holds until the process exits; the
 * call allocates nothing.  The first call in each CUDA context (on each device, with that device
 * current, and again after cudaDeviceReset re-creates the context) looks up the array's device
 * address, so make that first call before any stream capture.  All calls share the
 * array: calls whose work overlaps on the GPU (two streams, or two host threads) race and give
 * wrong results; calls ordered on one stream are safe.  Volumes whose reduction grid exceeds
 * 32768 blocks (ceil(columns / 256) * ceil((m + 1) / 4)) return HYSCO_EINVAL.  No status word is
 * kept: J = +inf means barrier-infeasible, NaN means non-finite input.  No Gauss-Newton
 * coefficients are stored (use the handle-based hysco_eval for hysco_hessvec / hysco_precond). */
int hysco_eval_static(const int64_t dims[3], const double spacing[3], int pe_dim, double alpha,
                      double beta, int img_dtype, const void* Ip, const void* Im, const float* b,
                      double* terms_dev, float* grad, hysco_stream_t stream);

#ifdef __cplusplus
}
#endif
#endif /* HYSCO_H */
