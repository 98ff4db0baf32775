/*
 * hysco_oracle.c -- plain double-precision CPU oracle for the HySCO field-map hot path
 * (Julian & Ruthotto, "PyHySCO: GPU-Enabled Susceptibility Artifact Distortion Correction in
 * Seconds", arXiv 2403.10706).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the package smoke check and the benchmark's
 * CPU-baseline leg may load this library.  It shares no code, header, table or constant with
 * the CUDA library and never calls it.  Every loop below is one formula of the paper, written
 * for a reader who checks it against the paper by eye: no blocking, no fusion, no reordering.
 * Loops over columns, nodes and cells run on OpenMP threads where each iteration writes its own
 * elements; every sum has a fixed order (a sum over cells is a sum of per-column sums taken in
 * column order, an inner product a sum of fixed 4096-term chunks taken in chunk order), so the
 * number of threads never changes a result.
 *
 * Notation (Sec. 2.1: Eq. 1 transform model, Eq. 2 distance, Eq. 3 barrier, Eq. 5 smoothness,
 * and the discretisation paragraph between them):
 *   - the image has dims d[0..2] (C order, last index fastest), spacing h[0..2] in mm, and the
 *     phase-encoding (PE) axis p.  m = d[p] cells along PE.  vol = h0*h1*h2 is the midpoint
 *     quadrature weight of one cell.
 *   - the field b lives on the e_p-staggered grid: m+1 nodes along p, cell centred along the two
 *     other axes.  b is stored in PE-voxel units (b_mm = h[p]*b); the objective is the paper's
 *     physical J.
 *   - per column cell j (nodes j, j+1):  bc_j = (b_j + b_{j+1})/2,  delta_j = b_{j+1} - b_j,
 *     t+_j = j + bc_j,  t-_j = j - bc_j  (cell centre j sits at index j).
 *   - 1D piecewise-linear image model along PE (Sec. 2.4 "Interp1D"): I(t) = (1-w) I[i] + w I[i+1],
 *     i = floor(t), w = t - i, I[k] = 0 outside 0..m-1; its slope is I[i+1] - I[i].
 *   - T+_j = I+(t+_j)(1 + delta_j), T-_j = I-(t-_j)(1 - delta_j), r_j = T+_j - T-_j  (Eq. 1).
 *   - D = vol/2 sum r_j^2 (Eq. 2), S = vol/2 h_p^2 b^T L b (Eq. 5, L = 7-point negative
 *     Laplacian with homogeneous Neumann ends, sum_d G_d^T G_d / h_d^2), P = vol/2 sum phi(delta_j)
 *     with phi(z) = z^4/(1-z^2) on (-1,1) and +inf elsewhere (Eq. 3); J = D + alpha S + beta P.
 *   - gradient  = vol [Jr^T r + alpha h_p^2 L b + beta/2 D^T phi'(delta)],
 *     GN Hessian = vol [Jr^T Jr + alpha h_p^2 L + beta/2 D^T diag(phi''(delta)) D]  (Sec. 2.3.1),
 *     where row j of the residual Jacobian Jr holds (a_j/2 - c_j) at node j and (a_j/2 + c_j) at
 *     node j+1, a_j = I+'(t+)(1+delta) + I-'(t-)(1-delta), c_j = I+(t+) + I-(t-).
 *
 * Two evaluation modes:
 *   contract = 1  positions t+-, the cell index i and the weight w are formed from the single-
 *                 precision field exactly as a single-precision implementation forms them
 *                 (bc = (b_j + b_{j+1}) * 0.5f; t = (float)j +- bc), so that cell indices can be
 *                 compared bit for bit; the OT cumulative sums are formed in single precision left
 *                 to right for the same reason.  Everything after those decisions is double.
 *   contract = 0  everything in double.
 *
 * Parity pins: see tests/test_oracle_*.py.  Nothing here is "parity unpinned".
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef struct {
  int64_t d[3];    /* image dims, C order */
  double h[3];     /* spacing in mm */
  int32_t p;       /* phase-encoding axis, 0..2 */
  int32_t pad_;
  double alpha;    /* smoothness weight (Eq. 4) */
  double beta;     /* barrier weight (Eq. 4) */
} orc_geom;

typedef struct {
  int32_t gn_iters;       /* fixed number of Gauss-Newton iterations (Sec. 2.3.1) */
  int32_t pcg_max_iters;  /* PCG iteration cap, 10 in the paper */
  int32_t ls_max_iters;   /* Armijo trials, step halved after each rejection */
  int32_t precond;        /* 0 = Jacobi (Sec. 2.3.1), 1 = exact per-column block (Sec. 2.3.1 end) */
  int32_t init;           /* 1 = OT initialisation (Sec. 2.2), 0 = start from b_inout */
  int32_t ot_blur;        /* 1 = 3x3x3 Gaussian blur (sigma 1 voxel) after OT (Sec. 2.4) */
  int32_t contract;       /* evaluation mode, see header */
  int32_t pad_;
  double pcg_rtol;        /* relative residual stop, 0.1 in the paper */
  double armijo_c1;       /* Armijo sufficient-decrease constant */
  double ot_eps;          /* positivity shift factor for OT */
} orc_opts;

/* per-iteration record written by orc_solve */
enum { ST_J, ST_D, ST_S, ST_P, ST_GNORM, ST_GQ, ST_GAMMA, ST_PCG_IT, ST_PCG_RELRES, ST_LS_TRIALS,
       ST_NFIELDS };

/* ------------------------------------------------------------------------------------------ */
/* geometry helpers                                                                            */
/* ------------------------------------------------------------------------------------------ */

/* Threads of the OpenMP loops (columns, nodes, fixed chunks): results do not depend on it. */
void orc_set_threads(int n) {
#ifdef _OPENMP
  if (n > 0) omp_set_num_threads(n);
#else
  (void)n;
#endif
}
int orc_max_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

static int64_t img_count(const orc_geom* g) { return g->d[0] * g->d[1] * g->d[2]; }
static int64_t fld_dim(const orc_geom* g, int ax) { return ax == g->p ? g->d[ax] + 1 : g->d[ax]; }
static int64_t fld_count(const orc_geom* g) {
  return fld_dim(g, 0) * fld_dim(g, 1) * fld_dim(g, 2);
}
static double cell_volume(const orc_geom* g) { return g->h[0] * g->h[1] * g->h[2]; }

/* C-order strides of the image and of the field */
static void img_strides(const orc_geom* g, int64_t s[3]) {
  s[2] = 1; s[1] = g->d[2]; s[0] = g->d[1] * g->d[2];
}
static void fld_strides(const orc_geom* g, int64_t s[3]) {
  s[2] = 1; s[1] = fld_dim(g, 2); s[0] = fld_dim(g, 1) * fld_dim(g, 2);
}

/* the two non-PE axes, in axis order */
static void inplane_axes(const orc_geom* g, int* q0, int* q1) {
  int k = 0, q[2];
  for (int ax = 0; ax < 3; ++ax) if (ax != g->p) q[k++] = ax;
  *q0 = q[0]; *q1 = q[1];
}
static int64_t column_count(const orc_geom* g) {
  int q0, q1; inplane_axes(g, &q0, &q1);
  return g->d[q0] * g->d[q1];
}
/* offsets of column `col` in the image and in the field, and its coordinates */
static void column_offsets(const orc_geom* g, int64_t col, int64_t* off_img, int64_t* off_fld,
                           int64_t* c0, int64_t* c1) {
  int q0, q1; inplane_axes(g, &q0, &q1);
  int64_t si[3], sf[3]; img_strides(g, si); fld_strides(g, sf);
  *c0 = col / g->d[q1];
  *c1 = col % g->d[q1];
  *off_img = *c0 * si[q0] + *c1 * si[q1];
  *off_fld = *c0 * sf[q0] + *c1 * sf[q1];
}

/* ------------------------------------------------------------------------------------------ */
/* the barrier function phi of Eq. 3 and its first two derivatives                             */
/* ------------------------------------------------------------------------------------------ */

void orc_phi(double z, double* f, double* df, double* d2f) {
  if (!(fabs(z) < 1.0)) {  /* outside (-1, 1): phi = +inf; derivatives unused there */
    *f = INFINITY; *df = 0.0; *d2f = 0.0;
    return;
  }
  double q = 1.0 - z * z;
  *f = z * z * z * z / q;
  *df = (4.0 * z * z * z - 2.0 * z * z * z * z * z) / (q * q);
  *d2f = (12.0 * z * z - 6.0 * z * z * z * z + 2.0 * z * z * z * z * z * z) / (q * q * q);
}

/* ------------------------------------------------------------------------------------------ */
/* cell geometry and the 1D linear image model                                                 */
/* ------------------------------------------------------------------------------------------ */

/* positions of cell j of a column given its two field nodes (averaging and finite difference
 * operators of the discretisation paragraph of Sec. 2.1) */
static void cell_positions(double bj, double bj1, int64_t j, int contract,
                           double* tp, double* tm, double* delta) {
  *delta = bj1 - bj;
  if (contract) {
    float bjf = (float)bj, bj1f = (float)bj1;
    float sum = bjf + bj1f;
    float bc = sum * 0.5f;
    float jf = (float)j;
    float tpf = jf + bc;
    float tmf = jf - bc;
    *tp = (double)tpf;
    *tm = (double)tmf;
  } else {
    double bc = 0.5 * (bj + bj1);
    *tp = (double)j + bc;
    *tm = (double)j - bc;
  }
}

/* linear interpolation of one image column (m values, stride st) at index coordinate t */
static void interp1(const float* col, int64_t st, int64_t m, double t,
                    double* val, double* slope, int64_t* cell) {
  double fi = floor(t);
  int64_t i = (int64_t)fi;
  double w = t - fi;
  double I0 = (i >= 0 && i < m) ? (double)col[i * st] : 0.0;
  double I1 = (i + 1 >= 0 && i + 1 < m) ? (double)col[(i + 1) * st] : 0.0;
  *val = (1.0 - w) * I0 + w * I1;
  *slope = I1 - I0;
  *cell = i;
}

/* ------------------------------------------------------------------------------------------ */
/* negative Laplacian L = sum_d G_d^T G_d / h_d^2 on the field grid (Eq. 5), Neumann ends      */
/* ------------------------------------------------------------------------------------------ */

void orc_laplacian(const orc_geom* g, const double* x, double* y) {
  int64_t n[3] = {fld_dim(g, 0), fld_dim(g, 1), fld_dim(g, 2)};
  int64_t s[3]; fld_strides(g, s);
#pragma omp parallel for schedule(static)
  for (int64_t i0 = 0; i0 < n[0]; ++i0)
    for (int64_t i1 = 0; i1 < n[1]; ++i1)
      for (int64_t i2 = 0; i2 < n[2]; ++i2) {
        int64_t idx[3] = {i0, i1, i2};
        int64_t k = i0 * s[0] + i1 * s[1] + i2 * s[2];
        double acc = 0.0;
        for (int ax = 0; ax < 3; ++ax) {
          double w = 1.0 / (g->h[ax] * g->h[ax]);
          if (idx[ax] > 0) acc += w * (x[k] - x[k - s[ax]]);
          if (idx[ax] < n[ax] - 1) acc += w * (x[k] - x[k + s[ax]]);
        }
        y[k] = acc;
      }
}

/* diagonal of L */
static void laplacian_diag(const orc_geom* g, double* y) {
  int64_t n[3] = {fld_dim(g, 0), fld_dim(g, 1), fld_dim(g, 2)};
  int64_t s[3]; fld_strides(g, s);
#pragma omp parallel for schedule(static)
  for (int64_t i0 = 0; i0 < n[0]; ++i0)
    for (int64_t i1 = 0; i1 < n[1]; ++i1)
      for (int64_t i2 = 0; i2 < n[2]; ++i2) {
        int64_t idx[3] = {i0, i1, i2};
        double acc = 0.0;
        for (int ax = 0; ax < 3; ++ax) {
          double w = 1.0 / (g->h[ax] * g->h[ax]);
          acc += w * (double)((idx[ax] > 0) + (idx[ax] < n[ax] - 1));
        }
        y[i0 * s[0] + i1 * s[1] + i2 * s[2]] = acc;
      }
}

/* Inner product as sums of fixed chunks of ORC_CHUNK terms, added in chunk order: the order of
 * every addition is fixed, whatever the number of threads. */
#define ORC_CHUNK 4096
static double dot(const double* a, const double* b, int64_t n) {
  int64_t nch = (n + ORC_CHUNK - 1) / ORC_CHUNK;
  double* part = malloc((nch > 0 ? nch : 1) * sizeof(double));
#pragma omp parallel for schedule(static)
  for (int64_t c = 0; c < nch; ++c) {
    double s = 0.0;
    int64_t end = (c + 1) * ORC_CHUNK < n ? (c + 1) * ORC_CHUNK : n;
    for (int64_t i = c * ORC_CHUNK; i < end; ++i) s += a[i] * b[i];
    part[c] = s;
  }
  double s = 0.0;
  for (int64_t c = 0; c < nch; ++c) s += part[c];
  free(part);
  return s;
}

/* ------------------------------------------------------------------------------------------ */
/* linearisation of the residual about b: r, the two nonzeros of each Jacobian row, phi', phi'' */
/* ------------------------------------------------------------------------------------------ */

typedef struct {
  double* r;      /* residual per cell (image shaped) */
  double* jl;     /* d r_j / d b_j      = a_j/2 - c_j */
  double* jr;     /* d r_j / d b_{j+1}  = a_j/2 + c_j */
  double* dphi;   /* phi'(delta_j) */
  double* d2phi;  /* phi''(delta_j) */
} orc_lin;

/* Computes D, P (and the linearisation / corrected images / cell indices when asked) for all
 * cells.  Returns the number of cells with |delta| >= 1 (barrier infeasible). */
static int64_t residual_pass(const orc_geom* g, const float* Ip, const float* Im, const double* b,
                             int contract, double* Dsum, double* Psum, orc_lin* lin,
                             double* Tp, double* Tm, int32_t* cell_p, int32_t* cell_m) {
  int64_t m = g->d[g->p];
  int64_t si[3], sf[3]; img_strides(g, si); fld_strides(g, sf);
  int64_t sti = si[g->p], stf = sf[g->p];
  int64_t ncols = column_count(g);
  int64_t bad = 0;
  /* per-column sums, added in column order below */
  double* dcol = malloc(ncols * sizeof(double));
  double* pcol = malloc(ncols * sizeof(double));
#pragma omp parallel for schedule(static) reduction(+ : bad)
  for (int64_t col = 0; col < ncols; ++col) {
    int64_t oi, of, c0, c1;
    column_offsets(g, col, &oi, &of, &c0, &c1);
    double dsum = 0.0, psum = 0.0;
    for (int64_t j = 0; j < m; ++j) {
      double bj = b[of + j * stf], bj1 = b[of + (j + 1) * stf];
      double tp, tm, delta;
      cell_positions(bj, bj1, j, contract, &tp, &tm, &delta);
      double Ipv, Ips, Imv, Ims;
      int64_t ip, im;
      interp1(Ip + oi, sti, m, tp, &Ipv, &Ips, &ip);
      interp1(Im + oi, sti, m, tm, &Imv, &Ims, &im);
      double tplus = Ipv * (1.0 + delta);    /* Eq. 1 with +v */
      double tminus = Imv * (1.0 - delta);   /* Eq. 1 with -v */
      double r = tplus - tminus;
      double f, df, d2f;
      orc_phi(delta, &f, &df, &d2f);
      if (!(fabs(delta) < 1.0)) ++bad;
      dsum += r * r;
      psum += f;
      int64_t cidx = oi + j * sti;
      if (lin) {
        double a = Ips * (1.0 + delta) + Ims * (1.0 - delta);
        double c = Ipv + Imv;
        lin->r[cidx] = r;
        lin->jl[cidx] = 0.5 * a - c;
        lin->jr[cidx] = 0.5 * a + c;
        lin->dphi[cidx] = df;
        lin->d2phi[cidx] = d2f;
      }
      if (Tp) Tp[cidx] = tplus;
      if (Tm) Tm[cidx] = tminus;
      if (cell_p) cell_p[cidx] = (int32_t)ip;
      if (cell_m) cell_m[cidx] = (int32_t)im;
    }
    dcol[col] = dsum;
    pcol[col] = psum;
  }
  double dsum = 0.0, psum = 0.0;
  for (int64_t col = 0; col < ncols; ++col) {
    dsum += dcol[col];
    psum += pcol[col];
  }
  free(dcol); free(pcol);
  double vol = cell_volume(g);
  *Dsum = 0.5 * vol * dsum;
  *Psum = 0.5 * vol * psum;
  return bad;
}

static double smoothness(const orc_geom* g, const double* b, double* Lb_scratch) {
  orc_laplacian(g, b, Lb_scratch);
  double hp = g->h[g->p];
  return 0.5 * cell_volume(g) * hp * hp * dot(b, Lb_scratch, fld_count(g));
}

/* J^T applied to a cell-shaped vector s, accumulated into node-shaped y (y += Jr^T s) */
static void jr_transpose_add(const orc_geom* g, const orc_lin* lin, const double* s, double* y) {
  int64_t m = g->d[g->p];
  int64_t si[3], sf[3]; img_strides(g, si); fld_strides(g, sf);
  int64_t ncols = column_count(g);
#pragma omp parallel for schedule(static)
  for (int64_t col = 0; col < ncols; ++col) {
    int64_t oi, of, c0, c1;
    column_offsets(g, col, &oi, &of, &c0, &c1);
    for (int64_t j = 0; j < m; ++j) {
      int64_t c = oi + j * si[g->p];
      y[of + j * sf[g->p]] += lin->jl[c] * s[c];
      y[of + (j + 1) * sf[g->p]] += lin->jr[c] * s[c];
    }
  }
}

/* cell-shaped u = Jr v */
static void jr_apply(const orc_geom* g, const orc_lin* lin, const double* v, double* u) {
  int64_t m = g->d[g->p];
  int64_t si[3], sf[3]; img_strides(g, si); fld_strides(g, sf);
  int64_t ncols = column_count(g);
#pragma omp parallel for schedule(static)
  for (int64_t col = 0; col < ncols; ++col) {
    int64_t oi, of, c0, c1;
    column_offsets(g, col, &oi, &of, &c0, &c1);
    for (int64_t j = 0; j < m; ++j) {
      int64_t c = oi + j * si[g->p];
      u[c] = lin->jl[c] * v[of + j * sf[g->p]] + lin->jr[c] * v[of + (j + 1) * sf[g->p]];
    }
  }
}

/* cell-shaped u = D v (forward difference along PE) */
static void fd_apply(const orc_geom* g, const double* v, double* u) {
  int64_t m = g->d[g->p];
  int64_t si[3], sf[3]; img_strides(g, si); fld_strides(g, sf);
  int64_t ncols = column_count(g);
#pragma omp parallel for schedule(static)
  for (int64_t col = 0; col < ncols; ++col) {
    int64_t oi, of, c0, c1;
    column_offsets(g, col, &oi, &of, &c0, &c1);
    for (int64_t j = 0; j < m; ++j)
      u[oi + j * si[g->p]] = v[of + (j + 1) * sf[g->p]] - v[of + j * sf[g->p]];
  }
}

/* node-shaped y += D^T s */
static void fd_transpose_add(const orc_geom* g, const double* s, double* y) {
  int64_t m = g->d[g->p];
  int64_t si[3], sf[3]; img_strides(g, si); fld_strides(g, sf);
  int64_t ncols = column_count(g);
#pragma omp parallel for schedule(static)
  for (int64_t col = 0; col < ncols; ++col) {
    int64_t oi, of, c0, c1;
    column_offsets(g, col, &oi, &of, &c0, &c1);
    for (int64_t j = 0; j < m; ++j) {
      double sj = s[oi + j * si[g->p]];
      y[of + (j + 1) * sf[g->p]] += sj;
      y[of + j * sf[g->p]] -= sj;
    }
  }
}

static int lin_alloc(orc_lin* lin, int64_t n) {
  lin->r = calloc(n, sizeof(double));
  lin->jl = calloc(n, sizeof(double));
  lin->jr = calloc(n, sizeof(double));
  lin->dphi = calloc(n, sizeof(double));
  lin->d2phi = calloc(n, sizeof(double));
  return lin->r && lin->jl && lin->jr && lin->dphi && lin->d2phi;
}
static void lin_free(orc_lin* lin) {
  free(lin->r); free(lin->jl); free(lin->jr); free(lin->dphi); free(lin->d2phi);
}

/* gradient of J from a linearisation (Sec. 2.3.1):  vol [Jr^T r + alpha h^2 L b + beta/2 D^T phi'] */
static void gradient_from_lin(const orc_geom* g, const orc_lin* lin, const double* b, double* grad) {
  int64_t nf = fld_count(g);
  double vol = cell_volume(g), hp = g->h[g->p];
  double* Lb = malloc(nf * sizeof(double));
  double* t = calloc(nf, sizeof(double));
  double* u = calloc(nf, sizeof(double));
  orc_laplacian(g, b, Lb);
  jr_transpose_add(g, lin, lin->r, t);
  fd_transpose_add(g, lin->dphi, u);
#pragma omp parallel for schedule(static)
  for (int64_t k = 0; k < nf; ++k)
    grad[k] = vol * (t[k] + g->alpha * hp * hp * Lb[k] + 0.5 * g->beta * u[k]);
  free(Lb); free(t); free(u);
}

/* GN Hessian-vector product from a linearisation:
 *   vol [Jr^T (Jr v) + alpha h^2 L v + beta/2 D^T (phi'' . (D v))] */
static void hessvec_from_lin(const orc_geom* g, const orc_lin* lin, const double* v, double* Hv) {
  int64_t nf = fld_count(g), nc = img_count(g);
  double vol = cell_volume(g), hp = g->h[g->p];
  double* Jv = malloc(nc * sizeof(double));
  double* Dv = malloc(nc * sizeof(double));
  double* Lv = malloc(nf * sizeof(double));
  double* t = calloc(nf, sizeof(double));
  double* u = calloc(nf, sizeof(double));
  jr_apply(g, lin, v, Jv);
  jr_transpose_add(g, lin, Jv, t);
  fd_apply(g, v, Dv);
#pragma omp parallel for schedule(static)
  for (int64_t c = 0; c < nc; ++c) Dv[c] *= lin->d2phi[c];
  fd_transpose_add(g, Dv, u);
  orc_laplacian(g, v, Lv);
#pragma omp parallel for schedule(static)
  for (int64_t k = 0; k < nf; ++k)
    Hv[k] = vol * (t[k] + g->alpha * hp * hp * Lv[k] + 0.5 * g->beta * u[k]);
  free(Jv); free(Dv); free(Lv); free(t); free(u);
}

/* diagonal of the GN Hessian (Jacobi preconditioner of Sec. 2.3.1) */
static void hessdiag_from_lin(const orc_geom* g, const orc_lin* lin, double* diag) {
  int64_t nf = fld_count(g), m = g->d[g->p];
  double vol = cell_volume(g), hp = g->h[g->p];
  int64_t si[3], sf[3]; img_strides(g, si); fld_strides(g, sf);
  double* jj = calloc(nf, sizeof(double));   /* sum_j Jr_{jk}^2 */
  double* pp = calloc(nf, sizeof(double));   /* sum_j D_{jk}^2 phi''_j */
  double* Ld = malloc(nf * sizeof(double));
  int64_t ncols = column_count(g);
#pragma omp parallel for schedule(static)
  for (int64_t col = 0; col < ncols; ++col) {
    int64_t oi, of, c0, c1;
    column_offsets(g, col, &oi, &of, &c0, &c1);
    for (int64_t j = 0; j < m; ++j) {
      int64_t c = oi + j * si[g->p];
      int64_t kl = of + j * sf[g->p], kr = of + (j + 1) * sf[g->p];
      jj[kl] += lin->jl[c] * lin->jl[c];
      jj[kr] += lin->jr[c] * lin->jr[c];
      pp[kl] += lin->d2phi[c];
      pp[kr] += lin->d2phi[c];
    }
  }
  laplacian_diag(g, Ld);
#pragma omp parallel for schedule(static)
  for (int64_t k = 0; k < nf; ++k)
    diag[k] = vol * (jj[k] + g->alpha * hp * hp * Ld[k] + 0.5 * g->beta * pp[k]);
  free(jj); free(pp); free(Ld);
}

/* The diagonal block of the GN Hessian belonging to one PE column: a tridiagonal matrix of order
 * m+1 (block-diagonal preconditioner, end of Sec. 2.3.1).  Neighbours in the other two axes only
 * contribute to its diagonal through L. */
static void column_block(const orc_geom* g, const orc_lin* lin, int64_t col,
                         double* dia, double* off) {
  int64_t m = g->d[g->p];
  int64_t si[3]; img_strides(g, si);
  double vol = cell_volume(g), hp = g->h[g->p];
  int q0, q1; inplane_axes(g, &q0, &q1);
  int64_t oi, of, c0, c1;
  column_offsets(g, col, &oi, &of, &c0, &c1);
  double inpl = (double)((c0 > 0) + (c0 < g->d[q0] - 1)) / (g->h[q0] * g->h[q0]) +
                (double)((c1 > 0) + (c1 < g->d[q1] - 1)) / (g->h[q1] * g->h[q1]);
  for (int64_t k = 0; k <= m; ++k) {
    double npe = (double)((k > 0) + (k < m)) / (hp * hp);
    dia[k] = g->alpha * hp * hp * (npe + inpl);
  }
  for (int64_t k = 0; k < m; ++k) off[k] = -g->alpha * hp * hp / (hp * hp);
  for (int64_t j = 0; j < m; ++j) {
    int64_t c = oi + j * si[g->p];
    double jl = lin->jl[c], jr = lin->jr[c], q = 0.5 * g->beta * lin->d2phi[c];
    dia[j] += jl * jl + q;
    dia[j + 1] += jr * jr + q;
    off[j] += jl * jr - q;
  }
  for (int64_t k = 0; k <= m; ++k) dia[k] *= vol;
  for (int64_t k = 0; k < m; ++k) off[k] *= vol;
}

/* Thomas algorithm for a symmetric tridiagonal system of order n (textbook LDL^T, no pivoting) */
static void thomas_solve(int64_t n, const double* dia, const double* off, const double* rhs,
                         double* x, double* work_c, double* work_d) {
  work_c[0] = n > 1 ? off[0] / dia[0] : 0.0;
  work_d[0] = rhs[0] / dia[0];
  for (int64_t i = 1; i < n; ++i) {
    double den = dia[i] - off[i - 1] * work_c[i - 1];
    work_c[i] = i < n - 1 ? off[i] / den : 0.0;
    work_d[i] = (rhs[i] - off[i - 1] * work_d[i - 1]) / den;
  }
  x[n - 1] = work_d[n - 1];
  for (int64_t i = n - 2; i >= 0; --i) x[i] = work_d[i] - work_c[i] * x[i + 1];
}

/* z = M^{-1} r for the per-column block preconditioner */
static void column_precond_from_lin(const orc_geom* g, const orc_lin* lin, const double* r,
                                    double* z) {
  int64_t m = g->d[g->p];
  int64_t sf[3]; fld_strides(g, sf);
  int64_t ncols = column_count(g);
  double *dia = malloc((m + 1) * sizeof(double)), *off = malloc((m + 1) * sizeof(double));
  double *rc = malloc((m + 1) * sizeof(double)), *zc = malloc((m + 1) * sizeof(double));
  double *w1 = malloc((m + 1) * sizeof(double)), *w2 = malloc((m + 1) * sizeof(double));
  for (int64_t col = 0; col < ncols; ++col) {
    int64_t oi, of, c0, c1;
    column_offsets(g, col, &oi, &of, &c0, &c1);
    column_block(g, lin, col, dia, off);
    for (int64_t k = 0; k <= m; ++k) rc[k] = r[of + k * sf[g->p]];
    thomas_solve(m + 1, dia, off, rc, zc, w1, w2);
    for (int64_t k = 0; k <= m; ++k) z[of + k * sf[g->p]] = zc[k];
  }
  free(dia); free(off); free(rc); free(zc); free(w1); free(w2);
}

/* z = M^{-1} r for the Jacobi preconditioner; a zero diagonal entry acts as 1 */
static void jacobi_precond(int64_t n, const double* diag, const double* r, double* z) {
  for (int64_t k = 0; k < n; ++k) z[k] = diag[k] > 0.0 ? r[k] / diag[k] : r[k];
}

/* ------------------------------------------------------------------------------------------ */
/* public entry points: objective, gradient, Hessian-vector product, preconditioners           */
/* ------------------------------------------------------------------------------------------ */

/* J, D, S, P at b (terms[0..3]); gradient, corrected images T+/T- and cell indices on request.
 * Returns the number of barrier-infeasible cells (J = +inf when nonzero). */
int64_t orc_eval(const orc_geom* g, const float* Ip, const float* Im, const double* b,
                 int contract, double* terms, double* grad, double* Tp, double* Tm,
                 int32_t* cell_p, int32_t* cell_m) {
  int64_t nc = img_count(g), nf = fld_count(g);
  orc_lin lin;
  int want_lin = grad != NULL;
  if (want_lin && !lin_alloc(&lin, nc)) return -1;
  double D, P;
  int64_t bad = residual_pass(g, Ip, Im, b, contract, &D, &P, want_lin ? &lin : NULL,
                              Tp, Tm, cell_p, cell_m);
  double* Lb = malloc(nf * sizeof(double));
  double S = smoothness(g, b, Lb);
  free(Lb);
  terms[1] = D; terms[2] = S; terms[3] = P;
  terms[0] = D + g->alpha * S + g->beta * P;
  if (want_lin) {
    gradient_from_lin(g, &lin, b, grad);
    lin_free(&lin);
  }
  return bad;
}

/* ------------------------------------------------------------------------------------------ */
/* adjoints (vector-Jacobian products) of the corrected images and of J, at fixed b            */
/* ------------------------------------------------------------------------------------------ */

/* Adjoint of the corrected images of Eq. 1 at b.  Given upstream sensitivities gTp, gTm (image
 * shaped; either may be NULL, meaning zero) it returns
 *   dIp = (dT+/dI+)^T gTp,  dIm = (dT-/dI-)^T gTm                         (image shaped)
 *   db  = (dT+/db)^T gTp + (dT-/db)^T gTm                                 (field shaped)
 * each output optional (NULL).  From the definitions, per cell j of a column:
 *   T+_j = [(1 - w) I+[i] + w I+[i+1]] (1 + delta_j),  i = floor(t+_j),  w = t+_j - i, so
 *   dT+_j/dI+[i] = (1 - w)(1 + delta_j),  dT+_j/dI+[i+1] = w (1 + delta_j)  (entries inside the
 *   column only: outside it the image is the constant 0);
 *   t+_j = j + (b_j + b_{j+1})/2 and delta_j = b_{j+1} - b_j, so
 *   dT+_j/db_j     = 1/2 I+'(t+)(1 + delta) - I+(t+),
 *   dT+_j/db_{j+1} = 1/2 I+'(t+)(1 + delta) + I+(t+);
 *   T-_j = I-(t-_j)(1 - delta_j), t-_j = j - (b_j + b_{j+1})/2, so
 *   dT-_j/db_j     = -1/2 I-'(t-)(1 - delta) + I-(t-),
 *   dT-_j/db_{j+1} = -1/2 I-'(t-)(1 - delta) - I-(t-).
 * I' is the slope of the cell that contains t (the right-hand derivative at an integer t). */
void orc_correct_adjoint(const orc_geom* g, const float* Ip, const float* Im, const double* b,
                         int contract, const double* gTp, const double* gTm, double* dIp,
                         double* dIm, double* db) {
  int64_t m = g->d[g->p];
  int64_t si[3], sf[3]; img_strides(g, si); fld_strides(g, sf);
  int64_t sti = si[g->p], stf = sf[g->p];
  int64_t ncols = column_count(g);
  if (dIp) memset(dIp, 0, img_count(g) * sizeof(double));
  if (dIm) memset(dIm, 0, img_count(g) * sizeof(double));
  if (db) memset(db, 0, fld_count(g) * sizeof(double));
  for (int64_t col = 0; col < ncols; ++col) {
    int64_t oi, of, c0, c1;
    column_offsets(g, col, &oi, &of, &c0, &c1);
    for (int64_t j = 0; j < m; ++j) {
      double bj = b[of + j * stf], bj1 = b[of + (j + 1) * stf];
      double tp, tm, delta;
      cell_positions(bj, bj1, j, contract, &tp, &tm, &delta);
      double Ipv, Ips, Imv, Ims;
      int64_t ip, im;
      interp1(Ip + oi, sti, m, tp, &Ipv, &Ips, &ip);
      interp1(Im + oi, sti, m, tm, &Imv, &Ims, &im);
      int64_t cidx = oi + j * sti;
      double gp = gTp ? gTp[cidx] : 0.0;
      double gm = gTm ? gTm[cidx] : 0.0;
      double wp = tp - floor(tp), wm = tm - floor(tm);
      if (dIp) {
        if (ip >= 0 && ip < m) dIp[oi + ip * sti] += gp * (1.0 - wp) * (1.0 + delta);
        if (ip + 1 >= 0 && ip + 1 < m) dIp[oi + (ip + 1) * sti] += gp * wp * (1.0 + delta);
      }
      if (dIm) {
        if (im >= 0 && im < m) dIm[oi + im * sti] += gm * (1.0 - wm) * (1.0 - delta);
        if (im + 1 >= 0 && im + 1 < m) dIm[oi + (im + 1) * sti] += gm * wm * (1.0 - delta);
      }
      if (db) {
        double dTp_dbj = 0.5 * Ips * (1.0 + delta) - Ipv;
        double dTp_dbj1 = 0.5 * Ips * (1.0 + delta) + Ipv;
        double dTm_dbj = -0.5 * Ims * (1.0 - delta) + Imv;
        double dTm_dbj1 = -0.5 * Ims * (1.0 - delta) - Imv;
        db[of + j * stf] += gp * dTp_dbj + gm * dTm_dbj;
        db[of + (j + 1) * stf] += gp * dTp_dbj1 + gm * dTm_dbj1;
      }
    }
  }
}

/* Gradient of J with respect to the two images at fixed b.  Only the distance term depends on
 * them: D = vol/2 sum_j r_j^2 with r_j = T+_j - T-_j (Eq. 2), so dJ/dI+- = (dT+-/dI+-)^T (+-vol r).
 * Returns the number of barrier-infeasible cells (the image gradient is still that of D). */
int64_t orc_image_grad(const orc_geom* g, const float* Ip, const float* Im, const double* b,
                       int contract, double* dIp, double* dIm) {
  int64_t nc = img_count(g);
  double* Tp = malloc(nc * sizeof(double));
  double* Tm = malloc(nc * sizeof(double));
  double* gp = malloc(nc * sizeof(double));
  double* gm = malloc(nc * sizeof(double));
  double D, P;
  int64_t bad = residual_pass(g, Ip, Im, b, contract, &D, &P, NULL, Tp, Tm, NULL, NULL);
  double vol = cell_volume(g);
  for (int64_t k = 0; k < nc; ++k) {
    double r = Tp[k] - Tm[k];
    gp[k] = vol * r;
    gm[k] = -vol * r;
  }
  orc_correct_adjoint(g, Ip, Im, b, contract, gp, gm, dIp, dIm, NULL);
  free(Tp); free(Tm); free(gp); free(gm);
  return bad;
}

/* GN Hessian about b applied to v */
int orc_hessvec(const orc_geom* g, const float* Ip, const float* Im, const double* b,
                int contract, const double* v, double* Hv) {
  orc_lin lin;
  if (!lin_alloc(&lin, img_count(g))) return -1;
  double D, P;
  residual_pass(g, Ip, Im, b, contract, &D, &P, &lin, NULL, NULL, NULL, NULL);
  hessvec_from_lin(g, &lin, v, Hv);
  lin_free(&lin);
  return 0;
}

/* diagonal of the GN Hessian about b */
int orc_hessdiag(const orc_geom* g, const float* Ip, const float* Im, const double* b,
                 int contract, double* diag) {
  orc_lin lin;
  if (!lin_alloc(&lin, img_count(g))) return -1;
  double D, P;
  residual_pass(g, Ip, Im, b, contract, &D, &P, &lin, NULL, NULL, NULL, NULL);
  hessdiag_from_lin(g, &lin, diag);
  lin_free(&lin);
  return 0;
}

/* preconditioner application z = M^{-1} r about b: kind 0 = Jacobi, 1 = per-column block */
int orc_precond(const orc_geom* g, const float* Ip, const float* Im, const double* b,
                int contract, int kind, const double* r, double* z) {
  int64_t nf = fld_count(g);
  orc_lin lin;
  if (!lin_alloc(&lin, img_count(g))) return -1;
  double D, P;
  residual_pass(g, Ip, Im, b, contract, &D, &P, &lin, NULL, NULL, NULL, NULL);
  if (kind == 0) {
    double* diag = malloc(nf * sizeof(double));
    hessdiag_from_lin(g, &lin, diag);
    jacobi_precond(nf, diag, r, z);
    free(diag);
  } else {
    column_precond_from_lin(g, &lin, r, z);
  }
  lin_free(&lin);
  return 0;
}

/* the tridiagonal diagonal block of one column (dia: m+1, off: m) */
int orc_column_block(const orc_geom* g, const float* Ip, const float* Im, const double* b,
                     int contract, int64_t col, double* dia, double* off) {
  orc_lin lin;
  if (!lin_alloc(&lin, img_count(g))) return -1;
  double D, P;
  residual_pass(g, Ip, Im, b, contract, &D, &P, &lin, NULL, NULL, NULL, NULL);
  column_block(g, &lin, col, dia, off);
  lin_free(&lin);
  return 0;
}

/* all column blocks at once, field shaped: dia at every node, off between node k and k+1 stored
 * at node k (0 at the last node) */
int orc_column_blocks(const orc_geom* g, const float* Ip, const float* Im, const double* b,
                      int contract, double* dia_f, double* off_f) {
  int64_t m = g->d[g->p];
  int64_t sf[3]; fld_strides(g, sf);
  orc_lin lin;
  if (!lin_alloc(&lin, img_count(g))) return -1;
  double D, P;
  residual_pass(g, Ip, Im, b, contract, &D, &P, &lin, NULL, NULL, NULL, NULL);
  double* dia = malloc((m + 1) * sizeof(double));
  double* off = malloc((m + 1) * sizeof(double));
  int64_t ncols = column_count(g);
  for (int64_t col = 0; col < ncols; ++col) {
    int64_t oi, of, c0, c1;
    column_offsets(g, col, &oi, &of, &c0, &c1);
    column_block(g, &lin, col, dia, off);
    for (int64_t k = 0; k <= m; ++k) {
      dia_f[of + k * sf[g->p]] = dia[k];
      off_f[of + k * sf[g->p]] = k < m ? off[k] : 0.0;
    }
  }
  free(dia); free(off);
  lin_free(&lin);
  return 0;
}

/* negative Laplacian of the field (exported for the null-space pin) */
void orc_apply_laplacian(const orc_geom* g, const double* x, double* y) { orc_laplacian(g, x, y); }

/* ------------------------------------------------------------------------------------------ */
/* optimal-transport initialisation (Sec. 2.2)                                                  */
/* ------------------------------------------------------------------------------------------ */

/* The positivity shift of Sec. 2.2: s = max(0, -min) + eps * max|I| over both images. */
static double ot_shift(const float* Ip, const float* Im, int64_t n, double eps, int contract) {
  float mn = Ip[0], mx = fabsf(Ip[0]);
  for (int64_t i = 0; i < n; ++i) {
    if (Ip[i] < mn) mn = Ip[i];
    if (Im[i] < mn) mn = Im[i];
    if (fabsf(Ip[i]) > mx) mx = fabsf(Ip[i]);
    if (fabsf(Im[i]) > mx) mx = fabsf(Im[i]);
  }
  if (contract) {
    float neg = -mn > 0.0f ? -mn : 0.0f;
    float e = (float)eps;
    float em = e * mx;
    float s = neg + em;
    return (double)s;
  }
  double neg = -(double)mn > 0.0 ? -(double)mn : 0.0;
  return neg + eps * (double)mx;
}

/* Normalised cumulative distribution of one shifted column at the m+1 nodes:
 * C(0) = 0, C(k) = sum_{j<k} i(j) / sum_{j<m} i(j).  contract: single precision, left to right.
 * Returns 0 when the column has no mass (C is then left undefined). */
static int column_cdf(const float* col, int64_t st, int64_t m, double shift, int contract,
                      double* C) {
  if (contract) {
    float s = (float)shift;
    float acc = 0.0f;
    float* tmp = malloc((m + 1) * sizeof(float));
    tmp[0] = 0.0f;
    for (int64_t j = 0; j < m; ++j) {
      float v = col[j * st] + s;
      acc = acc + v;
      tmp[j + 1] = acc;
    }
    float tot = tmp[m];
    int ok = tot > 0.0f;
    for (int64_t k = 0; k <= m; ++k) C[k] = ok ? (double)(tmp[k] / tot) : 0.0;
    free(tmp);
    return ok;
  }
  double acc = 0.0;
  C[0] = 0.0;
  for (int64_t j = 0; j < m; ++j) {
    acc += (double)col[j * st] + shift;
    C[j + 1] = acc;
  }
  double tot = C[m];
  if (!(tot > 0.0)) return 0;
  for (int64_t k = 0; k <= m; ++k) C[k] /= tot;
  return 1;
}

/* Pseudo-inverse of a CDF by the linear spline through (k, C(k)):
 * with k* = min{k : C(k+1) >= r}, C^{-1}(r) = k* + (r - C(k*)) / (C(k*+1) - C(k*)).
 * r <= 0 maps to 0.  *kstar receives k* (the merge index). */
static double cdf_inverse(const double* C, int64_t m, double r, int32_t* kstar) {
  if (r <= 0.0) { *kstar = 0; return 0.0; }
  int64_t k = 0;
  while (k < m - 1 && C[k + 1] < r) ++k;
  *kstar = (int32_t)k;
  double den = C[k + 1] - C[k];
  double x = (double)k + (r - C[k]) / den;
  if (x > (double)m) x = (double)m;
  return x;
}

/* separable 3-tap Gaussian, sigma = 1 voxel, replicate boundary, along one axis of the field */
static void blur_axis(const orc_geom* g, int ax, const double* x, double* y) {
  int64_t n[3] = {fld_dim(g, 0), fld_dim(g, 1), fld_dim(g, 2)};
  int64_t s[3]; fld_strides(g, s);
  double w = exp(-0.5), norm = 1.0 + 2.0 * w;
#pragma omp parallel for schedule(static)
  for (int64_t i0 = 0; i0 < n[0]; ++i0)
    for (int64_t i1 = 0; i1 < n[1]; ++i1)
      for (int64_t i2 = 0; i2 < n[2]; ++i2) {
        int64_t idx[3] = {i0, i1, i2};
        int64_t k = i0 * s[0] + i1 * s[1] + i2 * s[2];
        int64_t km = idx[ax] > 0 ? k - s[ax] : k;
        int64_t kp = idx[ax] < n[ax] - 1 ? k + s[ax] : k;
        y[k] = (w * x[km] + x[k] + w * x[kp]) / norm;
      }
}

/* the 3x3x3 Gaussian of Sec. 2.4 as three separable passes */
void orc_blur(const orc_geom* g, double* b) {
  int64_t nf = fld_count(g);
  double* t = malloc(nf * sizeof(double));
  blur_axis(g, 0, b, t);
  blur_axis(g, 1, t, b);
  blur_axis(g, 2, b, t);
  memcpy(b, t, nf * sizeof(double));
  free(t);
}

/* OT field-map initialisation, Sec. 2.2: for every node k of every column,
 *   b0_k = 1/4 [ (C+^{-1}(C-(k)) - k) - (C-^{-1}(C+(k)) - k) ],
 * i.e. half of the displacement of T- minus half of the displacement of T+, where
 * T+- = C_half^{-1} o C+-, C_half^{-1} = (C+^{-1} + C-^{-1})/2.  Columns without mass get 0.
 * kidx_p / kidx_m (nullable, field shaped) receive the merge indices k* of C-^{-1}(C+(k)) and
 * C+^{-1}(C-(k)). */
void orc_ot_init(const orc_geom* g, const float* Ip, const float* Im, double eps, int contract,
                 int blur, double* b0, int32_t* kidx_p, int32_t* kidx_m) {
  int64_t m = g->d[g->p];
  int64_t si[3], sf[3]; img_strides(g, si); fld_strides(g, sf);
  double shift = ot_shift(Ip, Im, img_count(g), eps, contract);
  int64_t ncols = column_count(g);
#pragma omp parallel
  {
  double* Cp = malloc((m + 1) * sizeof(double));
  double* Cm = malloc((m + 1) * sizeof(double));
#pragma omp for schedule(static)
  for (int64_t col = 0; col < ncols; ++col) {
    int64_t oi, of, c0, c1;
    column_offsets(g, col, &oi, &of, &c0, &c1);
    int okp = column_cdf(Ip + oi, si[g->p], m, shift, contract, Cp);
    int okm = column_cdf(Im + oi, si[g->p], m, shift, contract, Cm);
    for (int64_t k = 0; k <= m; ++k) {
      int64_t f = of + k * sf[g->p];
      if (!okp || !okm) {
        b0[f] = 0.0;
        if (kidx_p) kidx_p[f] = 0;
        if (kidx_m) kidx_m[f] = 0;
        continue;
      }
      int32_t kp, km;
      double xp = cdf_inverse(Cm, m, Cp[k], &kp);  /* C-^{-1}(C+(k)) */
      double xm = cdf_inverse(Cp, m, Cm[k], &km);  /* C+^{-1}(C-(k)) */
      b0[f] = 0.25 * ((xm - (double)k) - (xp - (double)k));
      if (kidx_p) kidx_p[f] = kp;
      if (kidx_m) kidx_m[f] = km;
    }
  }
  free(Cp); free(Cm);
  }
  if (blur) orc_blur(g, b0);
}

/* ------------------------------------------------------------------------------------------ */
/* GN-PCG with Armijo line search (Sec. 2.3.1)                                                  */
/* ------------------------------------------------------------------------------------------ */

/* preconditioned CG (Hestenes-Stiefel) for H q = rhs, q0 = 0; stops after max_it iterations, when
 * ||r|| / ||r0|| < rtol, or when p^T H p <= 0.  Returns the number of Hessian products. */
static int pcg(const orc_geom* g, const orc_lin* lin, const double* diag, int precond,
               const double* rhs, int max_it, double rtol, double* q, double* relres) {
  int64_t n = fld_count(g);
  double* r = malloc(n * sizeof(double));
  double* z = malloc(n * sizeof(double));
  double* p = malloc(n * sizeof(double));
  double* Hp = malloc(n * sizeof(double));
#pragma omp parallel for schedule(static)
  for (int64_t k = 0; k < n; ++k) { q[k] = 0.0; r[k] = rhs[k]; }
  double rr0 = dot(r, r, n);
  int it = 0;
  *relres = rr0 > 0.0 ? 1.0 : 0.0;
  if (rr0 > 0.0) {
    if (precond == 0) jacobi_precond(n, diag, r, z);
    else column_precond_from_lin(g, lin, r, z);
#pragma omp parallel for schedule(static)
    for (int64_t k = 0; k < n; ++k) p[k] = z[k];
    double rho = dot(r, z, n);
    for (int i = 0; i < max_it; ++i) {
      hessvec_from_lin(g, lin, p, Hp);
      double pHp = dot(p, Hp, n);
      if (!(pHp > 0.0)) break;
      double a = rho / pHp;
#pragma omp parallel for schedule(static)
      for (int64_t k = 0; k < n; ++k) { q[k] += a * p[k]; r[k] -= a * Hp[k]; }
      it = i + 1;
      double rr = dot(r, r, n);
      *relres = sqrt(rr) / sqrt(rr0);
      if (*relres < rtol) break;
      if (precond == 0) jacobi_precond(n, diag, r, z);
      else column_precond_from_lin(g, lin, r, z);
      double rho_new = dot(r, z, n);
      double beta = rho_new / rho;
      rho = rho_new;
#pragma omp parallel for schedule(static)
      for (int64_t k = 0; k < n; ++k) p[k] = z[k] + beta * p[k];
    }
  }
  free(r); free(z); free(p); free(Hp);
  return it;
}

/* J only (line-search trial) */
static double objective_only(const orc_geom* g, const float* Ip, const float* Im, const double* b,
                             int contract, double* Lb_scratch) {
  double D, P;
  residual_pass(g, Ip, Im, b, contract, &D, &P, NULL, NULL, NULL, NULL, NULL);
  double S = smoothness(g, b, Lb_scratch);
  return D + g->alpha * S + g->beta * P;
}

/* Full solve: optional OT init, then opts->gn_iters Gauss-Newton iterations
 *   b <- b + gamma q,  H q ~= -grad J by PCG,  gamma from Armijo backtracking (1, 1/2, 1/4, ...).
 * A rejected line search (or a non-descent q) leaves b unchanged for that iteration.  Stops early
 * only when J(b) is not finite (returns 1 for +inf, i.e. barrier infeasible; 2 for NaN).
 * stats (nullable): gn_iters x ST_NFIELDS doubles. */
/* Feasible start for the Gauss-Newton loop (a reading where the paper is silent): the barrier
 * of Eq. 3 is +inf unless |delta_j| < 1 in every cell, so J is +inf at a start outside that set
 * and no Armijo step can be accepted.  b = 0 is feasible; the start is halved until
 * max |delta| < 1 (power-of-two factors, exact).  Returns the factor applied. */
double orc_feasible_start(const orc_geom* g, double* b) {
  int64_t m = g->d[g->p];
  int64_t sf[3]; fld_strides(g, sf);
  int64_t stf = sf[g->p];
  int64_t ncols = column_count(g);
  double s = 0.0;
  for (int64_t col = 0; col < ncols; ++col) {
    int64_t oi, of, c0, c1;
    column_offsets(g, col, &oi, &of, &c0, &c1);
    for (int64_t j = 0; j < m; ++j) {
      double delta = b[of + (j + 1) * stf] - b[of + j * stf];
      if (fabs(delta) > s) s = fabs(delta);
    }
  }
  double f = 1.0;
  for (int k = 0; k < 64 && s * f >= 1.0; ++k) f *= 0.5;
  if (f != 1.0)
    for (int64_t i = 0; i < fld_count(g); ++i) b[i] *= f;
  return f;
}

int orc_solve(const orc_geom* g, const float* Ip, const float* Im, const orc_opts* o,
              double* b, double* stats) {
  int64_t nf = fld_count(g), nc = img_count(g);
  if (o->init) {
    orc_ot_init(g, Ip, Im, o->ot_eps, o->contract, o->ot_blur, b, NULL, NULL);
    orc_feasible_start(g, b);
  }
  orc_lin lin;
  if (!lin_alloc(&lin, nc)) return -1;
  double* grad = malloc(nf * sizeof(double));
  double* diag = malloc(nf * sizeof(double));
  double* rhs = malloc(nf * sizeof(double));
  double* q = malloc(nf * sizeof(double));
  double* bt = malloc(nf * sizeof(double));
  double* Lb = malloc(nf * sizeof(double));
  int status = 0;
  if (stats) for (int64_t i = 0; i < (int64_t)o->gn_iters * ST_NFIELDS; ++i) stats[i] = NAN;
  for (int it = 0; it < o->gn_iters; ++it) {
    double D, P;
    residual_pass(g, Ip, Im, b, o->contract, &D, &P, &lin, NULL, NULL, NULL, NULL);
    double S = smoothness(g, b, Lb);
    double J = D + g->alpha * S + g->beta * P;
    double* st = stats ? stats + (int64_t)it * ST_NFIELDS : NULL;
    if (st) { st[ST_J] = J; st[ST_D] = D; st[ST_S] = S; st[ST_P] = P; }
    if (!isfinite(J)) { status = isnan(J) ? 2 : 1; break; }
    gradient_from_lin(g, &lin, b, grad);
    if (o->precond == 0) hessdiag_from_lin(g, &lin, diag);
#pragma omp parallel for schedule(static)
    for (int64_t k = 0; k < nf; ++k) rhs[k] = -grad[k];
    double relres;
    int pit = pcg(g, &lin, diag, o->precond, rhs, o->pcg_max_iters, o->pcg_rtol, q, &relres);
    double gq = dot(grad, q, nf);
    double gamma = 0.0;
    int trials = 0;
    if (gq < 0.0) {
      double step = 1.0;
      for (int t = 0; t < o->ls_max_iters; ++t) {
        ++trials;
#pragma omp parallel for schedule(static)
        for (int64_t k = 0; k < nf; ++k) bt[k] = b[k] + step * q[k];
        double Jt = objective_only(g, Ip, Im, bt, o->contract, Lb);
        if (Jt <= J + o->armijo_c1 * step * gq) { gamma = step; break; }
        step *= 0.5;
      }
    }
    if (gamma > 0.0) {
#pragma omp parallel for schedule(static)
      for (int64_t k = 0; k < nf; ++k) b[k] += gamma * q[k];
    }
    if (st) {
      st[ST_GNORM] = sqrt(dot(grad, grad, nf));
      st[ST_GQ] = gq;
      st[ST_GAMMA] = gamma;
      st[ST_PCG_IT] = pit;
      st[ST_PCG_RELRES] = relres;
      st[ST_LS_TRIALS] = trials;
    }
  }
  lin_free(&lin);
  free(grad); free(diag); free(rhs); free(q); free(bt); free(Lb);
  return status;
}

/* PCG alone on the GN system about b (exported so that tests can pin it against a dense solve) */
int orc_pcg(const orc_geom* g, const float* Ip, const float* Im, const double* b, int contract,
            int precond, const double* rhs, int max_it, double rtol, double* q, double* relres) {
  int64_t nf = fld_count(g);
  orc_lin lin;
  if (!lin_alloc(&lin, img_count(g))) return -1;
  double D, P;
  residual_pass(g, Ip, Im, b, contract, &D, &P, &lin, NULL, NULL, NULL, NULL);
  double* diag = malloc(nf * sizeof(double));
  hessdiag_from_lin(g, &lin, diag);
  int it = pcg(g, &lin, diag, precond, rhs, max_it, rtol, q, relres);
  free(diag);
  lin_free(&lin);
  return it;
}

/* ------------------------------------------------------------------------------------------ */
/* implicit differentiation through the solve                                                  */
/* ------------------------------------------------------------------------------------------ */

/* At a stationary point b* of J the gradient g(b*; theta) = 0 defines b*(theta) for every input
 * theta (alpha, beta, the two images).  For a loss L(b*), the implicit function theorem with the
 * Gauss-Newton Hessian H of Sec. 2.3.1 standing in for the Hessian of J gives
 *   dL/dtheta = -(dg/dtheta)^T v,   H v = dL/db*.
 * The pieces, for a given v: */

/* v^T dg/dalpha and v^T dg/dbeta: g = vol [Jr^T r + alpha h_p^2 L b + beta/2 D^T phi'(delta)] is
 * affine in alpha and beta, so dg/dalpha = vol h_p^2 L b and dg/dbeta = vol/2 D^T phi'(delta). */
void orc_theta_dots(const orc_geom* g, const float* Ip, const float* Im, const double* b,
                    int contract, const double* v, double out[2]) {
  int64_t nf = fld_count(g), nc = img_count(g);
  double vol = cell_volume(g), hp = g->h[g->p];
  orc_lin lin;
  lin_alloc(&lin, nc);
  double D, P;
  residual_pass(g, Ip, Im, b, contract, &D, &P, &lin, NULL, NULL, NULL, NULL);
  double* Lb = malloc(nf * sizeof(double));
  double* u = calloc(nf, sizeof(double));
  orc_laplacian(g, b, Lb);
  fd_transpose_add(g, lin.dphi, u);
  double sa = 0.0, sb = 0.0;
  for (int64_t k = 0; k < nf; ++k) {
    sa += v[k] * vol * hp * hp * Lb[k];
    sb += v[k] * 0.5 * vol * u[k];
  }
  out[0] = sa;
  out[1] = sb;
  free(Lb); free(u);
  lin_free(&lin);
}

/* d/dI+- of F = v^T g.  Only the distance term depends on the images:
 *   F_D = vol sum_j r_j u_j,   u_j = (Jr v)_j = jl_j v_j + jr_j v_{j+1},
 * with r_j = I+(t+)(1 + delta) - I-(t-)(1 - delta), jl = a/2 - c, jr = a/2 + c,
 * a = I+'(t+)(1 + delta) + I-'(t-)(1 - delta), c = I+(t+) + I-(t-).  Per cell, for the two voxels
 * i, i+1 around t+ (weights 1 - w, w; slope I+[i+1] - I+[i]):
 *   dr/dI+[i]   = (1 - w)(1 + delta),           dr/dI+[i+1] = w (1 + delta),
 *   da/dI+[i]   = -(1 + delta),                 da/dI+[i+1] = (1 + delta),
 *   dc/dI+[i]   = 1 - w,                        dc/dI+[i+1] = w,
 * and du/dI = v_j (da/2 - dc) + v_{j+1} (da/2 + dc); likewise for I- with t-, (1 - delta) and
 * dr/dI- = -(...).  dF/dI[k] = vol sum over cells (u_j dr_j/dI[k] + r_j du_j/dI[k]). */
void orc_mixed_image_adjoint(const orc_geom* g, const float* Ip, const float* Im, const double* b,
                             int contract, const double* v, double* dIp, double* dIm) {
  int64_t m = g->d[g->p];
  int64_t si[3], sf[3]; img_strides(g, si); fld_strides(g, sf);
  int64_t sti = si[g->p], stf = sf[g->p];
  int64_t ncols = column_count(g);
  double vol = cell_volume(g);
  memset(dIp, 0, img_count(g) * sizeof(double));
  memset(dIm, 0, img_count(g) * sizeof(double));
  for (int64_t col = 0; col < ncols; ++col) {
    int64_t oi, of, c0, c1;
    column_offsets(g, col, &oi, &of, &c0, &c1);
    for (int64_t j = 0; j < m; ++j) {
      double bj = b[of + j * stf], bj1 = b[of + (j + 1) * stf];
      double vj = v[of + j * stf], vj1 = v[of + (j + 1) * stf];
      double tp, tm, delta;
      cell_positions(bj, bj1, j, contract, &tp, &tm, &delta);
      double Ipv, Ips, Imv, Ims;
      int64_t ip, im;
      interp1(Ip + oi, sti, m, tp, &Ipv, &Ips, &ip);
      interp1(Im + oi, sti, m, tm, &Imv, &Ims, &im);
      double r = Ipv * (1.0 + delta) - Imv * (1.0 - delta);
      double a = Ips * (1.0 + delta) + Ims * (1.0 - delta);
      double c = Ipv + Imv;
      double u = (0.5 * a - c) * vj + (0.5 * a + c) * vj1;
      double wp = tp - floor(tp), wm = tm - floor(tm);
      /* the two voxels of each image model and their derivatives */
      for (int s = 0; s < 2; ++s) {   /* s = 0: voxel i, s = 1: voxel i + 1 */
        double wpk = s == 0 ? 1.0 - wp : wp, wmk = s == 0 ? 1.0 - wm : wm;
        double sgn = s == 0 ? -1.0 : 1.0;   /* d(slope)/dI at voxel i, i + 1 */
        /* I+ */
        double dr = wpk * (1.0 + delta);
        double da = sgn * (1.0 + delta);
        double dc = wpk;
        double du = vj * (0.5 * da - dc) + vj1 * (0.5 * da + dc);
        int64_t k = ip + s;
        if (k >= 0 && k < m) dIp[oi + k * sti] += vol * (u * dr + r * du);
        /* I- */
        dr = -wmk * (1.0 - delta);
        da = sgn * (1.0 - delta);
        dc = wmk;
        du = vj * (0.5 * da - dc) + vj1 * (0.5 * da + dc);
        k = im + s;
        if (k >= 0 && k < m) dIm[oi + k * sti] += vol * (u * dr + r * du);
      }
    }
  }
}

/* The whole step: v = H^{-1} dL/db* by Jacobi PCG (x0 = 0, at most max_it iterations, relative
 * residual rtol), then dL/dI+- = -d(v^T g)/dI+-, dL/dalpha = -v^T dg/dalpha,
 * dL/dbeta = -v^T dg/dbeta.  Returns the PCG iteration count. */
int orc_solve_adjoint(const orc_geom* g, const float* Ip, const float* Im, const double* b,
                      int contract, const double* dLdb, int max_it, double rtol, double* v,
                      double* dIp, double* dIm, double* dtheta) {
  double relres;
  int it = orc_pcg(g, Ip, Im, b, contract, 0, dLdb, max_it, rtol, v, &relres);
  orc_mixed_image_adjoint(g, Ip, Im, b, contract, v, dIp, dIm);
  for (int64_t k = 0; k < img_count(g); ++k) { dIp[k] = -dIp[k]; dIm[k] = -dIm[k]; }
  double s[2];
  orc_theta_dots(g, Ip, Im, b, contract, v, s);
  dtheta[0] = -s[0];
  dtheta[1] = -s[1];
  return it;
}

/* ------------------------------------------------------------------------------------------ */
/* least-squares correction (Sec. 2.4 "Image Correction")                                     */
/* ------------------------------------------------------------------------------------------ */

/* Push-forward matrix of one PE column for direction s = +1 / -1: true cell j (the interval
 * [j - 1/2, j + 1/2] in cell-index coordinates, field nodes at its edges) is mapped to
 * [e_j, e_{j+1}] with e_j = j - 1/2 + s b_j, and its mass is spread uniformly there; distorted
 * cell i collects the part that falls in [i - 1/2, i + 1/2]:
 *   P[i][j] = |[i - 1/2, i + 1/2] ∩ [e_j, e_{j+1}]| / (e_{j+1} - e_j).
 * Needs e_{j+1} > e_j (|delta_j| < 1).  P is m x m, row-major, dense. */
static void pushforward_column(const double* bcol, int64_t stf, int64_t m, double s, double* P) {
  for (int64_t i = 0; i < m; ++i)
    for (int64_t j = 0; j < m; ++j) {
      double e0 = (double)j - 0.5 + s * bcol[j * stf];
      double e1 = (double)j + 0.5 + s * bcol[(j + 1) * stf];
      double lo = fmax(e0, (double)i - 0.5), hi = fmin(e1, (double)i + 0.5);
      P[i * m + j] = hi > lo ? (hi - lo) / (e1 - e0) : 0.0;
    }
}

/* Corrected image by least squares: per PE column, the true image I minimising
 *   |P+ I - I+|^2 + |P- I - I-|^2 + lambda |I|^2,
 * from the normal equations (P+^T P+ + P-^T P- + lambda Id) I = P+^T I+ + P-^T I- solved by a
 * textbook Cholesky factorisation.  lambda > 0 keeps cells whose mass leaves the column in both
 * images at 0.  Returns the number of columns whose field has |delta| >= 1 somewhere (left at 0). */
int64_t orc_ls_correct(const orc_geom* g, const float* Ip, const float* Im, const double* b,
                       double lambda, double* out) {
  int64_t m = g->d[g->p];
  int64_t si[3], sf[3]; img_strides(g, si); fld_strides(g, sf);
  int64_t sti = si[g->p], stf = sf[g->p];
  int64_t ncols = column_count(g);
  double* Pp = malloc(m * m * sizeof(double));
  double* Pm = malloc(m * m * sizeof(double));
  double* N = malloc(m * m * sizeof(double));
  double* rhs = malloc(m * sizeof(double));
  int64_t bad = 0;
  for (int64_t col = 0; col < ncols; ++col) {
    int64_t oi, of, c0, c1;
    column_offsets(g, col, &oi, &of, &c0, &c1);
    const double* bcol = b + of;
    int ok = 1;
    for (int64_t j = 0; j < m; ++j)
      if (!(fabs(bcol[(j + 1) * stf] - bcol[j * stf]) < 1.0)) ok = 0;
    if (!ok) {
      ++bad;
      for (int64_t j = 0; j < m; ++j) out[oi + j * sti] = 0.0;
      continue;
    }
    pushforward_column(bcol, stf, m, +1.0, Pp);
    pushforward_column(bcol, stf, m, -1.0, Pm);
    for (int64_t j = 0; j < m; ++j) {
      double r = 0.0;
      for (int64_t i = 0; i < m; ++i)
        r += Pp[i * m + j] * (double)Ip[oi + i * sti] + Pm[i * m + j] * (double)Im[oi + i * sti];
      rhs[j] = r;
      for (int64_t k = 0; k < m; ++k) {
        double a = 0.0;
        for (int64_t i = 0; i < m; ++i) a += Pp[i * m + j] * Pp[i * m + k] + Pm[i * m + j] * Pm[i * m + k];
        N[j * m + k] = a + (j == k ? lambda : 0.0);
      }
    }
    /* Cholesky N = L L^T (L in the lower triangle of N), then L y = rhs, L^T x = y */
    for (int64_t j = 0; j < m; ++j) {
      double d = N[j * m + j];
      for (int64_t k = 0; k < j; ++k) d -= N[j * m + k] * N[j * m + k];
      d = sqrt(d);
      N[j * m + j] = d;
      for (int64_t i = j + 1; i < m; ++i) {
        double a = N[i * m + j];
        for (int64_t k = 0; k < j; ++k) a -= N[i * m + k] * N[j * m + k];
        N[i * m + j] = a / d;
      }
    }
    for (int64_t j = 0; j < m; ++j) {
      double a = rhs[j];
      for (int64_t k = 0; k < j; ++k) a -= N[j * m + k] * rhs[k];
      rhs[j] = a / N[j * m + j];
    }
    for (int64_t j = m - 1; j >= 0; --j) {
      double a = rhs[j];
      for (int64_t k = j + 1; k < m; ++k) a -= N[k * m + j] * rhs[k];
      rhs[j] = a / N[j * m + j];
    }
    for (int64_t j = 0; j < m; ++j) out[oi + j * sti] = rhs[j];
  }
  free(Pp); free(Pm); free(N); free(rhs);
  return bad;
}

/* the dense push-forward matrix of one column (test access) */
void orc_pushforward_matrix(const double* bcol, int64_t m, double s, double* P) {
  pushforward_column(bcol, 1, m, s, P);
}

/* ------------------------------------------------------------------------------------------ */
/* ADMM (Sec. 2.3.2): the b-update                                                             */
/* ------------------------------------------------------------------------------------------ */

/* The splitting of Sec. 2.3.2 puts the PE-direction part S3 of the smoothness term into
 *   F(b) = D(b) + alpha S3(b) + beta P(b),
 * and the in-plane parts S1 + S2 into G(z).  In PE-voxel units S3 = vol/2 h_p^2 b^T (G_p^T G_p /
 * h_p^2) b = vol/2 sum over columns of sum_k (b_{k+1} - b_k)^2.  With the scaled multiplier u the
 * b-update minimises the column-separable
 *   F_c(b) = F(b) + rho vol / 2 ||b - c||^2,   c = z - u,
 * (the augmentation weight rho h^3 of Sec. 2.3.2 read as rho times the cell volume). */
static double smooth_pe(const orc_geom* g, const double* b, double* Lpe /* nullable: L_pe b */) {
  int64_t m = g->d[g->p];
  int64_t sf[3]; fld_strides(g, sf);
  int64_t stf = sf[g->p];
  int64_t ncols = column_count(g);
  double s = 0.0;
  if (Lpe) memset(Lpe, 0, fld_count(g) * sizeof(double));
  for (int64_t col = 0; col < ncols; ++col) {
    int64_t oi, of, c0, c1;
    column_offsets(g, col, &oi, &of, &c0, &c1);
    for (int64_t k = 0; k < m; ++k) {
      double d = b[of + (k + 1) * stf] - b[of + k * stf];
      s += d * d;
      if (Lpe) {                       /* G_p^T G_p b, one edge at a time */
        Lpe[of + (k + 1) * stf] += d;
        Lpe[of + k * stf] -= d;
      }
    }
  }
  return 0.5 * cell_volume(g) * s;
}

/* F_c at b: terms = {F_c, D, S3, P, prox} with prox = vol/2 ||b - c||^2 (so F_c = D + alpha S3 +
 * beta P + rho prox); gradient on request:
 *   vol [Jr^T r + alpha G_p^T G_p b + beta/2 D^T phi'(delta) + rho (b - c)].
 * Returns the number of barrier-infeasible cells. */
int64_t orc_admm_eval(const orc_geom* g, const float* Ip, const float* Im, const double* b,
                      int contract, double rho, const double* c, double* terms, double* grad) {
  int64_t nc = img_count(g), nf = fld_count(g);
  double vol = cell_volume(g);
  orc_lin lin;
  int want_lin = grad != NULL;
  if (want_lin && !lin_alloc(&lin, nc)) return -1;
  double D, P;
  int64_t bad = residual_pass(g, Ip, Im, b, contract, &D, &P, want_lin ? &lin : NULL, NULL, NULL,
                              NULL, NULL);
  double* Lpe = malloc(nf * sizeof(double));
  double S3 = smooth_pe(g, b, Lpe);
  double prox = 0.0;
  for (int64_t k = 0; k < nf; ++k) prox += (b[k] - c[k]) * (b[k] - c[k]);
  prox *= 0.5 * vol;
  terms[1] = D; terms[2] = S3; terms[3] = P; terms[4] = prox;
  terms[0] = D + g->alpha * S3 + g->beta * P + rho * prox;
  if (want_lin) {
    double* t = calloc(nf, sizeof(double));
    double* u = calloc(nf, sizeof(double));
    jr_transpose_add(g, &lin, lin.r, t);
    fd_transpose_add(g, lin.dphi, u);
    for (int64_t k = 0; k < nf; ++k)
      grad[k] = vol * (t[k] + g->alpha * Lpe[k] + 0.5 * g->beta * u[k] + rho * (b[k] - c[k]));
    free(t); free(u);
    lin_free(&lin);
  }
  free(Lpe);
  return bad;
}

/* The GN Hessian of F_c restricted to one PE column (it is block diagonal: F_c has no in-plane
 * coupling): vol [Jr^T Jr + alpha G_p^T G_p + beta/2 D^T diag(phi'') D + rho I], tridiagonal of
 * order m+1. */
static void admm_column_block(const orc_geom* g, const orc_lin* lin, int64_t col, double rho,
                              double* dia, double* off) {
  int64_t m = g->d[g->p];
  int64_t si[3]; img_strides(g, si);
  double vol = cell_volume(g);
  int64_t oi, of, c0, c1;
  column_offsets(g, col, &oi, &of, &c0, &c1);
  for (int64_t k = 0; k <= m; ++k) dia[k] = g->alpha * (double)((k > 0) + (k < m)) + rho;
  for (int64_t k = 0; k < m; ++k) off[k] = -g->alpha;
  for (int64_t j = 0; j < m; ++j) {
    int64_t c = oi + j * si[g->p];
    double jl = lin->jl[c], jr = lin->jr[c], q = 0.5 * g->beta * lin->d2phi[c];
    dia[j] += jl * jl + q;
    dia[j + 1] += jr * jr + q;
    off[j] += jl * jr - q;
  }
  for (int64_t k = 0; k <= m; ++k) dia[k] *= vol;
  for (int64_t k = 0; k < m; ++k) off[k] *= vol;
}

/* symmetric tridiagonal product y = T x of order n */
static void tridiag_apply(int64_t n, const double* dia, const double* off, const double* x,
                          double* y) {
  for (int64_t k = 0; k < n; ++k) {
    double v = dia[k] * x[k];
    if (k > 0) v += off[k - 1] * x[k - 1];
    if (k < n - 1) v += off[k] * x[k + 1];
    y[k] = v;
  }
}

/* BlockPCG (Sec. 2.3.2): the Jacobi-preconditioned CG of Sec. 2.3.1 run on every column's block
 * independently, with the column's own step sizes and its own stop (||r|| / ||r0|| < rtol after an
 * update, p^T H p <= 0, or max_it iterations).  q = 0 where the column's right-hand side is 0.
 * Returns the sum over columns of the iterations taken. */
static int64_t block_pcg(const orc_geom* g, const orc_lin* lin, double rho, const double* rhs,
                         int max_it, double rtol, double* q) {
  int64_t m = g->d[g->p], n = m + 1;
  int64_t sf[3]; fld_strides(g, sf);
  int64_t stf = sf[g->p];
  int64_t ncols = column_count(g), total = 0;
  double *dia = malloc(n * sizeof(double)), *off = malloc(n * sizeof(double));
  double *x = malloc(n * sizeof(double)), *r = malloc(n * sizeof(double));
  double *z = malloc(n * sizeof(double)), *p = malloc(n * sizeof(double));
  double *Hp = malloc(n * sizeof(double));
  for (int64_t col = 0; col < ncols; ++col) {
    int64_t oi, of, c0, c1;
    column_offsets(g, col, &oi, &of, &c0, &c1);
    admm_column_block(g, lin, col, rho, dia, off);
    for (int64_t k = 0; k < n; ++k) { x[k] = 0.0; r[k] = rhs[of + k * stf]; }
    double rr0 = 0.0;
    for (int64_t k = 0; k < n; ++k) rr0 += r[k] * r[k];
    if (rr0 > 0.0) {
      jacobi_precond(n, dia, r, z);
      for (int64_t k = 0; k < n; ++k) p[k] = z[k];
      double rz = 0.0;
      for (int64_t k = 0; k < n; ++k) rz += r[k] * z[k];
      for (int i = 0; i < max_it; ++i) {
        tridiag_apply(n, dia, off, p, Hp);
        double pHp = 0.0;
        for (int64_t k = 0; k < n; ++k) pHp += p[k] * Hp[k];
        if (!(pHp > 0.0)) break;
        double a = rz / pHp;
        for (int64_t k = 0; k < n; ++k) { x[k] += a * p[k]; r[k] -= a * Hp[k]; }
        ++total;
        double rr = 0.0;
        for (int64_t k = 0; k < n; ++k) rr += r[k] * r[k];
        if (sqrt(rr) / sqrt(rr0) < rtol) break;
        jacobi_precond(n, dia, r, z);
        double rz_new = 0.0;
        for (int64_t k = 0; k < n; ++k) rz_new += r[k] * z[k];
        double beta = rz_new / rz;
        rz = rz_new;
        for (int64_t k = 0; k < n; ++k) p[k] = z[k] + beta * p[k];
      }
    }
    for (int64_t k = 0; k < n; ++k) q[of + k * stf] = x[k];
  }
  free(dia); free(off); free(x); free(r); free(z); free(p); free(Hp);
  return total;
}

/* BlockPCG alone on the b-subproblem about b (exported for tests): q ~= -H^{-1} grad F_c. */
int64_t orc_block_pcg(const orc_geom* g, const float* Ip, const float* Im, const double* b,
                      int contract, double rho, const double* rhs, int max_it, double rtol,
                      double* q) {
  orc_lin lin;
  if (!lin_alloc(&lin, img_count(g))) return -1;
  double D, P;
  residual_pass(g, Ip, Im, b, contract, &D, &P, &lin, NULL, NULL, NULL, NULL);
  int64_t it = block_pcg(g, &lin, rho, rhs, max_it, rtol, q);
  lin_free(&lin);
  return it;
}

/* The dense block of one column (exported for tests) */
int orc_admm_column_block(const orc_geom* g, const float* Ip, const float* Im, const double* b,
                          int contract, double rho, int64_t col, double* dia, double* off) {
  orc_lin lin;
  if (!lin_alloc(&lin, img_count(g))) return -1;
  double D, P;
  residual_pass(g, Ip, Im, b, contract, &D, &P, &lin, NULL, NULL, NULL, NULL);
  admm_column_block(g, &lin, col, rho, dia, off);
  lin_free(&lin);
  return 0;
}

/* The b-update: gn_iters Gauss-Newton iterations on F_c (Sec. 2.3.2: the GN scheme of Sec. 2.3.1
 * with the search direction from BlockPCG), Armijo backtracking on F_c as in orc_solve.  Stops
 * early only when F_c is not finite (returns 1 for +inf, 2 for NaN).  stats (nullable):
 * gn_iters x 5 doubles {F_c before the step, gamma, grad^T q, BlockPCG iterations summed over
 * columns, line-search trials}. */
int orc_admm_bupdate(const orc_geom* g, const float* Ip, const float* Im, int contract,
                     double rho, const double* c, int gn_iters, int pcg_max_iters,
                     double pcg_rtol, int ls_max_iters, double armijo_c1, double* b,
                     double* stats) {
  int64_t nf = fld_count(g);
  double* grad = malloc(nf * sizeof(double));
  double* rhs = malloc(nf * sizeof(double));
  double* q = malloc(nf * sizeof(double));
  double* bt = malloc(nf * sizeof(double));
  orc_lin lin;
  if (!lin_alloc(&lin, img_count(g))) return -1;
  int status = 0;
  if (stats) for (int64_t i = 0; i < (int64_t)gn_iters * 5; ++i) stats[i] = NAN;
  for (int it = 0; it < gn_iters; ++it) {
    double terms[5];
    orc_admm_eval(g, Ip, Im, b, contract, rho, c, terms, grad);
    double F = terms[0];
    double* st = stats ? stats + (int64_t)it * 5 : NULL;
    if (st) st[0] = F;
    if (!isfinite(F)) { status = isnan(F) ? 2 : 1; break; }
    double D, P;
    residual_pass(g, Ip, Im, b, contract, &D, &P, &lin, NULL, NULL, NULL, NULL);
    for (int64_t k = 0; k < nf; ++k) rhs[k] = -grad[k];
    int64_t pit = block_pcg(g, &lin, rho, rhs, pcg_max_iters, pcg_rtol, q);
    double gq = dot(grad, q, nf);
    double gamma = 0.0;
    int trials = 0;
    if (gq < 0.0) {
      double step = 1.0;
      for (int t = 0; t < ls_max_iters; ++t) {
        ++trials;
        for (int64_t k = 0; k < nf; ++k) bt[k] = b[k] + step * q[k];
        double tt[5];
        orc_admm_eval(g, Ip, Im, bt, contract, rho, c, tt, NULL);
        if (tt[0] <= F + armijo_c1 * step * gq) { gamma = step; break; }
        step *= 0.5;
      }
    }
    if (gamma > 0.0) for (int64_t k = 0; k < nf; ++k) b[k] += gamma * q[k];
    if (st) { st[1] = gamma; st[2] = gq; st[3] = (double)pit; st[4] = trials; }
  }
  lin_free(&lin);
  free(grad); free(rhs); free(q); free(bt);
  return status;
}
