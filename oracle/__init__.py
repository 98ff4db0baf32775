"""Double-precision CPU oracle for the HySCO hot path (PyHySCO, arXiv 2403.10706).

TEST INFRASTRUCTURE ONLY: imported by tests/, by the package smoke check and by the
benchmark's CPU-baseline leg, never by the product path.  It is a ctypes wrapper around
oracle/hysco_oracle.c, which shares no code with the CUDA library.

All arrays are numpy, C-contiguous.  Images are float32 (the dtype the GPU path receives);
fields, gradients and vectors are float64.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "hysco_oracle.c")
_LIB = os.path.join(_HERE, "libhysco_oracle.so")

ST_FIELDS = ["J", "D", "S", "P", "gnorm", "gq", "gamma", "pcg_iters", "pcg_relres", "ls_trials"]
# per ADMM iteration (Problem.admm)
ADMM_FIELDS = ["J", "F_c", "rho", "r_primal", "s_dual", "rel_db", "rel_dz", "rel_du",
               "block_pcg_iters", "gamma"]


def build(force: bool = False) -> str:
    """Compile the oracle with plain gcc (IEEE semantics: no fast-math, no FP contraction)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        subprocess.check_call(["gcc", "-std=c11", "-O2", "-ffp-contract=off", "-fno-fast-math",
                               "-fopenmp", "-fPIC", "-shared", "-o", _LIB, _SRC, "-lm"])
    return _LIB


def set_threads(n: int) -> None:
    """OpenMP threads of the oracle's loops (the results do not depend on it)."""
    lib().orc_set_threads(int(n))


def max_threads() -> int:
    return int(lib().orc_max_threads())


class Geom(C.Structure):
    _fields_ = [("d", C.c_int64 * 3), ("h", C.c_double * 3), ("p", C.c_int32),
                ("pad_", C.c_int32), ("alpha", C.c_double), ("beta", C.c_double)]


class Opts(C.Structure):
    _fields_ = [("gn_iters", C.c_int32), ("pcg_max_iters", C.c_int32),
                ("ls_max_iters", C.c_int32), ("precond", C.c_int32), ("init", C.c_int32),
                ("ot_blur", C.c_int32), ("contract", C.c_int32), ("pad_", C.c_int32),
                ("pcg_rtol", C.c_double), ("armijo_c1", C.c_double), ("ot_eps", C.c_double)]


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(build())
        P = C.c_void_p
        _lib.orc_eval.restype = C.c_int64
        _lib.orc_eval.argtypes = [P, P, P, P, C.c_int, P, P, P, P, P, P]
        _lib.orc_hessvec.argtypes = [P, P, P, P, C.c_int, P, P]
        _lib.orc_hessdiag.argtypes = [P, P, P, P, C.c_int, P]
        _lib.orc_precond.argtypes = [P, P, P, P, C.c_int, C.c_int, P, P]
        _lib.orc_column_block.argtypes = [P, P, P, P, C.c_int, C.c_int64, P, P]
        _lib.orc_column_blocks.argtypes = [P, P, P, P, C.c_int, P, P]
        _lib.orc_apply_laplacian.argtypes = [P, P, P]
        _lib.orc_ot_init.argtypes = [P, P, P, C.c_double, C.c_int, C.c_int, P, P, P]
        _lib.orc_blur.argtypes = [P, P]
        _lib.orc_solve.argtypes = [P, P, P, P, P, P]
        _lib.orc_set_threads.argtypes = [C.c_int]
        _lib.orc_max_threads.restype = C.c_int
        _lib.orc_pcg.argtypes = [P, P, P, P, C.c_int, C.c_int, P, C.c_int, C.c_double, P, P]
        _lib.orc_phi.argtypes = [C.c_double, P, P, P]
        _lib.orc_correct_adjoint.argtypes = [P, P, P, P, C.c_int, P, P, P, P, P]
        _lib.orc_image_grad.restype = C.c_int64
        _lib.orc_image_grad.argtypes = [P, P, P, P, C.c_int, P, P]
        _lib.orc_theta_dots.argtypes = [P, P, P, P, C.c_int, P, P]
        _lib.orc_mixed_image_adjoint.argtypes = [P, P, P, P, C.c_int, P, P, P]
        _lib.orc_solve_adjoint.argtypes = [P, P, P, P, C.c_int, P, C.c_int, C.c_double, P, P, P,
                                           P]
        _lib.orc_ls_correct.restype = C.c_int64
        _lib.orc_ls_correct.argtypes = [P, P, P, P, C.c_double, P]
        _lib.orc_pushforward_matrix.argtypes = [P, C.c_int64, C.c_double, P]
        _lib.orc_feasible_start.restype = C.c_double
        _lib.orc_feasible_start.argtypes = [P, P]
        _lib.orc_admm_eval.restype = C.c_int64
        _lib.orc_admm_eval.argtypes = [P, P, P, P, C.c_int, C.c_double, P, P, P]
        _lib.orc_block_pcg.restype = C.c_int64
        _lib.orc_block_pcg.argtypes = [P, P, P, P, C.c_int, C.c_double, P, C.c_int, C.c_double,
                                       P]
        _lib.orc_admm_column_block.argtypes = [P, P, P, P, C.c_int, C.c_double, C.c_int64, P, P]
        _lib.orc_admm_bupdate.argtypes = [P, P, P, C.c_int, C.c_double, P, C.c_int, C.c_int,
                                          C.c_double, C.c_int, C.c_double, P, P]
    return _lib


def _p(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def _f32(a):
    return np.ascontiguousarray(a, dtype=np.float32)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def field_dims(dims, p):
    fd = list(dims)
    fd[p] += 1
    return tuple(fd)


def _rel(d, ref):
    """||d|| / ||ref|| with 0/0 = 0 and x/0 = inf (relative change of an ADMM iterate)."""
    nd, nr = np.linalg.norm(d.ravel()), np.linalg.norm(ref.ravel())
    if nr > 0.0:
        return nd / nr
    return 0.0 if nd == 0.0 else np.inf


class AdmmMixin:
    """ADMM of Sec. 2.3.2 (split F(b) = D + alpha S3 + beta P, G(z) = alpha (S1 + S2), constraint
    b = z, scaled multiplier u), on top of the b-update in hysco_oracle.c."""

    def inplane_axes(self):
        return [a for a in range(3) if a != self.pe_dim]

    def admm_eval(self, Ip, Im, b, rho, c, contract=True, grad=True):
        """F_c(b) = D + alpha S3 + beta P + rho vol/2 ||b - c||^2: dict(F_c, D, S3, P, prox,
        infeasible, grad?)."""
        terms = np.zeros(5)
        g = np.zeros(self.fdims) if grad else None
        bad = lib().orc_admm_eval(C.byref(self.g), _p(_f32(Ip)), _p(_f32(Im)), _p(_f64(b)),
                                  int(contract), float(rho), _p(_f64(c)), _p(terms), _p(g))
        out = dict(F_c=terms[0], D=terms[1], S3=terms[2], P=terms[3], prox=terms[4],
                   infeasible=int(bad))
        if grad:
            out["grad"] = g
        return out

    def admm_column_block(self, Ip, Im, b, rho, col, contract=True):
        m = self.dims[self.pe_dim]
        dia, off = np.zeros(m + 1), np.zeros(m)
        lib().orc_admm_column_block(C.byref(self.g), _p(_f32(Ip)), _p(_f32(Im)), _p(_f64(b)),
                                    int(contract), float(rho), int(col), _p(dia), _p(off))
        return dia, off

    def block_pcg(self, Ip, Im, b, rho, rhs, max_it=10, rtol=0.1, contract=True):
        """BlockPCG on the b-subproblem's GN system about b: (q, iterations summed over
        columns)."""
        q = np.zeros(self.fdims)
        it = lib().orc_block_pcg(C.byref(self.g), _p(_f32(Ip)), _p(_f32(Im)), _p(_f64(b)),
                                 int(contract), float(rho), _p(_f64(rhs)), int(max_it),
                                 float(rtol), _p(q))
        return q, int(it)

    def admm_bupdate(self, Ip, Im, b, rho, c, gn_iters=1, pcg_max_iters=10, pcg_rtol=0.1,
                     ls_max_iters=10, armijo_c1=1e-4, contract=True):
        """The b-update: returns (b_new, status, stats[gn_iters, 5])."""
        bb = _f64(b).copy()
        st = np.zeros((max(gn_iters, 1), 5))
        rc = lib().orc_admm_bupdate(C.byref(self.g), _p(_f32(Ip)), _p(_f32(Im)), int(contract),
                                    float(rho), _p(_f64(c)), int(gn_iters), int(pcg_max_iters),
                                    float(pcg_rtol), int(ls_max_iters), float(armijo_c1),
                                    _p(bb), _p(st))
        return bb, rc, st[:gn_iters]

    def admm_z_solve(self, rhs, rho):
        """The z-update of Sec. 2.3.2: (alpha H_G + rho I) z = rhs, H_G the Hessian of
        S1 + S2 with periodic ends (block circulant with circulant blocks per PE plane), solved
        by the 2D DFT over the in-plane axes: the eigenvalue of frequency (j0, j1) is
        rho + alpha sum_a (h_p / h_a)^2 (2 - 2 cos(2 pi j_a / n_a))."""
        axes = self.inplane_axes()
        hp = self.spacing[self.pe_dim]
        lam = np.full(self.fdims, float(rho))
        for a in axes:
            n = self.fdims[a]
            mu = 2.0 - 2.0 * np.cos(2.0 * np.pi * np.arange(n) / n)
            shape = [1, 1, 1]
            shape[a] = n
            lam = lam + self.g.alpha * (hp / self.spacing[a]) ** 2 * mu.reshape(shape)
        Z = np.fft.fftn(_f64(rhs), axes=axes) / lam
        return np.real(np.fft.ifftn(Z, axes=axes))

    def admm(self, Ip, Im, b=None, admm_iters=20, gn_iters=2, pcg_max_iters=10, pcg_rtol=0.1,
             ls_max_iters=10, armijo_c1=1e-4, rho0=None, tol=1e-3, mu=10.0, tau=2.0,
             init=True, ot_blur=True, ot_eps=1e-3, contract=False):
        """ADMM of Sec. 2.3.2.  Start: b from OT (feasible-start rule, as the GN solve) or the
        given b, z = b, u = 0, rho = rho0 (default alpha).  Iteration k:
          c = z - u;  b <- gn_iters GN steps on F_c (BlockPCG directions, Armijo on F_c);
          z <- (alpha H_G + rho I)^{-1} rho (b + u);  u <- u + b - z;
          r = ||b - z||, s = rho ||z - z_prev||; rho <- tau rho, u <- u / tau when r > mu s,
          rho <- rho / tau, u <- u tau when s > mu r (Boyd et al. 2011, Sec. 3.4.1);
          stop after the iteration in which the relative changes of b, z and u are all < tol.
        Returns (b, z, u, status, stats[admm_iters, len(ADMM_FIELDS)]), rows after the stop NaN."""
        if init:
            b = self.ot_init(Ip, Im, eps=ot_eps, contract=contract, blur=ot_blur)
            b, _ = self.feasible_start(b)
        else:
            b = _f64(b).copy()
        z, u = b.copy(), np.zeros(self.fdims)
        rho = float(self.g.alpha if rho0 is None else rho0)
        stats = np.full((max(admm_iters, 1), len(ADMM_FIELDS)), np.nan)
        status = 0
        for k in range(admm_iters):
            c = z - u
            b_prev, z_prev, u_prev = b, z, u
            b, status, bst = self.admm_bupdate(Ip, Im, b, rho, c, gn_iters, pcg_max_iters,
                                               pcg_rtol, ls_max_iters, armijo_c1, contract)
            if status != 0:
                break
            z = self.admm_z_solve(rho * (b + u), rho)
            u = u + b - z
            r = np.linalg.norm((b - z).ravel())
            s = rho * np.linalg.norm((z - z_prev).ravel())
            rel_db, rel_dz, rel_du = _rel(b - b_prev, b_prev), _rel(z - z_prev, z_prev), \
                _rel(u - u_prev, u_prev)
            Fc = self.admm_eval(Ip, Im, b, rho, c, contract=contract, grad=False)["F_c"]
            J = self.eval(Ip, Im, b, contract=contract, grad=False)["J"]
            stats[k] = [J, Fc, rho, r, s, rel_db, rel_dz, rel_du, bst[:, 3].sum(), bst[-1, 1]]
            if r > mu * s:
                rho, u = rho * tau, u / tau
            elif s > mu * r:
                rho, u = rho / tau, u * tau
            if rel_db < tol and rel_dz < tol and rel_du < tol:
                break
        return b, z, u, status, stats[:admm_iters]


class Problem(AdmmMixin):
    """Geometry + weights of one correction problem: image dims, spacing (mm), PE axis,
    alpha (smoothness) and beta (barrier) of Eq. 4."""

    def __init__(self, dims, spacing, pe_dim, alpha, beta):
        self.dims = tuple(int(x) for x in dims)
        self.spacing = tuple(float(x) for x in spacing)
        self.pe_dim = int(pe_dim)
        self.fdims = field_dims(self.dims, self.pe_dim)
        self.g = Geom((C.c_int64 * 3)(*self.dims), (C.c_double * 3)(*self.spacing),
                      self.pe_dim, 0, float(alpha), float(beta))

    def eval(self, Ip, Im, b, contract=True, grad=True, corrected=False, cells=False):
        """Returns dict(J, D, S, P, infeasible, grad?, Tp?, Tm?, cell_p?, cell_m?)."""
        Ip, Im, b = _f32(Ip), _f32(Im), _f64(b)
        terms = np.zeros(4)
        g = np.zeros(self.fdims) if grad else None
        Tp = np.zeros(self.dims) if corrected else None
        Tm = np.zeros(self.dims) if corrected else None
        cp = np.zeros(self.dims, np.int32) if cells else None
        cm = np.zeros(self.dims, np.int32) if cells else None
        bad = lib().orc_eval(C.byref(self.g), _p(Ip), _p(Im), _p(b), int(contract), _p(terms),
                             _p(g), _p(Tp), _p(Tm), _p(cp), _p(cm))
        out = dict(J=terms[0], D=terms[1], S=terms[2], P=terms[3], infeasible=int(bad))
        if grad:
            out["grad"] = g
        if corrected:
            out["Tp"], out["Tm"] = Tp, Tm
        if cells:
            out["cell_p"], out["cell_m"] = cp, cm
        return out

    def correct_adjoint(self, Ip, Im, b, gTp=None, gTm=None, contract=True):
        """Adjoint of the corrected images T+, T- at b for upstream sensitivities gTp, gTm
        (None = 0): returns (dIp, dIm, db)."""
        Ip, Im, b = _f32(Ip), _f32(Im), _f64(b)
        gTp = None if gTp is None else _f64(gTp)
        gTm = None if gTm is None else _f64(gTm)
        dIp, dIm, db = np.zeros(self.dims), np.zeros(self.dims), np.zeros(self.fdims)
        lib().orc_correct_adjoint(C.byref(self.g), _p(Ip), _p(Im), _p(b), int(contract),
                                  _p(gTp), _p(gTm), _p(dIp), _p(dIm), _p(db))
        return dIp, dIm, db

    def image_grad(self, Ip, Im, b, contract=True):
        """dJ/dI+ and dJ/dI- at fixed b."""
        Ip, Im, b = _f32(Ip), _f32(Im), _f64(b)
        dIp, dIm = np.zeros(self.dims), np.zeros(self.dims)
        lib().orc_image_grad(C.byref(self.g), _p(Ip), _p(Im), _p(b), int(contract), _p(dIp),
                             _p(dIm))
        return dIp, dIm

    def theta_dots(self, Ip, Im, b, v, contract=True):
        """(v^T dg/dalpha, v^T dg/dbeta) at b, g the gradient of J."""
        out = np.zeros(2)
        lib().orc_theta_dots(C.byref(self.g), _p(_f32(Ip)), _p(_f32(Im)), _p(_f64(b)),
                             int(contract), _p(_f64(v)), _p(out))
        return out[0], out[1]

    def mixed_image_adjoint(self, Ip, Im, b, v, contract=True):
        """(d(v^T g)/dI+, d(v^T g)/dI-) at b, v fixed."""
        dIp, dIm = np.zeros(self.dims), np.zeros(self.dims)
        lib().orc_mixed_image_adjoint(C.byref(self.g), _p(_f32(Ip)), _p(_f32(Im)), _p(_f64(b)),
                                      int(contract), _p(_f64(v)), _p(dIp), _p(dIm))
        return dIp, dIm

    def solve_adjoint(self, Ip, Im, b, dLdb, max_it=200, rtol=1e-10, contract=True):
        """Implicit differentiation at a solution b: returns (v, dL/dI+, dL/dI-, dL/dalpha,
        dL/dbeta, PCG iterations) with H v = dL/db."""
        v = np.zeros(self.fdims)
        dIp, dIm, dth = np.zeros(self.dims), np.zeros(self.dims), np.zeros(2)
        it = lib().orc_solve_adjoint(C.byref(self.g), _p(_f32(Ip)), _p(_f32(Im)), _p(_f64(b)),
                                     int(contract), _p(_f64(dLdb)), int(max_it), float(rtol),
                                     _p(v), _p(dIp), _p(dIm), _p(dth))
        return v, dIp, dIm, dth[0], dth[1], it

    def ls_correct(self, Ip, Im, b, lam=1e-8):
        """Least-squares corrected image at b (image shaped) and the count of skipped columns."""
        out = np.zeros(self.dims)
        bad = lib().orc_ls_correct(C.byref(self.g), _p(_f32(Ip)), _p(_f32(Im)), _p(_f64(b)),
                                   float(lam), _p(out))
        return out, int(bad)

    def feasible_start(self, b):
        """The solve's start rule for an OT field: returns (b scaled by 2^-k, 2^-k) with the
        smallest k >= 0 that brings max |delta| below 1."""
        bb = _f64(b).copy()
        f = lib().orc_feasible_start(C.byref(self.g), _p(bb))
        return bb, f

    def hessvec(self, Ip, Im, b, v, contract=True):
        Hv = np.zeros(self.fdims)
        lib().orc_hessvec(C.byref(self.g), _p(_f32(Ip)), _p(_f32(Im)), _p(_f64(b)),
                          int(contract), _p(_f64(v)), _p(Hv))
        return Hv

    def hessdiag(self, Ip, Im, b, contract=True):
        d = np.zeros(self.fdims)
        lib().orc_hessdiag(C.byref(self.g), _p(_f32(Ip)), _p(_f32(Im)), _p(_f64(b)),
                           int(contract), _p(d))
        return d

    def precond(self, Ip, Im, b, r, kind, contract=True):
        """z = M^{-1} r; kind 0 = Jacobi, 1 = per-column block."""
        z = np.zeros(self.fdims)
        lib().orc_precond(C.byref(self.g), _p(_f32(Ip)), _p(_f32(Im)), _p(_f64(b)),
                          int(contract), int(kind), _p(_f64(r)), _p(z))
        return z

    def column_block(self, Ip, Im, b, col, contract=True):
        m = self.dims[self.pe_dim]
        dia, off = np.zeros(m + 1), np.zeros(m)
        lib().orc_column_block(C.byref(self.g), _p(_f32(Ip)), _p(_f32(Im)), _p(_f64(b)),
                               int(contract), int(col), _p(dia), _p(off))
        return dia, off

    def column_blocks(self, Ip, Im, b, contract=True):
        """(dia, off) field shaped: the tridiagonal diagonal block of every PE column."""
        dia, off = np.zeros(self.fdims), np.zeros(self.fdims)
        lib().orc_column_blocks(C.byref(self.g), _p(_f32(Ip)), _p(_f32(Im)), _p(_f64(b)),
                                int(contract), _p(dia), _p(off))
        return dia, off

    def laplacian(self, x):
        y = np.zeros(self.fdims)
        lib().orc_apply_laplacian(C.byref(self.g), _p(_f64(x)), _p(y))
        return y

    def ot_init(self, Ip, Im, eps=1e-3, contract=True, blur=True, indices=False):
        b0 = np.zeros(self.fdims)
        kp = np.zeros(self.fdims, np.int32) if indices else None
        km = np.zeros(self.fdims, np.int32) if indices else None
        lib().orc_ot_init(C.byref(self.g), _p(_f32(Ip)), _p(_f32(Im)), float(eps),
                          int(contract), int(blur), _p(b0), _p(kp), _p(km))
        return (b0, kp, km) if indices else b0

    def blur(self, b):
        b = _f64(b).copy()
        lib().orc_blur(C.byref(self.g), _p(b))
        return b

    def pcg(self, Ip, Im, b, rhs, precond=0, max_it=10, rtol=0.1, contract=True):
        q = np.zeros(self.fdims)
        rel = np.zeros(1)
        it = lib().orc_pcg(C.byref(self.g), _p(_f32(Ip)), _p(_f32(Im)), _p(_f64(b)),
                           int(contract), int(precond), _p(_f64(rhs)), int(max_it), float(rtol),
                           _p(q), _p(rel))
        return q, it, rel[0]

    def solve(self, Ip, Im, b=None, gn_iters=10, pcg_max_iters=10, ls_max_iters=10, precond=0,
              init=True, ot_blur=True, contract=False, pcg_rtol=0.1, armijo_c1=1e-4,
              ot_eps=1e-3):
        """GN-PCG solve; returns (b, status, stats[gn_iters, len(ST_FIELDS)])."""
        o = Opts(gn_iters, pcg_max_iters, ls_max_iters, precond, int(init), int(ot_blur),
                 int(contract), 0, pcg_rtol, armijo_c1, ot_eps)
        bb = np.zeros(self.fdims) if b is None else _f64(b).copy()
        stats = np.zeros((max(gn_iters, 1), len(ST_FIELDS)))
        st = lib().orc_solve(C.byref(self.g), _p(_f32(Ip)), _p(_f32(Im)), C.byref(o), _p(bb),
                             _p(stats))
        return bb, st, stats[:gn_iters]


def phi(z):
    f, df, d2f = C.c_double(), C.c_double(), C.c_double()
    lib().orc_phi(float(z), C.byref(f), C.byref(df), C.byref(d2f))
    return f.value, df.value, d2f.value


def pushforward_matrix(bcol, sign):
    """Dense m x m push-forward matrix of one column (field values bcol, m + 1 nodes)."""
    bcol = _f64(bcol)
    m = bcol.size - 1
    P = np.zeros((m, m))
    lib().orc_pushforward_matrix(_p(bcol), m, float(sign), _p(P))
    return P
