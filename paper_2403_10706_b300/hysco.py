"""Torch-facing binding of libhysco: one method per C-ABI entry point, same names.

Tensors are passed as raw device pointers together with the current CUDA stream; every
computation runs in libhysco's kernels.  PyTorch only provides device memory and streams.
"""
from __future__ import annotations

import ctypes as C

import torch

from . import _lib

_DTYPES = {torch.float32: _lib.F32, torch.bfloat16: _lib.BF16, torch.float16: _lib.F16}


def _stream(device):
    return C.c_void_p(torch.cuda.current_stream(device).cuda_stream)


class Hysco:
    """One problem geometry (image dims, spacing in mm, PE axis) with weights alpha, beta (Eq. 4)
    and the image element type.  Owns the library handle (device workspace)."""

    def __init__(self, dims, spacing, pe_dim, alpha=300.0, beta=1e-4, dtype=torch.float32,
                 device=None):
        self.lib = _lib.load()
        device = torch.device("cuda") if device is None else torch.device(device)
        if device.index is None:
            device = torch.device("cuda", torch.cuda.current_device())
        self.device = device
        if dtype not in _DTYPES:
            raise TypeError(f"unsupported image dtype {dtype}")
        self.dtype = dtype
        self.dims = tuple(int(x) for x in dims)
        self.spacing = tuple(float(x) for x in spacing)
        self.pe_dim = int(pe_dim)
        self.alpha, self.beta = float(alpha), float(beta)
        self._h = C.c_void_p()
        with torch.cuda.device(self.device):
            _lib.check(self.lib.hysco_create((C.c_int64 * 3)(*self.dims),
                                             (C.c_double * 3)(*self.spacing), self.pe_dim,
                                             self.alpha, self.beta, _DTYPES[dtype],
                                             C.byref(self._h)), "hysco_create")
        fd = (C.c_int64 * 3)()
        _lib.check(self.lib.hysco_field_dims(self._h, fd), "hysco_field_dims")
        self.field_dims = tuple(fd)

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            self.lib.hysco_destroy(h)
            self._h = None

    # -- argument checks (marshalling only) ---------------------------------------------------
    def _img(self, t, name):
        if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == self.dtype
                and tuple(t.shape) == self.dims and t.is_contiguous()):
            raise ValueError(f"{name}: expected contiguous {self.dtype} CUDA tensor {self.dims}")
        return C.c_void_p(t.data_ptr())

    def _fld(self, t, name, dtype=torch.float32):
        if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == dtype
                and tuple(t.shape) == self.field_dims and t.is_contiguous()):
            raise ValueError(f"{name}: expected contiguous {dtype} CUDA tensor {self.field_dims}")
        return C.c_void_p(t.data_ptr())

    def _new_fld(self, dtype=torch.float32):
        return torch.empty(self.field_dims, dtype=dtype, device=self.device)

    # -- entry points -------------------------------------------------------------------------
    def init_ot(self, Ip, Im, blur=True, eps=1e-3, out=None):
        out = self._new_fld() if out is None else out
        _lib.check(self.lib.hysco_init_ot(self._h, self._img(Ip, "Ip"), self._img(Im, "Im"),
                                          self._fld(out, "out"), int(blur), float(eps),
                                          _stream(self.device)), "hysco_init_ot")
        return out

    def eval(self, Ip, Im, b, grad=True, terms=None):
        """Returns (terms[J, D, S, P] float64 CUDA tensor, grad or None)."""
        terms = torch.empty(4, dtype=torch.float64, device=self.device) if terms is None else terms
        g = self._new_fld() if grad is True else (grad if isinstance(grad, torch.Tensor) else None)
        _lib.check(self.lib.hysco_eval(self._h, self._img(Ip, "Ip"), self._img(Im, "Im"),
                                       self._fld(b, "b"), C.c_void_p(terms.data_ptr()),
                                       None if g is None else self._fld(g, "grad"),
                                       _stream(self.device)), "hysco_eval")
        return terms, g

    def hessvec(self, v, out=None):
        out = self._new_fld() if out is None else out
        _lib.check(self.lib.hysco_hessvec(self._h, self._fld(v, "v"), self._fld(out, "Hv"),
                                          _stream(self.device)), "hysco_hessvec")
        return out

    def precond(self, r, kind=_lib.PC_JACOBI, out=None):
        out = self._new_fld() if out is None else out
        _lib.check(self.lib.hysco_precond(self._h, self._fld(r, "r"), self._fld(out, "z"),
                                          int(kind), _stream(self.device)), "hysco_precond")
        return out

    def pcg(self, rhs, precond=_lib.PC_JACOBI, max_iters=10, rtol=0.1, pcg_path=0, out=None):
        """q ~= H^{-1} rhs by PCG about the field of the last eval (rhs = -grad in a GN step)."""
        out = self._new_fld() if out is None else out
        _lib.check(self.lib.hysco_pcg(self._h, self._fld(rhs, "rhs"), self._fld(out, "q"),
                                      int(precond), int(max_iters), float(rtol), int(pcg_path),
                                      _stream(self.device)), "hysco_pcg")
        return out

    def correct(self, Ip, Im, b):
        Tp = torch.empty(self.dims, dtype=torch.float32, device=self.device)
        Tm = torch.empty_like(Tp)
        _lib.check(self.lib.hysco_correct(self._h, self._img(Ip, "Ip"), self._img(Im, "Im"),
                                          self._fld(b, "b"), C.c_void_p(Tp.data_ptr()),
                                          C.c_void_p(Tm.data_ptr()), _stream(self.device)),
                   "hysco_correct")
        return Tp, Tm

    def correct_mean(self, Ip, Im, b):
        """The corrected image 1/2 (Tp + Tm) (hysco_correct_mean)."""
        T = torch.empty(self.dims, dtype=torch.float32, device=self.device)
        _lib.check(self.lib.hysco_correct_mean(self._h, self._img(Ip, "Ip"), self._img(Im, "Im"),
                                               self._fld(b, "b"), C.c_void_p(T.data_ptr()),
                                               _stream(self.device)), "hysco_correct_mean")
        return T

    def correct_mean_adjoint(self, Ip, Im, b, gT, want=(True, True, True)):
        """Adjoint of correct_mean for the upstream sensitivity gT: (dIp, dIm, db), each None when
        not wanted."""
        dIp = torch.empty(self.dims, dtype=torch.float32, device=self.device) if want[0] else None
        dIm = torch.empty(self.dims, dtype=torch.float32, device=self.device) if want[1] else None
        db = self._new_fld() if want[2] else None
        p = lambda t: None if t is None else C.c_void_p(t.data_ptr())  # noqa: E731
        _lib.check(self.lib.hysco_correct_mean_adjoint(
            self._h, self._img(Ip, "Ip"), self._img(Im, "Im"), self._fld(b, "b"),
            self._img_f32(gT, "gT"), p(dIp), p(dIm), p(db), _stream(self.device)),
            "hysco_correct_mean_adjoint")
        return dIp, dIm, db

    def ls_correct(self, Ip, Im, b, lam=1e-6):
        """Least-squares corrected image at b and the number of skipped columns."""
        out = torch.empty(self.dims, dtype=torch.float32, device=self.device)
        nbad = torch.zeros(1, dtype=torch.int32, device=self.device)
        _lib.check(self.lib.hysco_ls_correct(self._h, self._img(Ip, "Ip"), self._img(Im, "Im"),
                                             self._fld(b, "b"), float(lam),
                                             C.c_void_p(out.data_ptr()),
                                             C.c_void_p(nbad.data_ptr()), _stream(self.device)),
                   "hysco_ls_correct")
        return out, nbad

    def _img_f32(self, t, name):
        if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float32
                and tuple(t.shape) == self.dims and t.is_contiguous()):
            raise ValueError(f"{name}: expected contiguous float32 CUDA tensor {self.dims}")
        return C.c_void_p(t.data_ptr())

    def correct_adjoint(self, Ip, Im, b, gTp=None, gTm=None, want=(True, True, True)):
        """Adjoint of correct() at b: (dIp, dIm, db) for sensitivities gTp, gTm of Tp, Tm
        (None = 0); an output is None when its `want` flag is False."""
        dIp = torch.empty(self.dims, dtype=torch.float32, device=self.device) if want[0] else None
        dIm = torch.empty(self.dims, dtype=torch.float32, device=self.device) if want[1] else None
        db = self._new_fld() if want[2] else None
        opt = lambda t, f, name: None if t is None else f(t, name)   # noqa: E731
        _lib.check(self.lib.hysco_correct_adjoint(
            self._h, self._img(Ip, "Ip"), self._img(Im, "Im"), self._fld(b, "b"),
            opt(gTp, self._img_f32, "gTp"), opt(gTm, self._img_f32, "gTm"),
            opt(dIp, self._img_f32, "dIp"), opt(dIm, self._img_f32, "dIm"),
            opt(db, self._fld, "db"), _stream(self.device)), "hysco_correct_adjoint")
        return dIp, dIm, db

    def image_grad(self, Ip, Im, b, gJ=1.0, want=(True, True)):
        """gJ * dJ/dIp and gJ * dJ/dIm at fixed b (float32, image shaped)."""
        dIp = torch.empty(self.dims, dtype=torch.float32, device=self.device) if want[0] else None
        dIm = torch.empty(self.dims, dtype=torch.float32, device=self.device) if want[1] else None
        _lib.check(self.lib.hysco_image_grad(
            self._h, self._img(Ip, "Ip"), self._img(Im, "Im"), self._fld(b, "b"), float(gJ),
            None if dIp is None else self._img_f32(dIp, "dIp"),
            None if dIm is None else self._img_f32(dIm, "dIm"), _stream(self.device)),
            "hysco_image_grad")
        return dIp, dIm

    def implicit_parts(self, Ip, Im, b, v):
        """(dIp, dIm, dtheta[2] float64) = -(d(v^T g)/dI+-, v^T dg/dalpha, v^T dg/dbeta) at b."""
        dIp = torch.empty(self.dims, dtype=torch.float32, device=self.device)
        dIm = torch.empty_like(dIp)
        dth = torch.empty(2, dtype=torch.float64, device=self.device)
        _lib.check(self.lib.hysco_implicit_parts(
            self._h, self._img(Ip, "Ip"), self._img(Im, "Im"), self._fld(b, "b"),
            self._fld(v, "v"), self._img_f32(dIp, "dIp"), self._img_f32(dIm, "dIm"),
            C.c_void_p(dth.data_ptr()), _stream(self.device)), "hysco_implicit_parts")
        return dIp, dIm, dth

    def solve_adjoint(self, Ip, Im, b, dLdb, max_iters=200, rtol=1e-6):
        """Implicit differentiation at a solution b: (v, dL/dIp, dL/dIm, dL/d(alpha, beta)) with
        H v = dLdb (the parts through b only)."""
        v = self._new_fld()
        dIp = torch.empty(self.dims, dtype=torch.float32, device=self.device)
        dIm = torch.empty_like(dIp)
        dth = torch.empty(2, dtype=torch.float64, device=self.device)
        _lib.check(self.lib.hysco_solve_adjoint(
            self._h, self._img(Ip, "Ip"), self._img(Im, "Im"), self._fld(b, "b"),
            self._fld(dLdb, "dLdb"), int(max_iters), float(rtol), self._fld(v, "v"),
            self._img_f32(dIp, "dIp"), self._img_f32(dIm, "dIm"), C.c_void_p(dth.data_ptr()),
            _stream(self.device)), "hysco_solve_adjoint")
        return v, dIp, dIm, dth

    def solve(self, Ip, Im, b=None, gn_iters=10, pcg_max_iters=10, ls_max_iters=10,
              precond=_lib.PC_JACOBI, init=None, ot_blur=True, pcg_rtol=0.1, armijo_c1=1e-4,
              ot_eps=1e-3, stats=True, pcg_path=0, graph=True):
        """GN-PCG solve.  init defaults to OT when b is None.  Returns (b, stats or None)."""
        if init is None:
            init = b is None
        b = self._new_fld() if b is None else b
        o = _lib.Opts(gn_iters, pcg_max_iters, ls_max_iters, int(precond), int(init),
                      int(ot_blur), pcg_rtol, armijo_c1, ot_eps, int(pcg_path), int(not graph))
        st = (torch.full((max(gn_iters, 1), _lib.NSTATS), float("nan"), dtype=torch.float64,
                         device=self.device) if stats else None)
        _lib.check(self.lib.hysco_solve(self._h, self._img(Ip, "Ip"), self._img(Im, "Im"),
                                        self._fld(b, "b"), C.byref(o),
                                        None if st is None else C.c_void_p(st.data_ptr()),
                                        _stream(self.device)), "hysco_solve")
        return b, (st[:gn_iters] if st is not None else None)

    def admm(self, Ip, Im, b=None, stats=True, **kw):
        """ADMM of Sec. 2.3.2 (hysco_admm).  Keyword options are the fields of hysco_admm_opts
        (defaults from hysco_default_admm_opts; init defaults to OT when b is None).  Returns
        (b, stats [admm_iters, ADMM_NSTATS] float64 or None)."""
        o = _lib.default_admm_opts()
        kw.setdefault("init", int(b is None))
        for k, v in kw.items():
            if not hasattr(o, k) or k == "pad_":
                raise TypeError(f"unknown ADMM option {k}")
            setattr(o, k, type(getattr(o, k))(v))
        b = self._new_fld() if b is None else b
        st = (torch.full((max(o.admm_iters, 1), _lib.ADMM_NSTATS), float("nan"),
                         dtype=torch.float64, device=self.device) if stats else None)
        _lib.check(self.lib.hysco_admm(self._h, self._img(Ip, "Ip"), self._img(Im, "Im"),
                                       self._fld(b, "b"), C.byref(o),
                                       None if st is None else C.c_void_p(st.data_ptr()),
                                       _stream(self.device)), "hysco_admm")
        return b, (st[:o.admm_iters] if st is not None else None)

    def block_pcg(self, Ip, Im, b, rho, rhs, max_iters=10, rtol=0.1, out=None):
        """BlockPCG on the ADMM b-subproblem linearised at b (hysco_block_pcg): returns
        (q, iterations summed over columns as a 1-element int32 CUDA tensor)."""
        out = self._new_fld() if out is None else out
        it = torch.zeros(1, dtype=torch.int32, device=self.device)
        _lib.check(self.lib.hysco_block_pcg(self._h, self._img(Ip, "Ip"), self._img(Im, "Im"),
                                            self._fld(b, "b"), float(rho), self._fld(rhs, "rhs"),
                                            self._fld(out, "q"), int(max_iters), float(rtol),
                                            C.c_void_p(it.data_ptr()), _stream(self.device)),
                   "hysco_block_pcg")
        return out, it

    def admm_zsolve(self, v, rho, out=None):
        """The ADMM z-update alone: rho (alpha H_G + rho I)^{-1} v (hysco_admm_zsolve)."""
        out = self._new_fld() if out is None else out
        _lib.check(self.lib.hysco_admm_zsolve(self._h, self._fld(v, "v"), float(rho),
                                              self._fld(out, "z"), _stream(self.device)),
                   "hysco_admm_zsolve")
        return out

    def set_zsolve_path(self, path):
        """The z-update's arithmetic: 0 tensor cores (TF32 split pairs), 1 FP32 CUDA cores."""
        _lib.check(self.lib.hysco_set_zsolve_path(self._h, int(path)), "hysco_set_zsolve_path")

    def zsolve_path(self):
        """The z-update path in use (0 tensor cores, 1 CUDA cores)."""
        rc = self.lib.hysco_zsolve_path(self._h)
        _lib.check(min(rc, 0), "hysco_zsolve_path")
        return rc

    def pcg_plan(self):
        """(cooperative grid, on-chip slots per thread, slots per thread, threads per block) of
        the persistent PCG."""
        out = (C.c_int32 * 4)()
        _lib.check(self.lib.hysco_pcg_plan(self._h, out), "hysco_pcg_plan")
        return tuple(out)

    def set_pcg_onchip(self, onchip):
        """Limit the persistent PCG's on-chip slots (-1: the plan's maximum)."""
        _lib.check(self.lib.hysco_set_pcg_onchip(self._h, int(onchip)), "hysco_set_pcg_onchip")

    def last_status(self):
        """Numerical status of the last eval / solve / init_ot: 0 ok, 1 infeasible (J = +inf),
        -4 NaN.  Synchronises the current stream; raises only on a CUDA error."""
        st = self.lib.hysco_last_status(self._h, _stream(self.device))
        if st in (_lib.ECUDA, _lib.EINVAL):
            _lib.check(st, "hysco_last_status")
        return st

    def cell_indices(self, b):
        cp = torch.empty(self.dims, dtype=torch.int32, device=self.device)
        cm = torch.empty_like(cp)
        _lib.check(self.lib.hysco_cell_indices(self._h, self._fld(b, "b"),
                                               C.c_void_p(cp.data_ptr()),
                                               C.c_void_p(cm.data_ptr()), _stream(self.device)),
                   "hysco_cell_indices")
        return cp, cm

    def ot_indices(self, Ip, Im, eps=1e-3):
        kp = self._new_fld(torch.int32)
        km = self._new_fld(torch.int32)
        _lib.check(self.lib.hysco_ot_indices(self._h, self._img(Ip, "Ip"), self._img(Im, "Im"),
                                             float(eps), C.c_void_p(kp.data_ptr()),
                                             C.c_void_p(km.data_ptr()), _stream(self.device)),
                   "hysco_ot_indices")
        return kp, km


class HyscoBatch:
    """Many Hysco handles (pairs of any sizes, PE axes and image dtypes, one device) solved
    together by hysco_batch_solve.  Keeps its handles alive; argument marshalling only."""

    def __init__(self, handles):
        self.handles = list(handles)
        if not self.handles:
            raise ValueError("empty batch")
        self.lib = _lib.load()
        self.device = self.handles[0].device
        n = len(self.handles)
        arr = (C.c_void_p * n)(*[h._h.value for h in self.handles])
        self._b = C.c_void_p()
        _lib.check(self.lib.hysco_batch_create(n, arr, C.byref(self._b)), "hysco_batch_create")

    def __del__(self):
        b = getattr(self, "_b", None)
        if b is not None and b.value:
            self.lib.hysco_batch_destroy(b)
            self._b = None

    def _ptrs(self, items, check):
        n = len(self.handles)
        if len(items) != n:
            raise ValueError(f"expected {n} tensors")
        return (C.c_void_p * n)(*[check(h, t).value for h, t in zip(self.handles, items)])

    def _opts(self, gn_iters, pcg_max_iters, ls_max_iters, init, ot_blur, pcg_rtol, armijo_c1,
              ot_eps, graph):
        return _lib.Opts(gn_iters, pcg_max_iters, ls_max_iters, _lib.PC_JACOBI, int(init),
                         int(ot_blur), pcg_rtol, armijo_c1, ot_eps, 0, int(not graph))

    def solve(self, Ips, Ims, bs=None, gn_iters=10, pcg_max_iters=10, ls_max_iters=10, init=None,
              ot_blur=True, pcg_rtol=0.1, armijo_c1=1e-4, ot_eps=1e-3, stats=True, graph=True):
        """Solve every pair; returns (fields, per-pair stats or None)."""
        if init is None:
            init = bs is None
        bs = [h._new_fld() for h in self.handles] if bs is None else list(bs)
        o = self._opts(gn_iters, pcg_max_iters, ls_max_iters, init, ot_blur, pcg_rtol, armijo_c1,
                       ot_eps, graph)
        sts = ([torch.full((max(gn_iters, 1), _lib.NSTATS), float("nan"), dtype=torch.float64,
                           device=self.device) for _ in self.handles] if stats else None)
        sp = None if sts is None else (C.c_void_p * len(sts))(*[t.data_ptr() for t in sts])
        _lib.check(self.lib.hysco_batch_solve(
            self._b, self._ptrs(Ips, lambda h, t: h._img(t, "Ip")),
            self._ptrs(Ims, lambda h, t: h._img(t, "Im")),
            self._ptrs(bs, lambda h, t: h._fld(t, "b")), C.byref(o), sp, _stream(self.device)),
            "hysco_batch_solve")
        return bs, (None if sts is None else [t[:gn_iters] for t in sts])

    def tune(self, Ips, Ims, gn_iters=10, pcg_max_iters=10, ls_max_iters=10, ot_blur=True,
             pcg_rtol=0.1, armijo_c1=1e-4, ot_eps=1e-3):
        """Pick the schedule by timing short trial solves (synchronises); returns schedule()."""
        o = self._opts(gn_iters, pcg_max_iters, ls_max_iters, True, ot_blur, pcg_rtol, armijo_c1,
                       ot_eps, True)
        _lib.check(self.lib.hysco_batch_tune(
            self._b, self._ptrs(Ips, lambda h, t: h._img(t, "Ip")),
            self._ptrs(Ims, lambda h, t: h._img(t, "Im")), C.byref(o), _stream(self.device)),
            "hysco_batch_tune")
        return self.schedule()

    def schedule(self):
        """(branches, PCG policy, shared PCG grid blocks) in use; policy 0 / 1: one PCG launch
        shared by all pairs (blocks by field size, >= 1 / >= 2 per pair), 2: each pair's
        persistent PCG in turn, 3 / 4 / 5: waves of pairs whose PCGs share one launch per GN step
        (vectors packed to 1, 1.25, 1.5 times the on-chip capacity), 6 / 7 / 8: the same waves,
        each wave's whole GN loops in one persistent launch."""
        out = (C.c_int32 * 3)()
        _lib.check(self.lib.hysco_batch_schedule(self._b, out), "hysco_batch_schedule")
        return tuple(out)

    def set_schedule(self, branches, policy):
        _lib.check(self.lib.hysco_batch_set_schedule(self._b, int(branches), int(policy)),
                   "hysco_batch_set_schedule")
