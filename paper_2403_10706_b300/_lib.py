"""ctypes declarations of libhysco's C ABI (include/hysco.h).

Argument marshalling only.  Loading fails loudly when libhysco.so has not been built: there is
no CPU or Python fallback for any step of the path.
"""
from __future__ import annotations

import ctypes as C
import os
import re

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libhysco.so")
HEADER = os.path.join(os.path.dirname(HERE), "include", "hysco.h")

OK, INFEASIBLE, EINVAL, ECUDA, ENOMEM, ENONFINITE, ENOTREADY, ETIMEOUT = 0, 1, -1, -2, -3, -4, -5, -6
F32, BF16, F16 = 0, 1, 2
PC_JACOBI, PC_COLUMN = 0, 1
NSTATS = 10
STATS_FIELDS = ["J", "D", "S", "P", "gnorm", "gq", "gamma", "pcg_iters", "pcg_relres",
                "ls_trials"]


class Opts(C.Structure):
    _fields_ = [("gn_iters", C.c_int32), ("pcg_max_iters", C.c_int32),
                ("ls_max_iters", C.c_int32), ("precond", C.c_int32), ("init", C.c_int32),
                ("ot_blur", C.c_int32), ("pcg_rtol", C.c_double), ("armijo_c1", C.c_double),
                ("ot_eps", C.c_double), ("pcg_path", C.c_int32), ("no_graph", C.c_int32)]


class AdmmOpts(C.Structure):
    _fields_ = [("admm_iters", C.c_int32), ("gn_iters", C.c_int32),
                ("pcg_max_iters", C.c_int32), ("ls_max_iters", C.c_int32), ("init", C.c_int32),
                ("ot_blur", C.c_int32), ("no_graph", C.c_int32), ("pad_", C.c_int32),
                ("pcg_rtol", C.c_double), ("armijo_c1", C.c_double), ("ot_eps", C.c_double),
                ("rho0", C.c_double), ("tol", C.c_double), ("mu", C.c_double),
                ("tau", C.c_double)]


ADMM_NSTATS = 10


class HyscoError(RuntimeError):
    def __init__(self, status, what):
        super().__init__(f"{what}: {strerror(status)} (status {status})")
        self.status = status


_lib = None


def load():
    """The loaded libhysco (ctypes.CDLL) with argument types declared."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"libhysco.so is not built ({LIB_PATH}); run "
                          "`python -m paper_2403_10706_b300.build` or __graft_entry__.build()")
    lib = C.CDLL(LIB_PATH)
    P, I, D, I64P = C.c_void_p, C.c_int, C.c_double, C.POINTER(C.c_int64)
    sig = {
        "hysco_version": (C.c_char_p, []),
        "hysco_strerror": (C.c_char_p, [I]),
        "hysco_default_opts": (None, [C.POINTER(Opts)]),
        "hysco_default_admm_opts": (None, [C.POINTER(AdmmOpts)]),
        "hysco_admm": (I, [P, P, P, P, C.POINTER(AdmmOpts), P, P]),
        "hysco_block_pcg": (I, [P, P, P, P, D, P, P, I, D, P, P]),
        "hysco_admm_zsolve": (I, [P, P, D, P, P]),
        "hysco_create": (I, [I64P, C.POINTER(C.c_double), I, D, D, I, C.POINTER(P)]),
        "hysco_destroy": (None, [P]),
        "hysco_field_dims": (I, [P, I64P]),
        "hysco_init_ot": (I, [P, P, P, P, I, D, P]),
        "hysco_eval": (I, [P, P, P, P, P, P, P]),
        "hysco_hessvec": (I, [P, P, P, P]),
        "hysco_precond": (I, [P, P, P, I, P]),
        "hysco_pcg": (I, [P, P, P, I, I, D, I, P]),
        "hysco_correct": (I, [P, P, P, P, P, P, P]),
        "hysco_ls_correct": (I, [P, P, P, P, D, P, P, P]),
        "hysco_correct_adjoint": (I, [P, P, P, P, P, P, P, P, P, P]),
        "hysco_correct_mean": (I, [P, P, P, P, P, P]),
        "hysco_correct_mean_adjoint": (I, [P, P, P, P, P, P, P, P, P]),
        "hysco_image_grad": (I, [P, P, P, P, D, P, P, P]),
        "hysco_implicit_parts": (I, [P, P, P, P, P, P, P, P, P]),
        "hysco_solve_adjoint": (I, [P, P, P, P, P, I, D, P, P, P, P, P]),
        "hysco_solve": (I, [P, P, P, P, C.POINTER(Opts), P, P]),
        "hysco_last_status": (I, [P, P]),
        "hysco_cell_indices": (I, [P, P, P, P, P]),
        "hysco_ot_indices": (I, [P, P, P, D, P, P, P]),
        "hysco_eval_static": (I, [I64P, C.POINTER(C.c_double), I, D, D, I, P, P, P, P, P, P]),
        "hysco_batch_create": (I, [I, P, C.POINTER(P)]),
        "hysco_batch_destroy": (None, [P]),
        "hysco_batch_solve": (I, [P, P, P, P, C.POINTER(Opts), P, P]),
        "hysco_batch_tune": (I, [P, P, P, C.POINTER(Opts), P]),
        "hysco_batch_schedule": (I, [P, C.POINTER(C.c_int32)]),
        "hysco_batch_set_schedule": (I, [P, I, I]),
        "hysco_selftest_barrier": (I, [I, I, C.c_int64, P]),
        "hysco_pcg_plan": (I, [P, C.POINTER(C.c_int32)]),
        "hysco_set_pcg_onchip": (I, [P, I]),
        "hysco_set_zsolve_path": (I, [P, I]),
        "hysco_zsolve_path": (I, [P]),
        "hysco_selftest_zsolve": (I, [P, C.c_int64, P]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def strerror(status: int) -> str:
    return load().hysco_strerror(int(status)).decode()


def check(status: int, what: str) -> int:
    if status < 0:
        raise HyscoError(status, what)
    return status


def declared_functions(header: str = HEADER):
    """Names of the functions include/hysco.h declares."""
    text = open(header).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(hysco_[a-z_]+)\s*\(", text)))


def default_opts() -> Opts:
    o = Opts()
    load().hysco_default_opts(C.byref(o))
    return o


def default_admm_opts() -> AdmmOpts:
    o = AdmmOpts()
    load().hysco_default_admm_opts(C.byref(o))
    return o
