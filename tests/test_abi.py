"""Host-side checks of the C ABI that need no GPU: the library builds and loads, exports every
function include/hysco.h declares, and rejects bad arguments before touching the device."""
import ctypes as C
import os
import subprocess

import pytest

from paper_2403_10706_b300 import _lib, build


@pytest.fixture(scope="module")
def lib():
    build.build()
    return _lib.load()


def test_exports_every_declared_function(lib):
    declared = _lib.declared_functions()
    assert len(declared) >= 14
    out = subprocess.run(["nm", "-D", "--defined-only", _lib.LIB_PATH], capture_output=True,
                         text=True, check=True).stdout
    exported = {line.split()[-1] for line in out.splitlines() if " T " in line}
    missing = [f for f in declared if f not in exported]
    assert not missing, missing
    for f in declared:
        assert hasattr(lib, f)


def test_built_for_sm_103a_only():
    assert "arch=compute_103a,code=sm_103a" in " ".join(build.ARCH)


def test_strerror_and_version(lib):
    assert b"sm_103a" in lib.hysco_version()
    for st in (_lib.OK, _lib.INFEASIBLE, _lib.EINVAL, _lib.ECUDA, _lib.ENOMEM, _lib.ENONFINITE,
               _lib.ENOTREADY):
        assert _lib.strerror(st) != "unknown status"
    assert _lib.strerror(12345) == "unknown status"


def test_default_opts_are_the_papers(lib):
    o = _lib.default_opts()
    assert (o.pcg_max_iters, o.pcg_rtol, o.precond, o.init, o.ot_blur) == (10, 0.1, 0, 1, 1)


@pytest.mark.parametrize("dims,spacing,pe,alpha,beta,dtype", [
    ((4, 5, 6), (1, 1, 1), 3, 1.0, 1.0, 0),        # pe_dim out of range
    ((4, 5, 6), (1, 1, 1), -1, 1.0, 1.0, 0),
    ((4, 0, 6), (1, 1, 1), 1, 1.0, 1.0, 0),        # empty volume
    ((4, 1, 6), (1, 1, 1), 1, 1.0, 1.0, 0),        # fewer than 2 cells along PE
    ((4, 5, 6), (1, 0, 1), 1, 1.0, 1.0, 0),        # zero spacing
    ((4, 5, 6), (1, float("nan"), 1), 1, 1.0, 1.0, 0),
    ((4, 5, 6), (1, 1, 1), 1, -1.0, 1.0, 0),       # negative weight
    ((4, 5, 6), (1, 1, 1), 1, 1.0, float("inf"), 0),
    ((4, 5, 6), (1, 1, 1), 1, 1.0, 1.0, 7),        # unknown image dtype
    ((1 << 12, 1 << 12, 1 << 8), (1, 1, 1), 2, 1.0, 1.0, 0),   # more than 2^31 field nodes
])
def test_create_rejects_bad_arguments_before_any_device_call(lib, dims, spacing, pe, alpha, beta,
                                                             dtype):
    h = C.c_void_p(123)
    rc = lib.hysco_create((C.c_int64 * 3)(*dims), (C.c_double * 3)(*spacing), pe, alpha, beta,
                          dtype, C.byref(h))
    assert rc == _lib.EINVAL
    assert h.value is None


def test_null_handle_calls_are_rejected(lib):
    f = (C.c_float * 4)()
    assert lib.hysco_eval(None, f, f, f, f, None, None) == _lib.EINVAL
    assert lib.hysco_hessvec(None, f, f, None) == _lib.EINVAL
    assert lib.hysco_solve(None, f, f, f, None, None, None) == _lib.EINVAL
    assert lib.hysco_last_status(None, None) == _lib.EINVAL
    assert lib.hysco_field_dims(None, (C.c_int64 * 3)()) == _lib.EINVAL
    lib.hysco_destroy(None)


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    monkeypatch.setattr(_lib, "LIB_PATH", str(tmp_path / "absent.so"))
    monkeypatch.setattr(_lib, "_lib", None)
    with pytest.raises(ImportError):
        _lib.load()


def test_adjoint_and_batch_entry_points_reject_null_arguments(lib):
    """Host-side validation returns before any device work (no GPU needed)."""
    f = None
    assert lib.hysco_correct_adjoint(None, f, f, f, f, f, f, f, f, None) == _lib.EINVAL
    assert lib.hysco_image_grad(None, f, f, f, 1.0, f, f, None) == _lib.EINVAL
    out = C.c_void_p()
    assert lib.hysco_batch_create(0, None, C.byref(out)) == _lib.EINVAL
    assert lib.hysco_batch_create(2, None, C.byref(out)) == _lib.EINVAL
    assert lib.hysco_batch_solve(None, f, f, f, None, None, None) == _lib.EINVAL
    assert lib.hysco_batch_tune(None, f, f, None, None) == _lib.EINVAL
    assert lib.hysco_batch_schedule(None, (C.c_int32 * 3)()) == _lib.EINVAL
    lib.hysco_batch_destroy(None)
    assert lib.hysco_pcg_plan(None, (C.c_int32 * 4)()) == _lib.EINVAL
    assert lib.hysco_batch_set_schedule(None, 1, 0) == _lib.EINVAL
    assert lib.hysco_block_pcg(None, f, f, f, 1.0, f, f, 10, 0.1, None, None) == _lib.EINVAL
    assert lib.hysco_admm_zsolve(None, f, 1.0, f, None) == _lib.EINVAL
    assert lib.hysco_set_pcg_onchip(None, 0) == _lib.EINVAL


def test_barrier_selftest_rejects_bad_arguments_before_any_device_call(lib):
    for grid, missing, cycles in ((0, -1, 1000), (65, -1, 1000), (8, 8, 1000), (8, -2, 1000),
                                  (8, -1, 0), (8, -1, 5_000_000_000)):
        assert lib.hysco_selftest_barrier(grid, missing, cycles, None) == _lib.EINVAL
