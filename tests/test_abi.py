"""The C-ABI library loads and exports every entry point declared in include/ (no GPU).

Only argument checking is exercised here: no call in this file launches a kernel.
"""

import ctypes
import os
import re

import pytest

from paper_2502_04217_gb300 import binding

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "sdft_ipm.h")


@pytest.fixture(scope="module")
def lib():
    if not os.path.exists(binding.LIB_PATH):
        from paper_2502_04217_gb300 import build
        build.build()
    return binding.load()


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\*?\s*([A-Za-z_][A-Za-z0-9_]*)\s*\(", text, flags=re.M)
    return sorted(set(n for n in names if n not in ("if", "while")))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("ipm_create", "ipm_solve", "kkt_apply", "precond_apply", "ipm_destroy"):
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 15
    for name in names:
        assert hasattr(lib, name), name
        assert name in binding._SIGNATURES, name


def test_default_options(lib):
    o = binding.default_options()
    assert o.precision == binding.IPM_FP64
    assert o.gap_tol == 1e-6 and o.cg_tol == 1e-6 and o.cg_relative == 1 and o.tau == 0.995 and o.sigma == 0.1


@pytest.mark.parametrize("dims,why", [((22,), "factor 11"), ((13,), "prime 13"), ((8, 33), "factor 11"),
                                      ((4, 4, 4, 4), "ndim"), ((2048,), "too long"), ((1025,), "too long, odd"),
                                      ((0,), "empty"), ((1,), "one"), ((8, 1), "one"),
                                      ((625,), "odd, no factor 3, no launchable tile"),
                                      ((875, 4), "odd, no factor 3, no launchable tile"),
                                      ((4, 6, 625), "odd, no factor 3, no launchable tile")])
def test_create_rejects_bad_grids_without_gpu_work(lib, dims, why):
    h = ctypes.c_void_p()
    d = (ctypes.c_int64 * len(dims))(*dims)
    dummy = (ctypes.c_double * 4)()
    st = lib.ipm_create(ctypes.byref(h), len(dims), d, ctypes.cast(dummy, ctypes.c_void_p),
                        ctypes.cast(dummy, ctypes.c_void_p), 1.0, None, None)
    assert st == binding.IPM_ERR_ARG, why
    assert h.value is None
    assert binding.ipm_last_error(None)


def test_create_rejects_bad_options(lib):
    h = ctypes.c_void_p()
    d = (ctypes.c_int64 * 1)(8)
    dummy = (ctypes.c_double * 8)()
    o = binding.default_options(tau=1.5)
    st = lib.ipm_create(ctypes.byref(h), 1, d, ctypes.cast(dummy, ctypes.c_void_p),
                        ctypes.cast(dummy, ctypes.c_void_p), 1.0, ctypes.byref(o), None)
    assert st == binding.IPM_ERR_ARG and "tau" in binding.ipm_last_error(None)


def test_null_handle_calls_fail_cleanly(lib):
    assert lib.ipm_solve(None, None) == binding.IPM_ERR_ARG
    assert lib.kkt_apply(None, None, None) == binding.IPM_ERR_ARG
    assert lib.precond_apply(None, None, None) == binding.IPM_ERR_ARG
    lib.ipm_destroy(None)


def test_default_options_of_the_solver_variants(lib):
    o = binding.default_options()
    assert o.tile_engine == 0 and o.sigma_rule == 2 and o.sigma_min == 0.01
    assert o.exact_residual == 0 and o.precond_rho == 1.0 and o.pdl == 1 and o.krylov == 0 and o.tile_kstage == 0


@pytest.mark.parametrize("field,value,extra", [("tile_engine", 3, {}), ("sigma_rule", 3, {}), ("sigma_rule", -1, {}),
                                               ("sigma_min", -0.1, {}), ("sigma_min", 1.0, {}),
                                               ("sigma_min", 0.0, {"sigma_rule": 1}), ("sigma_min", 0.9, {"sigma_rule": 1}),
                                               ("exact_residual", 2, {}), ("precond_rho", -1.0, {}), ("pdl", 2, {}),
                                               ("krylov", 3, {}), ("krylov", -1, {}), ("precond_rho", float("inf"), {}),
                                               ("tile_kstage", 4, {}), ("tile_kstage", -1, {})])
def test_create_rejects_bad_variant_options(lib, field, value, extra):
    h = ctypes.c_void_p()
    d = (ctypes.c_int64 * 1)(8)
    dummy = (ctypes.c_double * 8)()
    o = binding.default_options(**{field: value}, **extra)
    st = lib.ipm_create(ctypes.byref(h), 1, d, ctypes.cast(dummy, ctypes.c_void_p),
                        ctypes.cast(dummy, ctypes.c_void_p), 1.0, ctypes.byref(o), None)
    assert st == binding.IPM_ERR_ARG and field in binding.ipm_last_error(None)
    assert h.value is None


@pytest.mark.parametrize("krylov", [1, 2])
def test_cr_and_car_reject_residual_replacement(lib, krylov):
    h = ctypes.c_void_p()
    d = (ctypes.c_int64 * 1)(8)
    dummy = (ctypes.c_double * 8)()
    o = binding.default_options(krylov=krylov, refine_every=5)
    st = lib.ipm_create(ctypes.byref(h), 1, d, ctypes.cast(dummy, ctypes.c_void_p),
                        ctypes.cast(dummy, ctypes.c_void_p), 1.0, ctypes.byref(o), None)
    assert st == binding.IPM_ERR_ARG and "refine_every" in binding.ipm_last_error(None)
    assert h.value is None


@pytest.mark.parametrize("dims", [(9,), (16, 15), (15, 16, 8)])
def test_noalloc_rejects_odd_extents_without_gpu_work(lib, dims):
    """The allocation-free G product keeps its even 2^a 3^b extents: odd grids (which
    ipm_create accepts) are refused before any GPU work."""
    d = (ctypes.c_int64 * len(dims))(*dims)
    dummy = (ctypes.c_double * 8)()
    st = lib.gapply_noalloc(len(dims), d, ctypes.cast(dummy, ctypes.c_void_p), ctypes.cast(dummy, ctypes.c_void_p),
                            ctypes.cast(dummy, ctypes.c_void_p), None)
    assert st == binding.IPM_ERR_ARG
    assert "even" in binding.ipm_last_error(None)
