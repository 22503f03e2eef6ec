"""The C-ABI library builds, loads and exports every entry point of include/rbc.h.

CPU-only: no compute call is made; argument validation paths return before any
CUDA call.
"""
import ctypes
import os
import re

import pytest

from paper_2001_01609_gb300 import build, rbc

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "rbc.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^[A-Za-z_][\w\s\*]*?\b(rbc_\w+|parareal_\w+)\s*\(", src, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    build.build()
    return rbc.load()


def test_header_declares_the_boundary():
    names = declared_functions()
    for n in ("rbc_create", "rbc_step_batch", "parareal_iterate", "rbc_nusselt", "parareal_create"):
        assert n in names
    assert set(names) == set(rbc.EXPORTS)


def test_library_exports_every_declared_symbol(lib):
    for n in declared_functions():
        assert hasattr(lib, n), n


def test_invalid_arguments_are_rejected_without_touching_the_device(lib):
    h = ctypes.c_void_p()
    for args in ((1e4, 1.0, 2.0, 63, 32, 1e-3), (1e4, 1.0, 2.0, 64, 31, 1e-3), (1e4, 1.0, 2.0, 64, 32, -1.0),
                 (1e4, 0.0, 2.0, 64, 32, 1e-3), (1e4, 1.0, 2.0, 48, 32, 1e-3), (1e4, 1.0, 2.0, 64, 6, 1e-3)):
        st = lib.rbc_create(*args, None, ctypes.byref(h))
        assert st == rbc.RBC_EINVAL
        assert h.value is None
    assert lib.rbc_create(1e4, 1.0, 2.0, 64, 32, 1e-3, None, None) == rbc.RBC_EINVAL
    assert lib.rbc_state_bytes(None) == 0
    assert lib.rbc_step_batch(None, None, 1, None, None, None) == rbc.RBC_EINVAL
    assert lib.parareal_create(None, None, 0.0, 1.0, 4, 0, 0.0, ctypes.byref(h)) == rbc.RBC_EINVAL
    assert lib.rbc_diagnostics(None, None, 1, None, None) == rbc.RBC_EINVAL
    assert lib.rbc_diag_size(None) == 0
    assert b"need" in lib.rbc_last_error() or len(lib.rbc_last_error()) > 0


def test_stage_factors_of_both_boundary_conditions_pass_the_residual_check(lib):
    """rbc_create builds and factors every stage matrix on the host, checks the
    solve residual (else RBC_EINVAL), and only then allocates on the device.
    Without a GPU that first allocation fails (RBC_ECUDA): reaching it means
    the unpivoted factors of the fixed-temperature and fixed-flux systems of
    these grids passed the check."""
    import torch
    if torch.cuda.is_available():
        pytest.skip("the check needs the device allocation to fail")
    h = ctypes.c_void_p()
    for bc in (rbc.RBC_FIXED_T, rbc.RBC_FIXED_FLUX):
        for Nx, Nz, dt, Ra in ((32, 16, 1e-3, 1e4), (256, 64, 2e-4, 1e6), (512, 128, 5e-5, 1e7),
                               (1024, 256, 2e-5, 1e8), (64, 8, 1e-2, 1e4)):
            o = rbc._Opts(rbc.RBC_FP64, bc, 0)
            st = lib.rbc_create(Ra, 1.0, 2.0, Nx, Nz, dt, ctypes.byref(o), ctypes.byref(h))
            assert st == rbc.RBC_ECUDA, (bc, Nx, Nz, lib.rbc_last_error())
            assert b"cudaMalloc" in lib.rbc_last_error()
            assert h.value is None
    o = rbc._Opts(rbc.RBC_FP64, 2, 0)
    assert lib.rbc_create(1e4, 1.0, 2.0, 32, 16, 1e-3, ctypes.byref(o), ctypes.byref(h)) == rbc.RBC_EINVAL


def test_binding_refuses_to_run_without_the_library(monkeypatch, tmp_path):
    monkeypatch.setattr(rbc, "_lib", None)
    monkeypatch.setattr(rbc, "LIB_PATH", str(tmp_path / "missing.so"))
    with pytest.raises(RuntimeError):
        rbc.Propagator(1e4, 1.0, 2.0, 16, 16, 1e-3)
