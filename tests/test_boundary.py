"""The C-ABI library builds, loads and exports every entry point include/echo.h
declares; argument checks that need no GPU behave as documented."""
import ctypes as C
import os
import re
import subprocess

import pytest

from paper_2401_03008_gb300 import echo

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared():
    src = open(os.path.join(ROOT, "include", "echo.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(echo_[a-z0-9_]+)\s*\(", src)))


def test_every_declared_symbol_is_exported():
    names = declared()
    assert len(names) >= 17
    L = echo.lib()
    for name in names:
        assert hasattr(L, name), name
    out = subprocess.run(["nm", "-D", "--defined-only", echo.lib_path()], capture_output=True,
                         text=True).stdout
    exported = set(re.findall(r"\bT (echo_[a-z0-9_]+)", out))
    assert set(names) <= exported, set(names) - exported
    assert set(echo.EXPORTS) == set(names)


def test_config_default():
    cfg = echo.Config()
    assert echo.lib().echo_config_default(C.byref(cfg)) == echo.ECHO_OK
    assert (cfg.nx, cfg.uct, cfg.ho, cfg.precision, cfg.rk_order) == (32, 1, 1, echo.FP64, 3)
    assert cfg.gamma_ad == pytest.approx(4 / 3) and cfg.cfl == 0.4 and cfg.c2p_tol == 1e-6


@pytest.mark.parametrize("field,value", [("nx", 0), ("lz", -1.0), ("gamma_ad", 1.0),
                                         ("cfl", 0.0), ("uct", 2), ("ho", 2), ("precision", 7),
                                         ("c2p_guess", 5), ("c2p_maxit", 0), ("rec", 2),
                                         ("rk_order", 4)])
def test_create_rejects_bad_config(field, value):
    L = echo.lib()
    cfg = echo.Config()
    L.echo_config_default(C.byref(cfg))
    setattr(cfg, field, value)
    h = C.c_void_p()
    assert L.echo_create(C.byref(cfg), C.byref(h)) == echo.ECHO_ERR_ARG
    assert not h.value
    assert L.echo_last_error(None)


def test_null_arguments_rejected():
    L = echo.lib()
    assert L.echo_create(None, None) == echo.ECHO_ERR_ARG
    assert L.echo_step(None, 1, 1.0, None, None) == echo.ECHO_ERR_ARG
    assert L.echo_set_state(None, None, None, None, 0) == echo.ECHO_ERR_ARG
    assert L.echo_destroy(None) == echo.ECHO_OK
    assert L.echo_launches(None) == 0


def test_create_without_gpu_reports_cuda_error():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    L = echo.lib()
    cfg = echo.Config()
    L.echo_config_default(C.byref(cfg))
    h = C.c_void_p()
    assert L.echo_create(C.byref(cfg), C.byref(h)) == echo.ECHO_ERR_CUDA
    with pytest.raises(echo.EchoError):
        echo.Solver(8, 8, 8)


@pytest.mark.parametrize("uct,ho,rec,expect", [(1, 1, 0, 7), (1, 0, 0, 4), (0, 1, 0, 5),
                                                (0, 0, 0, 3), (1, 1, 1, 6), (0, 0, 1, 2)])
def test_decomp_min_halo(uct, ho, rec, expect):
    """The upwind dependency radius of one substep: DER faces (3 with HO, else 1)
    + REC cells (2 for MP5, 1 linear) + INT faces (2 with HO, 1 without, 0 when
    the field is cell-centred)."""
    cfg = echo.make_config(8, 8, 8, uct=uct, ho=ho, rec=["mp5", "linear"][rec])
    assert echo.lib().echo_decomp_min_halo(C.byref(cfg)) == expect
    cfg.ho = 3
    assert echo.lib().echo_decomp_min_halo(C.byref(cfg)) == -1
    assert echo.lib().echo_decomp_min_halo(None) == -1


@pytest.mark.parametrize("blocks,halo,guess", [((3, 1, 1), 7, "prev"), ((2, 0, 1), 7, "prev"),
                                               ((2, 2, 2), 0, "prev"), ((2, 1, 1), 7, "mlp")])
def test_decomp_rejects_bad_arguments(blocks, halo, guess):
    L = echo.lib()
    cfg = echo.make_config(16, 8, 8, guess=guess)
    h = C.c_void_p()
    assert L.echo_decomp_create(C.byref(cfg), *blocks, halo, C.byref(h)) == echo.ECHO_ERR_ARG
    assert not h.value and L.echo_decomp_last_error(None)
    assert L.echo_decomp_create(None, 1, 1, 1, 1, C.byref(h)) == echo.ECHO_ERR_ARG
    assert L.echo_decomp_step(None, 1, 1.0, None, None) == echo.ECHO_ERR_ARG
    assert L.echo_decomp_destroy(None) == echo.ECHO_OK


@pytest.mark.parametrize("shape", [(2048, 2048, 512), (1 << 20, 1 << 11, 1)])
def test_create_rejects_grids_of_2_31_cells(shape):
    """Kernels index cells with 32-bit integers: 2^31 cells and more are refused
    before any device work."""
    L = echo.lib()
    cfg = echo.make_config(*shape)
    h = C.c_void_p()
    assert L.echo_create(C.byref(cfg), C.byref(h)) == echo.ECHO_ERR_ARG
    assert b"2^31" in L.echo_last_error(None)


def test_create_accepts_one_cell_per_direction_before_device_check():
    """A 1 x 1 x 1 grid is a valid configuration: without a GPU the call gets past the
    argument checks and stops at the device."""
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    L = echo.lib()
    cfg = echo.make_config(1, 1, 1)
    h = C.c_void_p()
    assert L.echo_create(C.byref(cfg), C.byref(h)) == echo.ECHO_ERR_CUDA


def test_binding_marshals_only_float64_arrays_of_the_right_size():
    """The binding passes numpy arrays as host pointers and CUDA tensors as device
    pointers; anything else is refused before the library is called."""
    import numpy as np
    torch = pytest.importorskip("torch")
    p, kind = echo._ptr(np.zeros(10), "x", 10)
    assert kind == echo.PTR_HOST and p.value
    assert echo._ptr(None, "x", 10) == (None, None)
    for bad in (np.zeros(10, dtype=np.float32), np.zeros((4, 5))[:, ::2], np.zeros(9),
                torch.zeros(10, dtype=torch.float64), [0.0] * 10):
        with pytest.raises(ValueError):
            echo._ptr(bad, "x", 10)
    with pytest.raises(ValueError):
        echo.Solver._same_kind(echo.PTR_HOST, echo.PTR_DEVICE)
    assert echo.Solver._same_kind(None, echo.PTR_DEVICE, None) == echo.PTR_DEVICE
    assert echo.Solver._same_kind(None, None) == echo.PTR_HOST
