"""echo_diagnostics_noalloc: the diagnostics of caller-owned device arrays for
callers that cannot allocate device memory (their memory belongs to a fixed pool
or another framework).  Through the C ABI it must agree with echo_diagnostics of a
context holding the same state, call after call, and reject grids larger than its
static scratch array.  This file is collected last on purpose."""
import ctypes as C

import numpy as np
import pytest

from paper_2401_03008_gb300 import echo
from paper_2401_03008_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


def _call(L, cons, bf, n, box, ho, out, kind):
    return L.echo_diagnostics_noalloc(
        C.c_void_p(cons), C.c_void_p(bf), n[0], n[1], n[2], box[0], box[1], box[2], ho, None,
        C.c_void_p(out), kind)


def test_noalloc_diagnostics_matches_context():
    import torch
    n, box = (40, 24, 20), (1.0, 0.8, 0.6)
    s = echo.Solver(*n, L=box)
    s.set_state(*wl.random_smooth_fields(*n, seed=41, L=box))
    s.step(3)
    cons, bf, w, t, step = s.get_state(device=True)
    ref = s.diagnostics()
    torch.cuda.synchronize()
    L = echo.lib()
    scale_c = torch.abs(cons).sum(dim=(1, 2, 3)).max().item()
    for call in range(2):
        out = np.full(11, np.nan)
        st = _call(L, cons.data_ptr(), bf.data_ptr(), n, box, 1, out.ctypes.data, echo.PTR_HOST)
        assert st == echo.ECHO_OK, L.echo_last_error(None)
        assert np.allclose(out[:8], ref["tot"], rtol=0, atol=1e-13 * scale_c), (call, out)
        assert out[8] == pytest.approx(ref["divb_max"], rel=1e-12, abs=1e-300)
        assert out[9] == pytest.approx(ref["divb_l2"], rel=1e-10, abs=1e-300)
        assert out[10] == ref["nonfinite"] == 0
    # device output buffer, second state
    s.step(1)
    cons2, bf2, _, _, _ = s.get_state(device=True)
    ref2 = s.diagnostics()
    dout = torch.full((11,), float("nan"), dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    st = _call(L, cons2.data_ptr(), bf2.data_ptr(), n, box, 1, dout.data_ptr(), echo.PTR_DEVICE)
    assert st == echo.ECHO_OK
    got = dout.cpu().numpy()
    assert np.allclose(got[:8], ref2["tot"], rtol=0, atol=1e-13 * scale_c)
    assert got[8] == pytest.approx(ref2["divb_max"], rel=1e-12, abs=1e-300)


def test_noalloc_rejects_oversize_grid():
    L = echo.lib()
    out = np.zeros(11)
    # the size check comes before any pointer is used, so NULL inputs are safe here
    st = _call(L, None, None, (128, 128, 128), (1.0, 1.0, 1.0), 1, out.ctypes.data,
               echo.PTR_HOST)
    assert st == echo.ECHO_ERR_ARG
    assert b"1048576" in L.echo_last_error(None)
    st = _call(L, None, None, (8, 8, 8), (1.0, 1.0, 1.0), 1, out.ctypes.data, echo.PTR_HOST)
    assert st == echo.ECHO_ERR_ARG
