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


@pytest.mark.parametrize("ho", [0, 1])
def test_noalloc_matches_oracle_on_a_stream(ho):
    """On a dedicated stream, at both INT/DER orders: a face field with a
    divergence (so div B is of order |B|/h) and a NaN planted in the host copy of
    the conserved state.  The call must give the oracle's div B (max and RMS) and
    totals of the finite variables, count the one non-finite value, and agree with
    echo_diagnostics of a context holding the same arrays."""
    import torch
    from oracle import oracle as orc
    n, box = (40, 24, 20), (1.0, 0.8, 0.6)
    s = echo.Solver(*n, L=box, ho=ho)
    s.set_state(*wl.random_smooth_fields(*n, seed=42, L=box))
    s.step(2)
    cons, bf, w, t, step = s.get_state()
    rng = np.random.default_rng(43)
    bf = np.ascontiguousarray(bf + 0.1 * rng.standard_normal(bf.shape))
    cons[1, 3, 4, 5] = np.nan
    g = orc.Grid(*n, *box, ho=ho)
    g.cons, g.bf = cons, bf
    div, tot = g.divb(), g.totals()
    s.set_conserved(cons, bf, w, t, step)
    ref = s.diagnostics()
    stream = torch.cuda.Stream()
    dc = torch.from_numpy(cons).cuda()
    db = torch.from_numpy(bf).cuda()
    torch.cuda.synchronize()
    L = echo.lib()
    out = np.full(11, np.inf)
    st = L.echo_diagnostics_noalloc(C.c_void_p(dc.data_ptr()), C.c_void_p(db.data_ptr()),
                                    n[0], n[1], n[2], box[0], box[1], box[2], ho,
                                    C.c_void_p(stream.cuda_stream), C.c_void_p(out.ctypes.data),
                                    echo.PTR_HOST)
    assert st == echo.ECHO_OK, L.echo_last_error(None)
    assert out[8] == pytest.approx(np.max(np.abs(div)), rel=1e-12)
    assert out[9] == pytest.approx(np.sqrt(np.mean(div * div)), rel=1e-12)
    assert out[10] == 1 == ref["nonfinite"]
    assert np.isnan(out[1]) and np.isnan(tot[1])
    for v in [0, 2, 3, 4, 5, 6, 7]:
        scale = np.abs(cons[v]).sum() if v < 5 else np.abs(bf[v - 5]).sum()
        assert abs(out[v] - tot[v]) <= 1e-13 * scale, v
        assert abs(out[v] - ref["tot"][v]) <= 1e-13 * scale, v
    assert out[8] == pytest.approx(ref["divb_max"], rel=1e-12)
