"""The benchmark's workload at its full size -- the decaying turbulence on 768^3 at
Lorentz factor 5, in the launch configuration bench.py times -- against the oracle
on sampled cells.

A cell's right-hand side depends only on the cells within the scheme's dependency
radius (echo_decomp_min_halo; pinned on the CPU by tests/test_decomp_radius.py): a
block of 4^3 owned cells with that many ghost layers, run by the oracle as its own
periodic grid, gives the whole grid's right-hand side on the owned cells.  So one
right-hand side of the full grid on the GPU is compared, element by element, with
oracle runs on sampled blocks: at the periodic corners, across the x rows of the
mixed path's row kernel, across the 128-cell segments of its y/z sweeps, inside."""
import ctypes as C
import math

import numpy as np
import pytest

from oracle import oracle as orc
from paper_2401_03008_gb300 import echo
from paper_2401_03008_gb300 import workloads as wl
from tests.parity import CONS_GROUPS, FACE_GROUPS, rel_errors

pytestmark = pytest.mark.gpu

N = 768
L = 2 * math.pi
SEED = 2401_03008
CENTRES = [(0, 0, 0), (767, 767, 767), (128, 128, 400), (383, 127, 256), (5, 600, 129),
           (500, 300, 700)]  # (i, j, k): owned cells c-2 .. c+1 along each direction


def _blocks(t, centres, halo, nown=4):
    """The sub-arrays [..., k, j, i] of a device tensor t ([..., nz, ny, nx]) over the
    padded blocks around the centres, as numpy arrays."""
    import torch
    out = []
    for (ci, cj, ck) in centres:
        ix = [torch.arange(c - 2 - halo, c - 2 + nown + halo, device=t.device) % N
              for c in (ci, cj, ck)]
        b = t.index_select(-1, ix[0]).index_select(-2, ix[1]).index_select(-3, ix[2])
        out.append(np.ascontiguousarray(b.cpu().numpy()))
    return out


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_full_size_turbulence_rhs_against_oracle_blocks(precision):
    import torch
    cfg = echo.make_config(N, N, N)
    halo = echo.lib().echo_decomp_min_halo(C.byref(cfg))
    assert halo == 7
    torch.cuda.empty_cache()
    tb = wl.Turbulence(N, seed=SEED, lorentz_max=5.0, device="cuda")
    st = (tb.prim5(), tb.bface_background(), tb.apot())
    tb.release()
    s = echo.Solver(N, N, N, L=(L, L, L), precision=precision)
    try:
        s.set_state(*st)
        del st
        torch.cuda.empty_cache()
        cons, bf, w, _, _ = s.get_state(device=True)
        scale_c = [float(cons[g].abs().max()) for g in CONS_GROUPS]
        scale_b = float(bf.abs().max())
        bc, bb, bw = _blocks(cons, CENTRES, halo), _blocks(bf, CENTRES, halo), \
            _blocks(w, CENTRES, halo)
        del cons, bf, w
        torch.cuda.empty_cache()
        rc, rb, amax = s.rhs(device=True)
        own = [(c[0], c[1], c[2]) for c in CENTRES]
        gc, gb = _blocks(rc, own, 0), _blocks(rb, own, 0)
        del rc, rb
        torch.cuda.empty_cache()
    finally:
        s.close()
        torch.cuda.empty_cache()
    h = L / N
    npad = 4 + 2 * halo
    errs = []
    for q in range(len(CENTRES)):
        g = orc.Grid(npad, npad, npad, npad * h, npad * h, npad * h)
        g.cons, g.bf, g.W = bc[q], bb[q], bw[q]
        orc_c, orc_b, oamax, bad = g.rhs()
        assert bad == 0
        sl = (Ellipsis, slice(halo, halo + 4), slice(halo, halo + 4), slice(halo, halo + 4))
        refc, refb = orc_c[sl], orc_b[sl]
        # the floor of the normalisation: the rate scale max|q| a_max / h of the flux
        # differences whose cancellation a right-hand side can be (as in the small-grid
        # right-hand-side parity tests)
        e = [rel_errors(gc[q][grp], refc[grp], [list(range(len(grp)))],
                        floor=scale_c[i] * amax / h) for i, grp in enumerate(CONS_GROUPS)]
        e.append(rel_errors(gb[q], refb, FACE_GROUPS, floor=scale_b * amax / h))
        errs.append(np.concatenate(e))
    errs = np.array(errs)
    if precision == "fp64":
        assert np.all(errs <= 1e-10), errs
    else:
        # FP32 reconstruction, fluxes and CT: within FP32 rounding of the rate scale;
        # a limiter decision that FP32 rounding flips at one face stays below 1e-4
        assert np.all(errs <= 1e-4), errs
        assert np.mean(errs) <= 2e-6, errs
