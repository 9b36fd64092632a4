"""The dependency radius behind the decomposed grid's minimum halo, pinned on the
CPU with the oracle: the right-hand side that a padded block computes on its own
(periodic inside the block, as the GPU blocks do) equals the whole grid's on the
block's owned cells, bit for bit, once the block carries echo_decomp_min_halo ghost
layers, and differs with one layer less, for every scheme the library offers."""
import ctypes as C

import numpy as np
import pytest

from oracle import oracle as orc
from paper_2401_03008_gb300 import echo
from paper_2401_03008_gb300 import workloads as wl

N = (20, 18, 16)


def _global(uct, ho, rec):
    # unit cells (L = N) keep h = 1 exact in both the global grid and the padded block
    L = tuple(float(v) for v in N)
    prim, bg, apot = wl.random_smooth_fields(*N, seed=81, L=L)
    g = orc.Grid(*N, *L, uct=uct, ho=ho, rec=rec, nthreads=4)
    if uct:
        g.set_state(prim, bg, apot)
    else:
        c = wl.CPA(*N, m=(1, 1, 1), L=L)
        g.set_state(c.prim5(), c.bcell())
    return g


def _block_rhs(g, uct, ho, rec, lo, nloc, halo):
    """rhs of the padded block of owned cells [lo, lo + nloc) along x (the other
    directions whole), run as its own periodic grid."""
    nz, ny, nx = g.shape
    idx = (np.arange(lo - halo, lo + nloc + halo)) % nx
    npad = nloc + 2 * halo
    b = orc.Grid(npad, ny, nz, float(npad), float(ny), float(nz), uct=uct, ho=ho, rec=rec,
                 nthreads=4)
    b.cons = np.ascontiguousarray(g.cons[..., idx])
    b.bf = np.ascontiguousarray(g.bf[..., idx])
    b.W = np.ascontiguousarray(g.W[..., idx])
    rc, rb, _, bad = b.rhs()
    assert bad == 0
    return rc[..., halo:halo + nloc], rb[..., halo:halo + nloc]


@pytest.mark.parametrize("uct,ho,rec", [(1, 1, 0), (1, 0, 0), (0, 1, 0), (0, 0, 0),
                                        (1, 1, 1), (0, 0, 1)])
def test_min_halo_is_the_dependency_radius(uct, ho, rec):
    cfg = echo.make_config(*N, uct=uct, ho=ho, rec=["mp5", "linear"][rec])
    radius = echo.lib().echo_decomp_min_halo(C.byref(cfg))
    g = _global(uct, ho, rec)
    W0 = g.W.copy()
    rc, rb, _, bad = g.rhs()
    assert bad == 0
    g.W = W0  # each block starts from the same warm guess as the whole grid did
    lo, nloc = 6, 7
    own_c, own_b = rc[..., lo:lo + nloc], rb[..., lo:lo + nloc]
    bc, bb = _block_rhs(g, uct, ho, rec, lo, nloc, radius)
    assert np.array_equal(bc, own_c) and np.array_equal(bb, own_b)
    bc, bb = _block_rhs(g, uct, ho, rec, lo, nloc, radius - 1)
    assert not (np.array_equal(bc, own_c) and np.array_equal(bb, own_b))
