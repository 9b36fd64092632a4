"""GPU path (libecho through its C ABI) against the FP64 oracle, element by element.

Sizes span several 256-thread blocks with ragged tails; the full-size checks run
the 256^3 grid of the benchmark in its launch configuration and compare with
oracle runs that reduce to one line, or with properties that hold at any size."""
import math

import numpy as np
import pytest

from oracle import oracle as orc
from paper_2401_03008_gb300 import echo
from paper_2401_03008_gb300 import workloads as wl
from tests.parity import (CONS_GROUPS, FACE_GROUPS, FP64_TOL, PRIM_GROUPS, assert_parity,
                          rel_errors)

pytestmark = pytest.mark.gpu


def make_pair(n, L=(1.0, 1.0, 1.0), ho=1, precision="fp64", state=None, **kw):
    nx, ny, nz = n
    g = orc.Grid(nx, ny, nz, *L, ho=ho)
    s = echo.Solver(nx, ny, nz, L=L, ho=ho, precision=precision, **kw)
    prim, bg, apot = state
    g.set_state(prim, bg, apot)
    s.set_state(prim, bg, apot)
    return g, s


def smooth(n, seed, L=(1.0, 1.0, 1.0)):
    return wl.random_smooth_fields(*n, seed=seed, L=L)


def cpa_state(n, m, L=(1.0, 1.0, 1.0)):
    c = wl.CPA(*n, m=m, L=L)
    return c, (c.prim5(), c.bface_background(), c.apot())


@pytest.mark.parametrize("ho", [0, 1])
def test_set_state_parity(ho):
    g, s = make_pair((33, 17, 9), ho=ho, state=smooth((33, 17, 9), 31))
    cons, bf, w, t, step = s.get_state()
    assert_parity(cons, g.cons, CONS_GROUPS, tol=1e-14, what="cons")
    assert_parity(bf, g.bf, FACE_GROUPS, tol=1e-14, what="bface")
    assert np.max(np.abs(w - g.W) / g.W) < 1e-14
    assert t == 0.0 and step == 0


@pytest.mark.parametrize("ho", [0, 1])
@pytest.mark.parametrize("case", ["smooth", "cpa_oblique"])
def test_rhs_parity(ho, case):
    if case == "smooth":
        n, L, st = (40, 24, 20), (1.0, 0.8, 0.6), smooth((40, 24, 20), 32, L=(1.0, 0.8, 0.6))
    else:
        n, L = (16, 16, 16), (1.0, 1.0, 1.0)
        st = cpa_state(n, (1, 1, 1))[1]
    g, s = make_pair(n, L=L, ho=ho, state=st)
    cons0, bf0 = g.cons.copy(), g.bf.copy()
    rc, rb, amax, bad, prim = g.rhs(with_prims=True)
    grc, grb, gamax = s.rhs()
    assert bad == 0
    assert gamax == pytest.approx(amax, rel=1e-13)
    # a right-hand side can be small by cancellation of O(q a/h) flux differences
    # (dD/dt of the Alfven wave is truncation-sized): its rounding is relative to
    # that rate scale, which is the floor of the normalisation
    hmin = min(L[d] / n[d] for d in range(3))
    for got, ref, q, groups, what in ((grc, rc, cons0, CONS_GROUPS, "rhs cells"),
                                      (grb, rb, bf0, FACE_GROUPS, "rhs faces")):
        for grp in groups:
            floor = np.max(np.abs(q[grp])) * amax / hmin
            assert_parity(got[grp], ref[grp], [list(range(len(grp)))], floor=floor, what=what)


def test_primitives_parity():
    g, s = make_pair((40, 24, 20), state=smooth((40, 24, 20), 33))
    assert_parity(s.primitives(), g.primitives(), PRIM_GROUPS, tol=1e-13, what="prims")


def test_steps_parity_alfven_32():
    """The 32^3 Alfven wave along x, FP64, 20 SSP-RK3 steps at CFL 0.4.  The GPU runs
    the library's Newton tolerance (1e-6 with the polishing step); the oracle is run
    twice, with that tolerance and with 1e-12, so the inversion's result is checked
    against a tighter solve too, not only against the same stopping rule."""
    n = (32, 32, 32)
    c, st = cpa_state(n, (1, 0, 0))
    g, s = make_pair(n, state=st)
    g.step(20)
    done, t = s.step(20)
    assert done == 20
    assert t == pytest.approx(g.t, rel=1e-13)
    assert_parity(s.primitives(), g.primitives(), PRIM_GROUPS, what="prims after 20 steps")
    cons, bf, w, t2, step = s.get_state()
    assert step == 20
    assert_parity(cons, g.cons, CONS_GROUPS, what="cons")
    assert_parity(bf, g.bf, FACE_GROUPS, what="bface")
    tight = orc.Grid(*n, tol=1e-12)
    tight.set_state(*st)
    tight.step(20)
    assert tight.t == pytest.approx(g.t, rel=1e-13)
    assert_parity(s.primitives(), tight.primitives(), PRIM_GROUPS, what="vs oracle at tol 1e-12")
    assert_parity(cons, tight.cons, CONS_GROUPS, what="cons vs oracle at tol 1e-12")


@pytest.mark.parametrize("ho", [0, 1])
def test_steps_parity_ragged(ho):
    n, L = (33, 17, 9), (1.0, 0.7, 0.45)
    g, s = make_pair(n, L=L, ho=ho, state=smooth(n, 34, L=L))
    g.step(6)
    s.step(6)
    assert_parity(s.primitives(), g.primitives(), PRIM_GROUPS, what="prims")


def test_steps_parity_oblique():
    n = (24, 20, 16)
    c, st = cpa_state(n, (1, 1, 1))
    g, s = make_pair(n, state=st)
    g.step(6)
    s.step(6)
    assert_parity(s.primitives(), g.primitives(), PRIM_GROUPS, what="prims")


def test_step_lands_on_t_end():
    n = (16, 16, 16)
    c, st = cpa_state(n, (1, 1, 0))
    g, s = make_pair(n, state=st)
    t_end = 0.05
    g.step(1000, t_end=t_end)
    done, t = s.step(1000, t_end=t_end)
    assert t == t_end and g.t == t_end
    assert done == g.steps
    assert_parity(s.primitives(), g.primitives(), PRIM_GROUPS, what="prims")
    done2, t2 = s.step(10, t_end=t_end)
    assert done2 == 0 and t2 == t_end


@pytest.mark.parametrize("m,shape", [((1, 0, 0), (256, 1, 1)), ((0, 1, 0), (1, 256, 1)),
                                     ((0, 0, 1), (1, 1, 256))])
def test_full_size_axis_wave(m, shape):
    """256^3 with the wave along one axis: every line along it must equal the
    oracle's one-line run (the benchmark's grid and launch configuration)."""
    n = (256, 256, 256)
    c = wl.CPA(*n, m=m)
    s = echo.Solver(*n)
    s.set_state(c.prim5(), c.bface_background(), c.apot())
    s.step(2)
    got = s.primitives()
    c1 = wl.CPA(*shape, m=m)
    g = orc.Grid(*shape)
    g.set_state(c1.prim5(), c1.bface_background(), c1.apot())
    g.step(2)
    ref = np.broadcast_to(g.primitives(), got.shape)
    assert_parity(got, ref, PRIM_GROUPS, what="256^3 axis wave")


def test_full_size_oblique_translation_invariance():
    """256^3 with k along (1,1,1): the exact state depends on i+j+k only, so the
    computed state must be invariant under (i,j,k) -> (i+1, j-1, k) and
    (i, j+1, k-1) up to rounding; a block or tile edge handled differently
    would break it by far more."""
    n = (256, 256, 256)
    c = wl.CPA(*n, m=(1, 1, 1))
    s = echo.Solver(*n)
    s.set_state(c.prim5(), c.bface_background(), c.apot())
    s.step(1)
    p = s.primitives()
    sh1 = np.roll(np.roll(p, 1, axis=3), -1, axis=2)
    sh2 = np.roll(np.roll(p, 1, axis=2), -1, axis=1)
    for sh in (sh1, sh2):
        e = rel_errors(sh, p, PRIM_GROUPS)
        assert np.all(e < 1e-12), e
    # and the step agrees with the exact solution to truncation level
    ex = c.exact_prim8(s.diagnostics()["t"])
    assert np.max(rel_errors(p, ex, PRIM_GROUPS)) < 1e-4


def test_conservation_divb_determinism():
    n = (48, 40, 32)
    st = smooth(n, 35)
    s = echo.Solver(*n)
    s.set_state(*st)
    d0 = s.diagnostics()
    s.step(10)
    d1 = s.diagnostics()
    d2 = s.diagnostics()
    assert d1 == d2
    cons, bf, w, t, step = s.get_state()
    scale = np.abs(cons).sum(axis=(1, 2, 3)).max()
    assert np.max(np.abs(np.array(d1["tot"]) - np.array(d0["tot"]))) <= 1e-13 * scale
    h = 1.0 / 48
    assert d1["divb_max"] <= 1e-12 * np.abs(bf).max() / h
    assert d0["divb_max"] <= 1e-12 * np.abs(bf).max() / h
    assert d1["c2p_failures"] == 0 and d1["nonfinite"] == 0
    assert 1.0 <= d1["newton_it_mean"] <= 6.0


def test_c2p_failure_rolls_back():
    """A Newton cap the second stage cannot meet: echo_step reports ECHO_ERR_C2P and
    the state, t and step count are those at the start of the failed step."""
    n = (16, 16, 16)
    c, st = cpa_state(n, (1, 1, 1))
    # stage 1 starts from the exact W of the initial data and converges in 2
    # iterations; the later stages need 3, so a cap of 2 fails there
    s = echo.Solver(*n, maxit=2)
    s.set_state(*st)
    cons0, bf0, _, t0, step0 = s.get_state()
    with pytest.raises(echo.EchoError) as ei:
        s.step(3)
    assert ei.value.status == echo.ECHO_ERR_C2P
    assert "stage 2" in str(ei.value) or "stage 3" in str(ei.value), str(ei.value)
    cons1, bf1, _, t1, step1 = s.get_state()
    assert np.array_equal(cons0, cons1) and np.array_equal(bf0, bf1)
    assert t1 == t0 and step1 == step0


@pytest.mark.parametrize("kw", [dict(), dict(precision="mixed", sweeps="fused"),
                                dict(precision="mixed", sweeps="separate")])
def test_unphysical_state_reported(kw):
    """A cell whose energy lies below its rest mass: every inversion kernel (the
    mixed path's inversion fused with the x sweep included) reports it, and the step
    is rolled back."""
    n = (12, 10, 8)
    s = echo.Solver(*n, **kw)
    s.set_state(*smooth(n, 36))
    cons, bf, w, t, step = s.get_state()
    cons[4, 3, 2, 1] = 0.1 * cons[0, 3, 2, 1]  # energy below the rest mass
    s.set_conserved(cons, bf, w, t, step)
    with pytest.raises(echo.EchoError) as ei:
        s.step(1)
    assert ei.value.status == echo.ECHO_ERR_C2P
    cons1, _, _, _, _ = s.get_state()
    assert np.array_equal(cons, cons1)


def test_checkpoint_resume_bit_exact():
    n = (24, 16, 12)
    st = smooth(n, 37)
    a = echo.Solver(*n)
    a.set_state(*st)
    a.step(4)
    b = echo.Solver(*n)
    b.set_state(*st)
    b.step(2)
    cons, bf, w, t, step = b.get_state()
    b.close()
    c = echo.Solver(*n)
    c.set_conserved(cons, bf, w, t, step)
    c.step(2)
    ra, rc = a.get_state(), c.get_state()
    for x, y in zip(ra[:3], rc[:3]):
        assert np.array_equal(x, y)
    assert ra[3] == rc[3] and ra[4] == rc[4] == 4


def test_l1_error_and_device_pointers():
    import torch
    n = (20, 18, 16)
    c, st = cpa_state(n, (1, 1, 0))
    s = echo.Solver(*n)
    s.set_state(*[torch.from_numpy(x).cuda() for x in st])
    h = echo.Solver(*n)
    h.set_state(*st)
    assert np.array_equal(s.get_state()[0], h.get_state()[0])
    s.step(3)
    h.step(3)
    ex = c.exact_prim8(s.diagnostics()["t"])
    p = s.primitives()
    l1 = s.l1_error(ex)
    assert np.allclose(l1, np.mean(np.abs(p - ex), axis=(1, 2, 3)), rtol=1e-12, atol=1e-300)
    l1d = s.l1_error(torch.from_numpy(ex).cuda())
    assert np.array_equal(l1, l1d)
    rc, rb, am = s.rhs(device=True)
    rch, rbh, amh = h.rhs()
    assert np.array_equal(rc.cpu().numpy(), rch) and np.array_equal(rb.cpu().numpy(), rbh)
    pd = s.primitives(device=True)
    assert np.array_equal(pd.cpu().numpy(), h.primitives())


def test_mixed_precision_close_to_oracle():
    """FP32 reconstruction/fluxes/CT with FP64 inversion and RK: the L1 distance to
    the FP64 oracle stays within 1e-6 of the field scale on the 32^3 wave."""
    n = (32, 32, 32)
    c, st = cpa_state(n, (1, 0, 0))
    g, s = make_pair(n, precision="mixed", state=st)
    g.step(20)
    s.step(20)
    p, ref = s.primitives(), g.primitives()
    for grp in PRIM_GROUPS:
        scale = np.max(np.abs(ref[grp]))
        for v in grp:
            assert np.mean(np.abs(p[v] - ref[v])) / scale < 1e-6, v


def test_fma_probe_plausible():
    s = echo.Solver(8, 8, 8)
    f64 = s.probe_fma_peak("fp64")
    f32 = s.probe_fma_peak("fp32")
    assert 1e11 < f64 < 1e14 and 1e13 < f32 < 1e15


@pytest.mark.parametrize("ho", [0, 1])
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_cell_centred_variant_parity(ho, precision):
    """UCT off: the field is cell-centred and all 8 components take the HLL flux."""
    n = (24, 20, 16)
    c = wl.CPA(*n, m=(1, 1, 1))
    st = (c.prim5(), c.bcell(), None)
    g = orc.Grid(*n, uct=0, ho=ho)
    g.set_state(*st)
    s = echo.Solver(*n, ho=ho, uct=0, precision=precision)
    s.set_state(*st)
    cons0 = g.cons.copy()
    rc, rb, amax, bad = g.rhs()
    grc, grb, gamax = s.rhs()
    if precision == "fp64":
        hmin = 1.0 / 24
        for got, ref, q, groups in ((grc, rc, cons0, CONS_GROUPS), (grb, rb, g.bf, FACE_GROUPS)):
            for grp in groups:
                floor = np.max(np.abs(q[grp])) * amax / hmin
                assert_parity(got[grp], ref[grp], [list(range(len(grp)))], floor=floor)
    g.step(5)
    s.step(5)
    tol = FP64_TOL if precision == "fp64" else 1e-5
    assert_parity(s.primitives(), g.primitives(), PRIM_GROUPS, tol=tol, what="uct off")


def test_cell_centred_turbulence_parity():
    n = 20
    tb = wl.Turbulence(n, seed=105, lorentz_max=2.0)
    st = (tb.prim5(), tb.bcell(), None)
    L = (2 * np.pi,) * 3
    g = orc.Grid(n, n, n, *L, uct=0, ho=0)
    g.set_state(*st)
    s = echo.Solver(n, n, n, L=L, uct=0, ho=0)
    s.set_state(*st)
    g.step(4)
    s.step(4)
    assert_parity(s.primitives(), g.primitives(), PRIM_GROUPS, what="turbulence, uct off")


@pytest.mark.parametrize("uct", [1, 0])
def test_fast_variant_parity(uct):
    """Linear reconstruction with SSP-RK2 (the faster variant of Sec. 4)."""
    n = (24, 20, 16)
    c = wl.CPA(*n, m=(1, 1, 1))
    st = (c.prim5(), c.bcell(), None) if uct == 0 else (c.prim5(), c.bface_background(), c.apot())
    ho = uct
    g = orc.Grid(*n, uct=uct, ho=ho, rec=1, rk=2)
    g.set_state(*st)
    s = echo.Solver(*n, uct=uct, ho=ho, rec="linear", rk_order=2)
    s.set_state(*st)
    g.step(6)
    done, t = s.step(6)
    assert done == 6 and t == pytest.approx(g.t, rel=1e-13)
    assert_parity(s.primitives(), g.primitives(), PRIM_GROUPS, what="linear + RK2")


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_turbulence_2d_parity(precision):
    """The 2.5-D set-up of Sec. 5 (nz = 1, sigma0 = 100) over one time unit on 80^2:
    the z sweeps wrap onto the one layer and the z-edge field carries the in-plane
    dynamics.  FP64 element by element; mixed within the FP32 reconstruction error."""
    n = 80
    tb = wl.Turbulence2D(n, seed=106)
    st = (tb.prim5(), tb.bface_background(), tb.apot())
    g = orc.Grid(n, n, 1, *tb.L, nthreads=8)
    g.set_state(*st)
    s = echo.Solver(n, n, 1, L=tb.L, precision=precision)
    s.set_state(*st)
    assert g.step(100000, t_end=1.0) == 0
    done, t = s.step(100000, 1.0)
    assert t == 1.0 and done == len(g.dts)
    tol = FP64_TOL if precision == "fp64" else 1e-5
    assert_parity(s.primitives(), g.primitives(), PRIM_GROUPS, tol=tol, what="2.5-D turbulence")
    d = s.diagnostics()
    # div B stays at the round-off of the precision the curl of E is taken in
    b_over_h = tb.B0 * n / (2 * np.pi)
    assert d["divb_max"] < (1e-11 if precision == "fp64" else 1e-7) * b_over_h
    assert d["c2p_failures"] == 0


def _oracle_view(n, L, ho, cons, bf):
    """An oracle grid holding a given state (for its totals and div B)."""
    g = orc.Grid(*n, *L, ho=ho)
    g.cons = np.ascontiguousarray(cons)
    g.bf = np.ascontiguousarray(bf)
    return g


@pytest.mark.parametrize("ho", [0, 1])
def test_diagnostics_match_oracle(ho):
    """echo_diagnostics against the oracle on the same states (Sec. 3: UCT keeps the
    discrete div B at round-off; the periodic box conserves the totals):
      - after 3 steps of both, the Newton statistics (calls, summed iterations,
        largest count) equal the oracle's: same guesses, same stopping rule;
      - the conserved totals equal orc_totals of the GPU's state to rounding;
      - on a face field that is not solenoidal (div B of order |B|/h), max |div B|
        and its RMS equal those of orc_divb, which checks the stencil, the divisor
        and the RMS normalisation;
      - a non-finite value planted in the state is counted."""
    n, L = (40, 24, 20), (1.0, 0.8, 0.6)
    g, s = make_pair(n, L=L, ho=ho, state=smooth(n, 38, L=L))
    assert g.step(3) == 0
    s.step(3)
    d = s.diagnostics()
    ncell = int(np.prod(n))
    assert d["c2p_calls"] == g.stats.cells == 9 * ncell
    assert round(d["newton_it_mean"] * d["c2p_calls"]) == g.stats.iters
    assert d["newton_it_max"] == g.stats.itmax
    assert d["c2p_failures"] == g.stats.failures == 0
    cons, bf, w, t, step = s.get_state()
    ref = _oracle_view(n, L, ho, cons, bf)
    tot = ref.totals()
    scale = np.abs(cons).sum(axis=(1, 2, 3)).max()
    assert np.max(np.abs(np.array(d["tot"]) - tot)) <= 1e-13 * scale
    # div B of the stepped state is round-off on both sides
    h = min(L[q] / n[q] for q in range(3))
    assert d["divb_max"] <= 1e-12 * np.abs(bf).max() / h
    assert np.max(np.abs(ref.divb())) <= 1e-12 * np.abs(bf).max() / h
    # a face field with a divergence
    rng = np.random.default_rng(39)
    bfr = bf + 0.1 * rng.standard_normal(bf.shape)
    s.set_conserved(cons, bfr, w, t, step)
    d2 = s.diagnostics()
    div = _oracle_view(n, L, ho, cons, bfr).divb()
    assert np.max(np.abs(div)) > 1.0
    assert d2["divb_max"] == pytest.approx(np.max(np.abs(div)), rel=1e-12)
    assert d2["divb_l2"] == pytest.approx(np.sqrt(np.mean(div * div)), rel=1e-12)
    face_tot = _oracle_view(n, L, ho, cons, bfr).totals()[5:]
    assert np.max(np.abs(np.array(d2["tot"][5:]) - face_tot)) <= 1e-13 * np.abs(bfr).sum()
    assert d2["nonfinite"] == 0
    bad = cons.copy()
    bad[2, 5, 6, 7] = np.nan
    s.set_conserved(bad, bfr, w, t, step)
    assert s.diagnostics()["nonfinite"] == 1


@pytest.mark.parametrize("sweeps", ["fused", "separate"])
def test_mixed_sweep_kernels_against_oracle(sweeps):
    """The mixed path with each kind of y/z sweep kernel (the fused TMA sweep forced
    on a grid small enough that the automatic choice would not take it): one
    right-hand side of a smooth state on 40 x 24 x 20 and 20 steps of the 32^3 wave,
    against the FP64 oracle within the FP32 rounding of the reconstruction."""
    n, L = (40, 24, 20), (1.0, 0.8, 0.6)
    g, s = make_pair(n, L=L, precision="mixed", sweeps=sweeps, state=smooth(n, 39, L=L))
    cons0 = g.cons.copy()
    rc, rb, amax, bad = g.rhs()
    grc, grb, gamax = s.rhs()
    assert gamax == pytest.approx(amax, rel=1e-6)
    hmin = min(L[d] / n[d] for d in range(3))
    for got, ref, q, groups in ((grc, rc, cons0, CONS_GROUPS), (grb, rb, g.bf, FACE_GROUPS)):
        for grp in groups:
            floor = np.max(np.abs(q[grp])) * amax / hmin
            assert_parity(got[grp], ref[grp], [list(range(len(grp)))], tol=2e-6, floor=floor,
                          what="mixed rhs (%s sweeps)" % sweeps)
    c, st = cpa_state((32, 32, 32), (1, 0, 0))
    g, s = make_pair((32, 32, 32), precision="mixed", sweeps=sweeps, state=st)
    g.step(20)
    s.step(20)
    p, ref = s.primitives(), g.primitives()
    for grp in PRIM_GROUPS:
        scale = np.max(np.abs(ref[grp]))
        for v in grp:
            assert np.mean(np.abs(p[v] - ref[v])) / scale < 1e-6, (sweeps, v)


@pytest.mark.parametrize("n", [(8, 12, 10), (1024, 4, 3), (1032, 4, 3)])
def test_row_kernel_at_its_limits(n):
    """The mixed path's inversion fused with the x sweep holds a whole row in shared
    memory: the shortest and the longest row it takes (8 and 1024 cells) against the
    oracle, and one cell more than it takes, where the separate kernels run."""
    L = (1.0, 0.5, 0.4)
    g, s = make_pair(n, L=L, precision="mixed", sweeps="fused", state=smooth(n, 44, L=L))
    cons0 = g.cons.copy()
    rc, rb, amax, bad = g.rhs()
    s.profile(True)
    s.profile_read(reset=True)
    grc, grb, gamax = s.rhs()
    prof = s.profile_read(reset=True)
    fused = n[0] <= 1024
    assert (prof.get("c2p_sweep_x", (0, 0.0))[0] == 1) == fused, prof
    assert (prof.get("int_c2p", (0, 0.0))[0] == 1) == (not fused), prof
    assert gamax == pytest.approx(amax, rel=1e-6)
    hmin = min(L[d] / n[d] for d in range(3))
    for got, ref, q, groups in ((grc, rc, cons0, CONS_GROUPS), (grb, rb, g.bf, FACE_GROUPS)):
        for grp in groups:
            floor = np.max(np.abs(q[grp])) * amax / hmin
            assert_parity(got[grp], ref[grp], [list(range(len(grp)))], tol=2e-6, floor=floor,
                          what="mixed rhs, rows of %d" % n[0])


def test_fused_sweep_agrees_with_separate_and_repeats_bit_for_bit():
    """The turbulence at its full amplitude on 96^3, where most warps limit some
    reconstructions: the fused sweep gives the separate kernels' right-hand side to
    FP32 rounding, and exactly the same bits on every repetition (each thread waits
    for every plane it reads, including the first ones of its segment)."""
    n = 96
    tb = wl.Turbulence(n, seed=2401_03008, lorentz_max=5.0)
    st = (tb.prim5(), tb.bface_background(), tb.apot())
    L = (2 * np.pi,) * 3
    out = {}
    for sweeps in ("fused", "separate"):
        s = echo.Solver(n, n, n, L=L, precision="mixed", sweeps=sweeps)
        reps = []
        for rep in range(3):
            s.set_state(*st)
            reps.append(s.rhs())
        s.close()
        for r in reps[1:]:
            assert np.array_equal(r[0], reps[0][0]) and np.array_equal(r[1], reps[0][1])
            assert r[2] == reps[0][2]
        out[sweeps] = reps[0]
    (fc, fb, fa), (sc_, sb, sa) = out["fused"], out["separate"]
    assert fa == pytest.approx(sa, rel=1e-6)
    scale = np.abs(sc_).max(axis=(1, 2, 3)).max()
    assert np.max(np.abs(fc - sc_)) <= 1e-4 * scale
    assert np.max(np.abs(fb - sb)) <= 1e-4 * np.abs(sb).max()
