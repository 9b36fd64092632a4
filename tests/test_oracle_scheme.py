"""Pins of the oracle's grid-level scheme: brute force on tiny grids, the exact time
derivative of the Alfven wave, conservation, div B, and convergence order."""
import math

import numpy as np
import pytest

from oracle import oracle as orc
from paper_2401_03008_gb300 import workloads as wl
from tests.bruteforce import BruteRHS

GAM = 4.0 / 3.0


def smooth_grid(nx, ny, nz, seed, ho=1, L=(1.0, 1.0, 1.0)):
    prim, bg, apot = wl.random_smooth_fields(nx, ny, nz, seed=seed, L=L)
    g = orc.Grid(nx, ny, nz, *L, ho=ho)
    g.set_state(prim, bg, apot)
    return g


def cpa_grid(n, m, ho=1, t=0.0, **kw):
    nx, ny, nz = n
    cpa = wl.CPA(nx, ny, nz, m=m, **kw)
    g = orc.Grid(nx, ny, nz, ho=ho)
    g.set_state(cpa.prim5(t), cpa.bface_background(), cpa.apot(t))
    return g, cpa


@pytest.mark.parametrize("ho", [0, 1])
def test_brute_force_rhs(ho):
    """The oracle's L(U) equals a naive per-output evaluation on a 5x4x3 grid
    (unequal sizes catch swapped axes; the 6-point stencils wrap around)."""
    g = smooth_grid(5, 4, 3, seed=21, ho=ho, L=(1.0, 0.8, 0.6))
    W0 = g.W.copy()
    rc, rb, amax, bad, prim = g.rhs(with_prims=True)
    assert bad == 0 and g.stats.rec_fallbacks == 0
    br = BruteRHS(g.cons, g.bf, W0, L=(1.0, 0.8, 0.6), ho=ho)
    scale_c = np.max(np.abs(rc), axis=(1, 2, 3)) + 1e-300
    scale_b = np.max(np.abs(rb)) + 1e-300
    for k in range(3):
        for j in range(4):
            for i in range(5):
                pos = (i, j, k)
                assert np.allclose(br.prim(pos), prim[:, k, j, i], rtol=0, atol=1e-14)
                got = rc[:, k, j, i]
                np.testing.assert_allclose(br.rhs_cell(pos), got, rtol=0,
                                           atol=1e-13 * scale_c.max())
                for a in range(3):
                    assert abs(br.rhs_face(a, pos) - rb[a, k, j, i]) <= 1e-13 * scale_b
    amax_b = max(max(f[1], f[2]) for f in br._face.values())
    assert amax == amax_b


@pytest.mark.parametrize("ho", [0, 1])
def test_initial_field_divergence_free(ho):
    """B = background + curl A has zero discrete divergence with the same DER."""
    g = smooth_grid(7, 6, 5, seed=22, ho=ho)
    bmax = np.max(np.abs(g.bf))
    h = 1.0 / 7
    assert np.max(np.abs(g.divb())) <= 1e-13 * bmax / h


def _dxi(fun, xi, d=1e-3):
    """fourth-order central difference in the phase"""
    return (-fun(xi + 2 * d) + 8 * fun(xi + d) - 8 * fun(xi - d) + fun(xi - 2 * d)) / (12 * d)


def _exact_rates(cpa, shape):
    """d/dt of the conserved cell variables and of the face field on the exact wave."""
    nz, ny, nx = shape
    w = -cpa.kmag * cpa.vA  # dU/dt = w dU/dxi

    def phase(off):
        x = (np.arange(nx) + off[0]) / nx * cpa.L[0]
        y = (np.arange(ny) + off[1]) / ny * cpa.L[1]
        z = (np.arange(nz) + off[2]) / nz * cpa.L[2]
        X, Y, Z = np.meshgrid(x, y, z, indexing="ij")
        return (cpa.k[0] * X + cpa.k[1] * Y + cpa.k[2] * Z).transpose(2, 1, 0)

    xi = phase((0.5, 0.5, 0.5)).ravel()

    def cons_of(xs):
        prim, B = cpa.state_along(xs)
        return np.array([orc.prim2cons(prim[:, q], B[:, q], GAM) for q in range(xs.size)]).T

    rc = w * _dxi(cons_of, xi).reshape((5,) + shape)
    rb = np.empty((3,) + shape)
    offs = [(1.0, 0.5, 0.5), (0.5, 1.0, 0.5), (0.5, 0.5, 1.0)]
    for a in range(3):
        xa = phase(offs[a])
        dB = cpa.eta * cpa.B0 * (-cpa.Y[a] * np.sin(xa) + cpa.Z[a] * np.cos(xa))
        rb[a] = w * dB
    return rc, rb


def test_rhs_converges_to_exact_time_derivative():
    """L(U) on the sampled wave approaches the exact dU/dt (a traveling profile:
    dU/dt = -|k| v_A dU/dxi) at high order: every term, sign and index of the
    right-hand side takes part."""
    errs = []
    for n in (16, 32, 64):
        g, cpa = cpa_grid((n, n, 1), m=(1, 1, 0))
        rc, rb, amax, bad = g.rhs()
        ec, eb = _exact_rates(cpa, g.shape)
        err = max(np.max(np.abs(rc - ec)), np.max(np.abs(rb - eb)))
        errs.append(err)
    orders = [math.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert orders[-1] > 3.5, (errs, orders)
    assert errs[-1] < 1e-4


def test_conservation_and_divb_over_steps():
    """Periodic fluxes telescope (totals of D, S, U and face B conserved) and UCT
    keeps the discrete divergence at round-off."""
    g = smooth_grid(8, 6, 5, seed=23)
    t0 = g.totals()
    assert g.step(3) == 0
    t1 = g.totals()
    scale = np.abs(g.cons).sum(axis=(1, 2, 3)).max()
    assert np.max(np.abs(t1 - t0)) <= 1e-13 * scale
    bmax = np.max(np.abs(g.bf))
    assert np.max(np.abs(g.divb())) <= 1e-12 * bmax * 8


@pytest.mark.parametrize("m,n", [((1, 0, 0), (16, 1, 1)), ((0, 1, 0), (1, 16, 1)),
                                 ((0, 0, 1), (1, 1, 16))])
def test_axis_waves_agree(m, n):
    """The same 1-D wave along x, y and z gives the same numbers (with the
    components permuted), so no direction is treated differently."""
    g, cpa = cpa_grid(n, m)
    g.step(5)
    p = g.primitives()
    d = m.index(1)
    line = np.moveaxis(p, 3 - d, -1).reshape(8, -1)
    if not hasattr(test_axis_waves_agree, "ref"):
        test_axis_waves_agree.ref = {}
    test_axis_waves_agree.ref[d] = (line, g.dts)
    if len(test_axis_waves_agree.ref) == 3:
        (l0, dt0), (l1, dt1), (l2, dt2) = (test_axis_waves_agree.ref[q] for q in range(3))
        assert np.allclose(dt0, dt1, rtol=1e-14) and np.allclose(dt0, dt2, rtol=1e-14)
        assert np.allclose(l0[0], l1[0], atol=1e-13) and np.allclose(l0[0], l2[0], atol=1e-13)


def _l1_after_period(n, m):
    g, cpa = cpa_grid(n, m)
    g.step(100000, t_end=cpa.period)
    assert abs(g.t - cpa.period) < 1e-13
    p = g.primitives()
    ex = cpa.exact_prim8(g.t)
    return np.mean(np.abs(p - ex), axis=(1, 2, 3))


def test_convergence_order_one_period():
    """After one period the wave must be back at its initial state, with an L1
    error that falls faster than second order as h -> 0 (dt proportional to h,
    so the third-order Runge-Kutta error ends up dominating)."""
    errs = [_l1_after_period((n, 1, 1), (1, 0, 0)) for n in (16, 32, 64)]
    e = [np.max(x[1:4]) for x in errs]
    order = math.log2(e[1] / e[2])
    assert order > 2.5, (e, order)
    assert e[2] < 1e-4


@pytest.mark.slow
def test_convergence_order_oblique():
    errs = [_l1_after_period((n, n, 1), (1, 1, 0)) for n in (8, 16, 32)]
    e = [np.max(x[1:4]) for x in errs]
    assert math.log2(e[1] / e[2]) > 2.5, e


def test_c2p_failure_counted():
    g = smooth_grid(4, 4, 4, seed=24)
    g.cons[4, 0, 0, 0] = 0.1 * g.cons[0, 0, 0, 0]   # energy below rest mass
    rc, rb, amax, bad = g.rhs()
    assert bad == 1 and g.stats.failures >= 1


def _cpa_cell_grid(n, m, ho):
    nx, ny, nz = n
    cpa = wl.CPA(nx, ny, nz, m=m)
    g = orc.Grid(nx, ny, nz, uct=0, ho=ho)
    g.set_state(cpa.prim5(), cpa.bcell())
    return g, cpa


@pytest.mark.parametrize("ho", [0, 1])
def test_cell_centred_variant_converges_and_conserves(ho):
    """UCT off (Sec. 3: the field is then cell-centred like the other variables and
    all 8 components take the HLL flux): the right-hand side approaches the exact
    time derivative of the wave, and the totals are conserved."""
    errs = []
    for n in (16, 32, 64):
        g, cpa = _cpa_cell_grid((n, n, 1), (1, 1, 0), ho)
        rc, rb, amax, bad = g.rhs()
        ec, _ = _exact_rates(cpa, g.shape)
        w = -cpa.kmag * cpa.vA
        X = (np.arange(n) + 0.5) / n
        xi = (cpa.k[0] * X[None, :] + cpa.k[1] * X[:, None])[None]
        eb = np.array([w * cpa.eta * cpa.B0 * (-cpa.Y[a] * np.sin(xi) + cpa.Z[a] * np.cos(xi))
                       for a in range(3)])
        errs.append(max(np.max(np.abs(rc - ec)), np.max(np.abs(rb - eb))))
    order = math.log2(errs[1] / errs[2])
    assert order > (1.8 if ho == 0 else 3.5), (errs, order)
    g, cpa = _cpa_cell_grid((8, 6, 5), (1, 1, 1), ho)
    t0 = g.totals()
    assert g.step(3) == 0
    scale = np.abs(g.cons).sum(axis=(1, 2, 3)).max()
    assert np.max(np.abs(g.totals() - t0)) <= 1e-13 * scale


def test_fast_variant_second_order():
    """Linear reconstruction with SSP-RK2 (the faster variant of Sec. 4): second
    order on the wave, conservative."""
    errs = []
    for n in (32, 64, 128):
        cpa = wl.CPA(n, 1, 1, m=(1, 0, 0))
        g = orc.Grid(n, 1, 1, rec=1, rk=2)
        g.set_state(cpa.prim5(), cpa.bface_background(), cpa.apot())
        g.step(100000, t_end=0.25 * cpa.period)
        p = g.primitives()
        errs.append(np.max(np.mean(np.abs(p - cpa.exact_prim8(g.t)), axis=(1, 2, 3))[1:4]))
    order = math.log2(errs[1] / errs[2])
    assert 1.6 < order < 3.0, (errs, order)
    g = orc.Grid(8, 6, 5, rec=1, rk=2)
    prim, bg, apot = wl.random_smooth_fields(8, 6, 5, seed=25)
    g.set_state(prim, bg, apot)
    t0 = g.totals()
    assert g.step(3) == 0
    scale = np.abs(g.cons).sum(axis=(1, 2, 3)).max()
    assert np.max(np.abs(g.totals() - t0)) <= 1e-13 * scale
    assert np.max(np.abs(g.divb())) <= 1e-12 * np.abs(g.bf).max() * 8
