"""The 2.5-D turbulence set-up of Sec. 5 and the isotropised spectra of Fig. 5:
the printed parameters, the a-posteriori amplitude normalisation, the solenoidal
fluctuations, and the shell spectrum against closed forms."""
import math
import os

import numpy as np
import pytest

from oracle import oracle as orc
from paper_2401_03008_gb300 import spectra
from paper_2401_03008_gb300 import workloads as wl


def _golden(golden_dir):
    out = {}
    with open(os.path.join(golden_dir, "paper_printed_values.txt")) as f:
        for line in f:
            line = line.split("#")[0].strip()
            if line:
                k, v = line.split("=")
                out[k.strip()] = float(v)
    return out


def test_background_matches_printed_values(golden_dir):
    g = _golden(golden_dir)
    tb = wl.Turbulence2D(32, seed=1)
    assert tb.B0 == g["turb.B0"] and tb.p0 == g["turb.p0"] and tb.rho0 == g["turb.rho0"]
    assert abs(tb.vA - g["turb.vA"]) < 0.01
    p = tb.prim5()
    assert np.all(p[0] == 1.0) and np.all(p[4] == 50.0) and np.all(p[3] == 0.0)
    assert np.all(tb.bface_background()[2] == 10.0)


def test_mode_set_is_the_disc_of_radius_four():
    """kx = 0..4, ky = -4..4, 1 <= |k| <= 4 (Sec. 5): 28 wave vectors; the phases
    of v and B differ."""
    tb = wl.Turbulence2D(32, seed=2)
    ks = {tuple(map(int, k)) for k in tb.modes}
    ref = {(kx, ky) for kx in range(5) for ky in range(-4, 5) if 1 <= kx * kx + ky * ky <= 16}
    assert ks == ref and len(ks) == len(tb.modes) == 28
    assert not np.allclose(tb.phv, tb.phB)


@pytest.mark.parametrize("n", [32, 64])
def test_amplitudes_normalised_and_solenoidal(n):
    """<|dv|>/v_A = <|dB|>/B0 = 0.25 over the grid (the field measured after the
    discrete curl at the cell centres), div v = 0 mode by mode, discrete div B at
    round-off, and all fluctuation energy at 1 <= |k| <= 4."""
    tb = wl.Turbulence2D(n, seed=3)
    p = tb.prim5()
    dv = np.sqrt(p[1, 0] ** 2 + p[2, 0] ** 2)
    assert dv.mean() / tb.vA == pytest.approx(0.25, rel=1e-12)
    g = orc.Grid(n, n, 1, *tb.L)
    g.set_state(p, tb.bface_background(), tb.apot())
    q = g.primitives()
    dB = np.sqrt(q[5, 0] ** 2 + q[6, 0] ** 2)
    # the discrete curl and INT of the staggered field against the pointwise
    # sample: a 4th-order difference, 3.2e-4 at 32^2 for |k| h up to 0.79
    assert dB.mean() / tb.B0 == pytest.approx(0.25, rel=4e-4 * (32 / n) ** 4)
    assert np.max(np.abs(q[7] - tb.B0)) < 1e-12
    assert np.max(np.abs(g.divb())) < 1e-11 * tb.B0 * n
    vx, vy = (np.fft.fft2(p[c, 0]) for c in (1, 2))
    kk = np.fft.fftfreq(n) * n
    div = kk[None, :] * vx + kk[:, None] * vy
    assert np.max(np.abs(div)) < 1e-10 * np.max(np.abs(vx))
    k, E = spectra.shell_spectrum([p[1, 0], p[2, 0]])
    assert np.sum(E[5:]) < 1e-24 * np.sum(E) and E[0] < 1e-24 * np.sum(E)


def test_shell_spectrum_single_mode_and_parseval():
    """a cos(k.x) puts a^2/2 in the shell round(|k|); the shells hold the variance
    of a band-limited field (Parseval)."""
    n = 64
    x = 2 * np.pi * np.arange(n) / n
    X, Y = np.meshgrid(x, x, indexing="xy")
    f = 0.7 * np.cos(3 * X + 4 * Y + 0.3)
    k, E = spectra.shell_spectrum([f])
    assert E[5] == pytest.approx(0.49 / 2, rel=1e-12)
    assert np.sum(E) - E[5] < 1e-28
    rng = np.random.default_rng(4)
    F = np.fft.fft2(rng.normal(size=(n, n)))
    kk = np.sqrt((np.fft.fftfreq(n) * n)[None, :] ** 2 + (np.fft.fftfreq(n) * n)[:, None] ** 2)
    F[kk > n // 2 - 1] = 0
    g = np.fft.ifft2(F).real
    k, E = spectra.shell_spectrum([g, 2 * g])
    assert np.sum(E) == pytest.approx(5 * np.var(g), rel=1e-12)


def test_spectrum_slope_of_a_synthetic_power_law():
    """Random-phase modes with |f_k| proportional to |k|^-a fill shells of about
    2 pi k modes each, so E(k) ~ k^(1 - 2a): a = 4/3 gives the -5/3 slope."""
    n = 256
    rng = np.random.default_rng(5)
    kx = np.fft.fftfreq(n) * n
    kk = np.sqrt(kx[None, :] ** 2 + kx[:, None] ** 2)
    amp = np.where(kk > 0, np.maximum(kk, 1) ** (-4.0 / 3.0), 0.0)
    F = amp * np.exp(2j * np.pi * rng.uniform(size=(n, n)))
    f = np.fft.ifft2(F).real
    k, E = spectra.shell_spectrum([f])
    assert spectra.slope(k, E, 8, 96) == pytest.approx(-5.0 / 3.0, abs=0.05)


def test_oracle_run_keeps_the_invariants():
    """One time unit of the oracle on 32^2: totals conserved, div B at round-off,
    the fluctuations decay slowly (no blow-up), no failed inversion."""
    n = 32
    tb = wl.Turbulence2D(n, seed=6)
    g = orc.Grid(n, n, 1, *tb.L, nthreads=4)
    g.set_state(tb.prim5(), tb.bface_background(), tb.apot())
    t0 = g.totals()
    assert g.step(100000, t_end=1.0) == 0 and g.stats.failures == 0
    assert abs(g.t - 1.0) < 1e-13
    scale = np.abs(g.cons).sum(axis=(1, 2, 3)).max()
    assert np.max(np.abs(g.totals() - t0)) <= 1e-12 * scale
    assert np.max(np.abs(g.divb())) < 1e-10 * tb.B0 * n
    q = g.primitives()
    dB = np.sqrt(q[5, 0] ** 2 + q[6, 0] ** 2).mean() / tb.B0
    assert 0.15 < dB < 0.35 and math.isfinite(dB)
