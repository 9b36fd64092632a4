"""The learned Newton starting guess on the GPU: tensor-core inference and the
training gradients against the FP64 oracle (rounded at the same bf16 points), and
the gain of a trained network over the cold guess, with the Newton result
unchanged."""
import numpy as np
import pytest

from oracle import mlp
from oracle import oracle as orc
from paper_2401_03008_gb300 import echo
from paper_2401_03008_gb300 import workloads as wl
from tests.parity import PRIM_GROUPS, assert_parity

pytestmark = pytest.mark.gpu


def _samples(n, seed):
    prim, B = wl.random_states(n, seed=seed, lorentz_max=5.0, sigma_max=20.0)
    u = np.array([orc.prim2cons(prim[:, q], B[:, q], 4 / 3) for q in range(n)]).T
    v2 = np.sum(prim[1:4] ** 2, axis=0)
    W = (prim[0] + 4 * prim[4]) / (1 - v2)
    return mlp.features(u, B), W / u[4]


def test_forward_matches_oracle():
    import torch
    x, t = _samples(1000, 61)  # not a multiple of 32: ragged last warp
    w = wl.mlp_init(62)
    y = echo.mlp_forward(w, torch.from_numpy(x.astype(np.float32)).cuda()).cpu().numpy()
    # the oracle gets the features the GPU saw (float32) and rounds at the same points.
    # Inference uses the hardware tanh (absolute error about 2^-11 per activation):
    # through the 64 x 64 layer and the output dot product that stays below
    # sum |w3| * 2^-10 plus a bf16 rounding flip or two of the hidden layer
    ref, _ = mlp.forward(w.astype(np.float64), x.astype(np.float32).astype(np.float64), bf=True)
    p = mlp.unpack(w.astype(np.float64))
    bound = np.sum(np.abs(p["w3"])) * 2.0 ** -10 + 2e-3
    assert np.max(np.abs(y - ref)) < bound
    ref64, _ = mlp.forward(w.astype(np.float64), x)
    assert np.max(np.abs(y - ref64)) < 2e-2


def test_gradient_matches_oracle():
    import torch
    x, t = _samples(512, 63)
    w = wl.mlp_init(64)
    xf = x.astype(np.float32)
    loss, g = echo.mlp_grad(w, torch.from_numpy(xf).cuda(),
                            torch.from_numpy(t.astype(np.float32)).cuda())
    lref, gref = mlp.loss_grad(w.astype(np.float64), xf.astype(np.float64),
                               t.astype(np.float32).astype(np.float64), bf=True)
    assert loss == pytest.approx(lref, rel=1e-4)
    assert np.linalg.norm(g - gref) / np.linalg.norm(gref) < 1e-3
    # every parameter block separately
    o = 0
    for name, shape in mlp.SIZES:
        m = int(np.prod(shape))
        gb, rb = g[o:o + m], gref[o:o + m]
        assert np.linalg.norm(gb - rb) <= 1e-3 * np.linalg.norm(rb) + 1e-7, name
        o += m


def test_trained_guess_gains_over_cold_guess():
    """Harvest states from a turbulence run, train on the GPU, and run a turbulence
    field of another seed with the cold, learned and previous-W guesses: the
    learned guess needs fewer Newton iterations than the cold one, and every guess
    gives the same primitives (the iteration runs to tolerance)."""
    import torch
    n = 48
    tb = wl.Turbulence(n, seed=101, lorentz_max=2.0)
    st = (tb.prim5(), tb.bface_background(), tb.apot())
    L = (2 * np.pi,) * 3
    s = echo.Solver(n, n, n, L=L)
    s.set_state(*st)
    cap = 400000
    feats = torch.empty((cap, 5), dtype=torch.float32, device="cuda")
    target = torch.empty(cap, dtype=torch.float32, device="cuda")
    cnt = s.mlp_harvest(10, 8, feats, target)
    assert cnt == min(cap, 10 * 3 * n ** 3 // 8)
    w0 = wl.mlp_init(102)
    w, hist = echo.mlp_train(feats[:cnt].contiguous(), target[:cnt].contiguous(), w0, epochs=6,
                             batch=1024, lr=3e-3, lr_decay=0.7)
    assert hist[-1] < 0.05 * hist[0], hist
    # another seed
    tb2 = wl.Turbulence(n, seed=103, lorentz_max=2.0)
    st2 = (tb2.prim5(), tb2.bface_background(), tb2.apot())
    res = {}
    for guess in ("cold", "mlp", "prev"):
        r = echo.Solver(n, n, n, L=L, guess=guess)
        if guess == "mlp":
            r.mlp_load(w)
        r.set_state(*st2)
        r.step(4)
        d = r.diagnostics()
        res[guess] = (d["newton_it_mean"], d["c2p_fallbacks"], r.primitives())
    assert res["mlp"][0] < res["cold"][0], {k: v[:2] for k, v in res.items()}
    assert res["mlp"][1] < 0.01 * 4 * 3 * n ** 3
    assert_parity(res["mlp"][2], res["prev"][2], PRIM_GROUPS, what="mlp vs prev guess")
    assert_parity(res["cold"][2], res["prev"][2], PRIM_GROUPS, what="cold vs prev guess")


def test_turbulence_parity_with_oracle():
    n = 24
    tb = wl.Turbulence(n, seed=104, lorentz_max=2.0)
    st = (tb.prim5(), tb.bface_background(), tb.apot())
    L = (2 * np.pi,) * 3
    g = orc.Grid(n, n, n, *L)
    g.set_state(*st)
    s = echo.Solver(n, n, n, L=L)
    s.set_state(*st)
    g.step(5)
    s.step(5)
    assert_parity(s.primitives(), g.primitives(), PRIM_GROUPS, what="turbulence 24^3")
