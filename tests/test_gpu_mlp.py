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
    """Tensor-core inference (f16 operands, FP32 accumulation, hardware tanh on f16
    pairs) against the oracle's forward pass rounded at the same points: every
    sample within the worst-case bound of the hardware tanh's error, the mean error
    well inside it (a wrong fragment mapping or layer would be off by O(0.1) on
    most samples); and close to the exact FP64 network."""
    import torch
    x, t = _samples(1000, 61)  # not a multiple of 32: ragged last warp
    for seed in (62, 67):
        w = wl.mlp_init(seed)
        y = echo.mlp_forward(w, torch.from_numpy(x.astype(np.float32)).cuda()).cpu().numpy()
        w64 = w.astype(np.float64)
        ref, _ = mlp.forward_infer(w64, x.astype(np.float32).astype(np.float64))
        err = np.abs(y - ref)
        assert np.max(err) <= mlp.infer_bound(w64), (np.max(err), mlp.infer_bound(w64))
        assert np.mean(err) <= 0.1 * mlp.infer_bound(w64), np.mean(err)
        ref64, _ = mlp.forward(w64, x)
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


def _fp32_features(u, B):
    """The oracle's features of the states the GPU sees, rounded to float32 (the
    GPU forms them in float32 from the rounded components)."""
    return mlp.features(u, B).astype(np.float32).astype(np.float64)


def test_harvest_matches_oracle_features_and_targets():
    """echo_mlp_harvest with stride 1 returns, in cell order, the features of every
    cell and its converged W/U after each inversion.  Stage 1 inverts the initial
    state and stage 2 the state after the first stage update; both are compared
    with the oracle's features (oracle/mlp.features of its own state and INT field)
    and its converged W/U, within float32 rounding."""
    import torch
    n = (20, 12, 9)
    ncell = int(np.prod(n))
    L = (1.0, 0.8, 0.6)
    st = wl.random_smooth_fields(*n, seed=107, amp=0.6, L=L)
    s = echo.Solver(*n, L=L)
    s.set_state(*st)
    cap = 3 * ncell
    feats = torch.empty((cap, 5), dtype=torch.float32, device="cuda")
    target = torch.empty(cap, dtype=torch.float32, device="cuda")
    assert s.mlp_harvest(1, 1, feats, target) == cap
    f = feats.cpu().numpy().astype(np.float64)
    tg = target.cpu().numpy().astype(np.float64)
    g = orc.Grid(*n, *L)
    g.set_state(*st)
    rc, rb, amax, bad, prim = g.rhs(with_prims=True)
    assert bad == 0
    checks = [(g.cons.reshape(5, -1).copy(), prim[5:8].reshape(3, -1).copy(), g.W.reshape(-1).copy())]
    dt = 0.4 * min(L[q] / n[q] for q in range(3)) / amax
    g.cons = np.ascontiguousarray(g.cons + dt * rc)
    g.bf = np.ascontiguousarray(g.bf + dt * rb)
    rc2, rb2, _, bad2, prim2 = g.rhs(with_prims=True)
    assert bad2 == 0
    checks.append((g.cons.reshape(5, -1).copy(), prim2[5:8].reshape(3, -1).copy(),
                   g.W.reshape(-1).copy()))
    for stage, (u, B, W) in enumerate(checks):
        got = f[stage * ncell:(stage + 1) * ncell]
        ref = mlp.features(u, B)
        assert np.all(np.abs(got - ref) <= 2e-6 * np.maximum(1.0, np.abs(ref))), stage
        assert np.all(np.abs(got[:, 3] - ref[:, 3]) <= 1e-5), stage
        tref = W / u[4]
        assert np.allclose(tg[stage * ncell:(stage + 1) * ncell], tref, rtol=2e-7, atol=0), stage


def _trained_weights(n=32, seed=108, steps=6):
    """A network trained on the GPU on states harvested from a turbulence run."""
    import torch
    tb = wl.Turbulence(n, seed=seed, lorentz_max=3.0)
    L = (2 * np.pi,) * 3
    h = echo.Solver(n, n, n, L=L)
    h.set_state(tb.prim5(), tb.bface_background(), tb.apot())
    cap = steps * 3 * n ** 3 // 2
    feats = torch.empty((cap, 5), dtype=torch.float32, device="cuda")
    target = torch.empty(cap, dtype=torch.float32, device="cuda")
    cnt = h.mlp_harvest(steps, 2, feats, target)
    h.close()
    w, hist = echo.mlp_train(feats[:cnt].contiguous(), target[:cnt].contiguous(),
                             wl.mlp_init(seed + 1), epochs=6, batch=1024, lr=3e-3, lr_decay=0.7)
    return w


def test_in_step_guess_matches_oracle():
    """The learned guess the inversion starts from, W0 = U y: echo_mlp_guess (the
    device feature map and the tensor-core network) against U times the oracle's
    forward pass on the oracle's features, within the hardware-tanh bound; then one
    right-hand-side evaluation with the network selected against the oracle run
    with exactly these guesses as its caller array: the same Newton iterations and
    the same rejected guesses, so the guess computed inside the inversion kernel is
    the one echo_mlp_guess returns."""
    w = _trained_weights()
    n = (24, 24, 24)
    L = (2 * np.pi,) * 3
    tb = wl.Turbulence(24, seed=109, lorentz_max=3.0)
    st = (tb.prim5(), tb.bface_background(), tb.apot())
    s = echo.Solver(*n, L=L, guess="mlp")
    s.mlp_load(w)
    s.set_state(*st)
    w0 = s.mlp_guess()
    g = orc.Grid(*n, *L)
    g.set_state(*st)
    _, _, _, _, prim = g.rhs(with_prims=True)   # the INT field of the state
    u = g.cons.reshape(5, -1)
    x = _fp32_features(u, prim[5:8].reshape(3, -1))
    y, _ = mlp.forward_infer(w.astype(np.float64), x)
    bound = mlp.infer_bound(w.astype(np.float64))
    err = np.abs(w0.reshape(-1) - u[4] * y)
    assert np.all(err <= u[4] * bound + 1e-6 * np.abs(w0.reshape(-1)))
    assert np.mean(err / u[4]) <= 0.1 * bound
    # the oracle from the same state with these guesses
    g2 = orc.Grid(*n, *L, guess=orc.GUESS_ARRAY)
    g2.set_state(*st)
    g2.guessarr = np.ascontiguousarray(w0)
    rc, rb, amax, bad = g2.rhs()
    s.diagnostics(reset=True)
    grc, grb, gamax = s.rhs()
    d = s.diagnostics()
    assert d["c2p_calls"] == g2.stats.cells
    assert round(d["newton_it_mean"] * d["c2p_calls"]) == g2.stats.iters
    assert d["c2p_fallbacks"] == g2.stats.fallbacks
    assert gamax == pytest.approx(amax, rel=1e-13)


def test_adam_steps_match_oracle():
    """Training on one batch of 64 states: each epoch is one Adam step.  The GPU's
    parameters after one and after two steps equal the oracle's Adam update
    (oracle/mlp.adam_step, pinned by a hand-computed case) applied to the GPU's own
    gradient at the previous parameters, to float32 rounding."""
    import torch
    x, t = _samples(64, 65)
    xf = torch.from_numpy(x.astype(np.float32)).cuda()
    tf = torch.from_numpy(t.astype(np.float32)).cuda()
    w0 = wl.mlp_init(66)
    lr = 1e-2
    w1, _ = echo.mlp_train(xf, tf, w0, epochs=1, batch=64, lr=lr, lr_decay=1.0)
    w2, _ = echo.mlp_train(xf, tf, w0, epochs=2, batch=64, lr=lr, lr_decay=1.0)
    _, g0 = echo.mlp_grad(w0, xf, tf)
    ref1, m1, v1 = mlp.adam_step(w0.astype(np.float64), g0, np.zeros(mlp.NPARAM),
                                 np.zeros(mlp.NPARAM), 1, lr)
    assert np.max(np.abs(w1 - ref1)) < 1e-6
    # each parameter moved by about lr on the first step (mhat / sqrt(vhat) = sign g)
    moved = np.abs(w1 - w0)[np.abs(g0) > 1e-6]
    assert np.all(np.abs(moved - lr) < 1e-4)
    _, g1 = echo.mlp_grad(w1, xf, tf)
    ref2, _, _ = mlp.adam_step(w1.astype(np.float64), g1, m1, v1, 2, lr)
    assert np.max(np.abs(w2 - ref2)) < 2e-6


def test_learned_guess_pays_on_a_resume_without_w():
    """A checkpoint resumed without its Newton guess W has no previous solution: the
    method without the network starts every cell's first inversion from W0 = U.
    With a network trained on 9.4e6 states of the same workload family (another seed)
    loaded, that inversion starts from the learned guess instead: fewer Newton
    iterations, less inversion time (the best of four resumes each, FP64 path), and
    the same primitives (the iteration runs to tolerance either way)."""
    import torch
    L = (2 * np.pi,) * 3

    def turb(m, seed):
        tb = wl.Turbulence(m, seed=seed, lorentz_max=5.0, device="cuda")
        return (tb.prim5(), tb.bface_background(), tb.apot())

    h = echo.Solver(128, 128, 128, L=L)
    h.set_state(*turb(128, 112))
    cap = 10_000_000
    feats = torch.empty((cap, 5), dtype=torch.float32, device="cuda")
    target = torch.empty(cap, dtype=torch.float32, device="cuda")
    cnt = h.mlp_harvest(12, 8, feats, target)
    h.close()
    w, hist = echo.mlp_train(feats[:cnt].contiguous(), target[:cnt].contiguous(),
                             wl.mlp_init(113), epochs=4, batch=4096, lr=3e-3, lr_decay=0.6)
    del feats, target
    n = 128
    a = echo.Solver(n, n, n, L=L)
    a.set_state(*turb(n, 114))
    a.step(3)
    cons, bf, _, t, step = a.get_state(device=True)
    a.close()
    res = {}
    for name in ("cold", "learned"):
        r = echo.Solver(n, n, n, L=L)
        if name == "learned":
            r.mlp_load(w)
        times, its = [], []
        for rep in range(4):
            r.set_conserved(cons, bf, None, t, step)
            r.diagnostics(reset=True)
            r.profile(True)
            r.profile_read(reset=True)
            r.rhs(device=True)
            prof = r.profile_read(reset=True)
            r.profile(False)
            d = r.diagnostics()
            times.append(prof["int_c2p"][1])
            its.append((d["newton_it_mean"], d["c2p_fallbacks"]))
        res[name] = (min(times), its[-1][0], its[-1][1], r.primitives())
        r.close()
    summary = {k: v[:3] for k, v in res.items()}
    assert res["learned"][1] < res["cold"][1], summary
    assert res["learned"][2] < 0.01 * n ** 3, summary
    assert res["learned"][0] < res["cold"][0], summary
    assert_parity(res["learned"][3], res["cold"][3], PRIM_GROUPS, what="learned vs cold restart")


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_turbulence_lorentz5_parity_with_oracle(precision):
    """The benchmark's turbulence at its full amplitude (largest Lorentz factor 5,
    sigma0 = 10) on 64^3, the coarsest grid on which the oracle's first steps run
    clean: 5 SSP-RK3 steps, FP64 element by element at the 1e-10 bar, the mixed
    path within its L1 bound (1e-6 of each field's scale)."""
    n = 64
    tb = wl.Turbulence(n, seed=111, lorentz_max=5.0)
    st = (tb.prim5(), tb.bface_background(), tb.apot())
    L = (2 * np.pi,) * 3
    g = orc.Grid(n, n, n, *L)
    g.set_state(*st)
    assert g.step(5) == 0
    s = echo.Solver(n, n, n, L=L, precision=precision)
    s.set_state(*st)
    done, t = s.step(5)
    # the mixed path takes the speed maximum (hence dt) in FP32
    assert done == 5 and t == pytest.approx(g.t, rel=1e-12 if precision == "fp64" else 1e-6)
    p, ref = s.primitives(), g.primitives()
    if precision == "fp64":
        assert_parity(p, ref, PRIM_GROUPS, what="turbulence, Lorentz factor 5, 64^3")
    else:
        for grp in PRIM_GROUPS:
            scale = np.max(np.abs(ref[grp]))
            for v in grp:
                assert np.mean(np.abs(p[v] - ref[v])) / scale < 1e-6, v
    d = s.diagnostics()
    assert d["c2p_failures"] == 0
