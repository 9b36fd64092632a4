"""Pins of the MLP oracle: backpropagation against finite differences, the bfloat16
rounding against torch, and the invariances the features must have."""
import numpy as np
import pytest

from oracle import mlp
from oracle import oracle as orc
from paper_2401_03008_gb300 import workloads as wl


def _batch(n, seed):
    prim, B = wl.random_states(n, seed=seed, lorentz_max=5.0, sigma_max=20.0)
    u = np.array([orc.prim2cons(prim[:, q], B[:, q], 4 / 3) for q in range(n)]).T
    v2 = np.sum(prim[1:4] ** 2, axis=0)
    W = (prim[0] + 4 * prim[4]) / (1 - v2)
    return u, B, W


def test_gradient_matches_finite_differences():
    u, B, W = _batch(40, 51)
    x = mlp.features(u, B)
    t = W / u[4]
    theta = wl.mlp_init(52).astype(np.float64)
    loss, g = mlp.loss_grad(theta, x, t)
    rng = np.random.default_rng(53)
    for i in rng.choice(mlp.NPARAM, 60, replace=False).tolist() + [mlp.NPARAM - 1, 0]:
        e = np.zeros(mlp.NPARAM)
        h = 1e-6
        e[i] = h
        lp, _ = mlp.loss_grad(theta + e, x, t)
        lm, _ = mlp.loss_grad(theta - e, x, t)
        fd = (lp - lm) / (2 * h)
        assert g[i] == pytest.approx(fd, rel=1e-6, abs=1e-10), i


def test_bf16_rounding_matches_torch():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(54)
    x = np.concatenate([rng.normal(size=5000) * 10.0 ** rng.uniform(-8, 8, 5000),
                        np.array([0.0, -0.0, 1.0, 1.00390625, 1.01171875, 65504.0])])
    ref = torch.from_numpy(x.astype(np.float32)).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(mlp.bf16(x), ref)


def test_features_invariant_under_rotation_and_scaling():
    u, B, W = _batch(50, 55)
    x = mlp.features(u, B)
    th = 0.7
    R = np.array([[np.cos(th), -np.sin(th), 0], [np.sin(th), np.cos(th), 0], [0, 0, 1.0]])
    u2 = u.copy()
    u2[1:4] = R @ u[1:4]
    B2 = R @ B
    assert np.allclose(mlp.features(u2, B2), x, rtol=1e-12, atol=1e-14)
    # energy densities scale by lam, B by sqrt(lam): the features do not change
    lam = 3.7
    u3 = u * lam
    assert np.allclose(mlp.features(u3, B * np.sqrt(lam)), x, rtol=1e-12, atol=1e-14)
    assert np.all((x[:, 3] >= 0) & (x[:, 3] <= 1)) and np.all(x[:, 0] > 0)


def test_bf16_emulation_is_close_to_fp64():
    u, B, W = _batch(256, 56)
    x = mlp.features(u, B)
    t = W / u[4]
    theta = wl.mlp_init(57).astype(np.float64)
    l64, g64 = mlp.loss_grad(theta, x, t)
    lbf, gbf = mlp.loss_grad(theta, x, t, bf=True)
    assert abs(lbf - l64) / l64 < 1e-2
    assert np.linalg.norm(gbf - g64) / np.linalg.norm(g64) < 2e-2


def test_adam_step_hand_computed():
    """Two Adam steps on three parameters, worked by hand (lr 0.01, beta1 0.9,
    beta2 0.999, eps 1e-8).  Step 1, g = (0.1, -0.2, 0): m = 0.1 g, v = 0.001 g^2,
    so the bias-corrected mhat = g and vhat = g^2, and each parameter moves by
    lr g / (|g| + eps): 0.01 * 0.1 / 0.10000001 = 0.0099999990000001 and
    0.01 * 0.2 / 0.20000001 = 0.0099999995; the parameter with g = 0 stays.
    Step 2, g = (0.05, 0.1, -0.3): m = (0.014, -0.008, -0.03),
    v = (1.249e-5, 4.996e-5, 9.0e-5); mhat = m / 0.19 = (0.0736842105, -0.0421052632,
    -0.1578947368), vhat = v / 0.001999 = (0.0062481241, 0.0249924962,
    0.0450225113); the updates lr mhat / (sqrt(vhat) + eps) give the values below
    (decimal arithmetic to 30 digits)."""
    theta = np.array([1.0, 2.0, 3.0])
    m = v = np.zeros(3)
    theta, m, v = mlp.adam_step(theta, [0.1, -0.2, 0.0], m, v, 1, 0.01)
    assert np.allclose(m, [0.01, -0.02, 0.0], rtol=1e-14, atol=0)
    assert np.allclose(v, [1e-5, 4e-5, 0.0], rtol=1e-14, atol=0)
    assert np.allclose(theta, [0.9900000009999999, 2.0099999995, 3.0], rtol=1e-15, atol=0)
    theta, m, v = mlp.adam_step(theta, [0.05, 0.1, -0.3], m, v, 2, 0.01)
    assert np.allclose(theta, [0.9806782057911869, 2.0126633697281324, 3.0074413678849681],
                       rtol=1e-14, atol=0)


def test_f16_rounding_and_inference_model():
    """The f16 rounding of the inference model is IEEE half, round to nearest even
    (1 + 2^-11 is a tie that rounds to 1, 1 + 3 * 2^-11 rounds up to 1 + 2^-9, the
    largest half is 65504), and the rounded forward pass stays within the rounding
    it models of the exact FP64 network."""
    assert mlp.f16(1.0 + 2.0 ** -11) == 1.0
    assert mlp.f16(1.0 + 3 * 2.0 ** -11) == 1.0 + 2.0 ** -9
    assert mlp.f16(65504.0) == 65504.0 and mlp.f16(-0.1) == np.float16(-0.1)
    u, B, W = _batch(200, 54)
    x = mlp.features(u, B)
    theta = wl.mlp_init(55).astype(np.float64)
    y, _ = mlp.forward(theta, x)
    yi, (h1, h2) = mlp.forward_infer(theta, x)
    assert np.all(np.abs(h1) <= 1.0) and np.all(np.abs(h2) <= 1.0)
    assert np.array_equal(h1, mlp.f16(h1)) and np.array_equal(h2, mlp.f16(h2))
    assert 0.0 < np.max(np.abs(yi - y)) < 5e-3
