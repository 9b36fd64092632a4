"""FP64 oracle of the learned Newton starting guess (test infrastructure only).

The paper has no learned component; this follows the project's definition of it.
Network: 5 -> 64 -> 64 -> 1, tanh on both hidden layers, linear output.
Parameters (one flat float vector, 4609 values): W1[64][5], b1[64], W2[64][64],
b2[64], w3[64], b3.  Input: five rotation-invariant, dimensionless features of a
cell's conserved state; output: W/U (W = rho h G^2), so the guess is W0 = U * y.
Loss: mean squared error of y against the converged W/U.

bf16=True rounds, as the GPU does, the operands of the three products that run on
tensor cores to bfloat16 (round to nearest even): h1 and W2 in the forward layer-2
product, dz2 and h1 in the W2 gradient, dz2 and W2 in the h1 gradient.  Everything
else is FP64.
"""
import numpy as np

NIN, NH = 5, 64
SIZES = [("W1", (NH, NIN)), ("b1", (NH,)), ("W2", (NH, NH)), ("b2", (NH,)), ("w3", (NH,)),
         ("b3", (1,))]
NPARAM = sum(int(np.prod(s)) for _, s in SIZES)


def unpack(theta):
    out, o = {}, 0
    for name, shape in SIZES:
        m = int(np.prod(shape))
        out[name] = np.asarray(theta[o:o + m], dtype=np.float64).reshape(shape)
        o += m
    return out


def pack(p):
    return np.concatenate([np.asarray(p[name], dtype=np.float64).ravel() for name, _ in SIZES])


def bf16(x):
    """Round to bfloat16 (nearest even) and back to float64."""
    f = np.asarray(x, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def features(u, B):
    """u[5, n] = D, Sx, Sy, Sz, U; B[3, n] cell-centred field -> x[n, 5]:
    D/U, S^2/U^2, B^2/U, (S.B)^2/(S^2 B^2) (0 when S or B vanish), ln(U/D)."""
    D, S, U = u[0], u[1:4], u[4]
    S2 = np.sum(S * S, axis=0)
    B2 = np.sum(B * B, axis=0)
    SB = np.sum(S * B, axis=0)
    den = S2 * B2
    cos2 = np.where(den > 0, SB * SB / np.where(den > 0, den, 1.0), 0.0)
    return np.stack([D / U, S2 / (U * U), B2 / U, cos2, np.log(U / D)], axis=1)


def f16(x):
    """Round to IEEE half precision (nearest even) and back to float64."""
    return np.asarray(x, dtype=np.float64).astype(np.float16).astype(np.float64)


def forward(theta, x, bf=False):
    p = unpack(theta)
    r = bf16 if bf else (lambda a: a)
    z1 = x @ p["W1"].T + p["b1"]
    h1 = np.tanh(z1)
    z2 = r(h1) @ r(p["W2"]).T + p["b2"]
    h2 = np.tanh(z2)
    y = h2 @ p["w3"] + p["b3"][0]
    return y, (x, z1, h1, z2, h2)


def split16(a):
    """a = hi + lo with hi the f16 rounding of a and lo the f16 rounding of the rest."""
    hi = f16(a)
    return hi, f16(np.asarray(a, dtype=np.float64) - hi)


def forward_infer(theta, x):
    """The forward pass as the GPU's inference runs it, on f16 operands with exact
    accumulation: layer 1 from the split features and weights (x = xh + xl,
    W1 = Wh + Wl) as xh Wh + xl Wh + xh Wl; each tanh taken on the f16-rounded
    pre-activation and returned in f16; layer 2 on f16 W2; the output from the
    split w3 = hi + lo; the biases exact.  Returns y and the two hidden layers."""
    p = unpack(theta)
    xh, xl = split16(np.asarray(x, dtype=np.float64).astype(np.float32))
    Wh, Wl = split16(np.asarray(p["W1"]).astype(np.float32))
    z1 = xh @ Wh.T + xl @ Wh.T + xh @ Wl.T + p["b1"]
    h1 = f16(np.tanh(f16(z1)))
    z2 = h1 @ f16(p["W2"]).T + p["b2"]
    h2 = f16(np.tanh(f16(z2)))
    wh, wl = split16(np.asarray(p["w3"]).astype(np.float32))
    y = h2 @ wh + h2 @ wl + p["b3"][0]
    return y, (h1, h2)


def infer_bound(theta, ulps=2.0):
    """Per-sample bound on |y_gpu - y_oracle| from the hardware tanh: each hidden
    value may differ by `ulps` f16 units in the last place (2^-10 for |h| < 1) from
    the oracle's correctly rounded one; layer 1's differences reach y through
    |W2| and |w3|."""
    p = unpack(theta)
    e = ulps * 2.0 ** -11
    return float(np.sum(np.abs(p["w3"]) * (e + e * np.sum(np.abs(p["W2"]), axis=1))))


def loss_grad(theta, x, t, bf=False):
    """Mean squared error and its gradient (flat, like theta)."""
    p = unpack(theta)
    r = bf16 if bf else (lambda a: a)
    y, (x, z1, h1, z2, h2) = forward(theta, x, bf)
    B = x.shape[0]
    loss = np.mean((y - t) ** 2)
    dy = 2.0 * (y - t) / B
    g = {"w3": h2.T @ dy, "b3": np.array([np.sum(dy)])}
    dz2 = np.outer(dy, p["w3"]) * (1.0 - h2 * h2)
    g["b2"] = dz2.sum(axis=0)
    g["W2"] = r(dz2).T @ r(h1)
    dh1 = r(dz2) @ r(p["W2"])
    dz1 = dh1 * (1.0 - h1 * h1)
    g["b1"] = dz1.sum(axis=0)
    g["W1"] = dz1.T @ x
    return loss, pack(g)


def adam_step(theta, grad, m, v, t, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (Kingma & Ba, 2015), step number t >= 1:
    m <- beta1 m + (1 - beta1) g,  v <- beta2 v + (1 - beta2) g^2,
    theta <- theta - lr (m / (1 - beta1^t)) / (sqrt(v / (1 - beta2^t)) + eps).
    Returns the new (theta, m, v); the inputs are not modified."""
    g = np.asarray(grad, dtype=np.float64)
    m = beta1 * np.asarray(m, dtype=np.float64) + (1.0 - beta1) * g
    v = beta2 * np.asarray(v, dtype=np.float64) + (1.0 - beta2) * g * g
    mhat = m / (1.0 - beta1 ** t)
    vhat = v / (1.0 - beta2 ** t)
    return np.asarray(theta, dtype=np.float64) - lr * mhat / (np.sqrt(vhat) + eps), m, v
