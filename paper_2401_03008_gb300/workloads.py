"""Seeded synthetic inputs shared by the tests, the smoke check and the benchmark.

This module holds only the *problem definitions* (initial data sampled at the grid
positions and, for the Alfven wave, its exact solution).  It holds none of the
method's arithmetic: no reconstruction, flux, inversion or derivative.  The
conserved variables and the staggered field are built from these inputs by each
implementation on its own side (the CUDA library and the CPU oracle alike).

Grid convention (periodic, x fastest, arrays ``[var, nz, ny, nx]``):
  cell (i,j,k) at ((i+1/2)hx, (j+1/2)hy, (k+1/2)hz);
  face array d: the face half a cell above the cell centre along d;
  edge array c: the edge half a cell above the cell centre along both
  directions other than c (A_x at (i, j+1/2, k+1/2) and cyclic).
"""
import math

import numpy as np

GAMMA = 4.0 / 3.0


def _coords(nx, ny, nz, lx, ly, lz, off):
    """Positions of samples offset by ``off`` = (ox, oy, oz) cells from the lower
    cell corner; returns arrays broadcastable to [nz, ny, nx]."""
    hx, hy, hz = lx / nx, ly / ny, lz / nz
    x = (np.arange(nx) + off[0]) * hx
    y = (np.arange(ny) + off[1]) * hy
    z = (np.arange(nz) + off[2]) * hz
    return x[None, None, :], y[None, :, None], z[:, None, None]


# ---------------------------------------------------------------------------
# Circularly polarised Alfven wave (the paper's CPA-3D test, Sec. 4)
# ---------------------------------------------------------------------------

def alfven_speed(rho=1.0, p=1.0, B0=1.0, eta=1.0, gam=GAMMA):
    """Speed of the exact large-amplitude circularly polarised relativistic Alfven
    wave (Sec. 4, the v_A^2 equation): with E = rho h + B0^2 (1 + eta^2),
    v_A^2 = (B0^2 / E) / [ (1 + sqrt(1 - (2 eta B0^2 / E)^2)) / 2 ]."""
    rhoh = rho + gam / (gam - 1.0) * p
    e = rhoh + B0 * B0 * (1.0 + eta * eta)
    q = 2.0 * eta * B0 * B0 / e
    va2 = (B0 * B0 / e) / (0.5 * (1.0 + math.sqrt(1.0 - q * q)))
    return math.sqrt(va2)


def cpa_frame(kvec):
    """Right-handed orthonormal frame (X, Y, Z) with X along k.  Y = e x X / |e x X|
    with e = z (or x when k is along z), Z = X x Y.  For k along (1,1,1) this gives
    Y = (-1, 1, 0)/sqrt(2)."""
    X = np.asarray(kvec, dtype=np.float64)
    X = X / np.linalg.norm(X)
    e = np.array([0.0, 0.0, 1.0])
    if abs(abs(X[2]) - 1.0) < 1e-12:
        e = np.array([1.0, 0.0, 0.0])
    Y = np.cross(e, X)
    Y /= np.linalg.norm(Y)
    Z = np.cross(X, Y)
    return X, Y, Z


class CPA:
    """Circularly polarised Alfven wave along k = 2 pi (mx/lx, my/ly, mz/lz):
    B = B0 X + eta B0 (Y cos xi + Z sin xi), v = -v_A eta (Y cos xi + Z sin xi),
    rho and p uniform, xi = k.x - |k| v_A t (Sec. 4).  The transverse field is given
    through the edge vector potential A = -(eta B0/|k|) (Y cos xi + Z sin xi),
    whose curl is exactly the transverse part of B."""

    def __init__(self, nx, ny, nz, m=(1, 0, 0), L=(1.0, 1.0, 1.0), rho=1.0, p=1.0,
                 B0=1.0, eta=1.0, gam=GAMMA):
        self.n = (nx, ny, nz)
        self.L = tuple(float(v) for v in L)
        self.k = 2.0 * math.pi * np.array([m[0] / L[0], m[1] / L[1], m[2] / L[2]])
        self.kmag = float(np.linalg.norm(self.k))
        self.X, self.Y, self.Z = cpa_frame(self.k)
        self.rho, self.p, self.B0, self.eta, self.gam = rho, p, B0, eta, gam
        self.vA = alfven_speed(rho, p, B0, eta, gam)
        self.period = 2.0 * math.pi / (self.kmag * self.vA)

    def _phase(self, off, t):
        x, y, z = _coords(*self.n, *self.L, off)
        return self.k[0] * x + self.k[1] * y + self.k[2] * z - self.kmag * self.vA * t

    def prim5(self, t=0.0):
        """[5, nz, ny, nx]: rho, vx, vy, vz, p at cell centres."""
        nx, ny, nz = self.n
        xi = np.broadcast_to(self._phase((0.5, 0.5, 0.5), t), (nz, ny, nx))
        out = np.empty((5, nz, ny, nx))
        out[0] = self.rho
        out[4] = self.p
        c, s = np.cos(xi), np.sin(xi)
        for d in range(3):
            out[1 + d] = -self.vA * self.eta * (self.Y[d] * c + self.Z[d] * s)
        return out

    def bface_background(self):
        """[3, nz, ny, nx]: the uniform part B0 X on every face."""
        nx, ny, nz = self.n
        out = np.empty((3, nz, ny, nx))
        for d in range(3):
            out[d] = self.B0 * self.X[d]
        return out

    def apot(self, t=0.0):
        """[3, nz, ny, nx]: edge vector potential of the transverse field."""
        nx, ny, nz = self.n
        offs = [(0.5, 1.0, 1.0), (1.0, 0.5, 1.0), (1.0, 1.0, 0.5)]
        out = np.empty((3, nz, ny, nx))
        amp = -self.eta * self.B0 / self.kmag
        for c in range(3):
            xi = np.broadcast_to(self._phase(offs[c], t), (nz, ny, nx))
            out[c] = amp * (self.Y[c] * np.cos(xi) + self.Z[c] * np.sin(xi))
        return out

    def bcell(self, t=0.0):
        """[3, nz, ny, nx]: the exact field at cell centres (for the cell-centred
        variant without constrained transport)."""
        return np.ascontiguousarray(self.exact_prim8(t)[5:8])

    def exact_prim8(self, t):
        """[8, nz, ny, nx]: exact rho, v, p and B at cell centres at time t."""
        nx, ny, nz = self.n
        out = np.empty((8, nz, ny, nx))
        out[:5] = self.prim5(t)
        xi = np.broadcast_to(self._phase((0.5, 0.5, 0.5), t), (nz, ny, nx))
        c, s = np.cos(xi), np.sin(xi)
        for d in range(3):
            out[5 + d] = self.B0 * self.X[d] + self.eta * self.B0 * (self.Y[d] * c + self.Z[d] * s)
        return out

    def state_along(self, xi):
        """Primitives and field on the wave as functions of the phase xi (1-D arrays):
        returns prim[5, m], B[3, m]."""
        xi = np.asarray(xi, dtype=np.float64)
        c, s = np.cos(xi), np.sin(xi)
        prim = np.empty((5, xi.size))
        B = np.empty((3, xi.size))
        prim[0] = self.rho
        prim[4] = self.p
        for d in range(3):
            prim[1 + d] = -self.vA * self.eta * (self.Y[d] * c + self.Z[d] * s)
            B[d] = self.B0 * self.X[d] + self.eta * self.B0 * (self.Y[d] * c + self.Z[d] * s)
        return prim, B


# ---------------------------------------------------------------------------
# Random single-cell states (for the inversion tests)
# ---------------------------------------------------------------------------

def random_states(n, seed, lorentz_max=10.0, sigma_max=100.0, sigma_min=1e-3,
                  theta_min=1e-2, theta_max=1e2):
    """n random physical states: rho log-uniform in [0.1, 10], temperature p/rho
    log-uniform in [theta_min, theta_max], Lorentz factor log-uniform in
    [1, lorentz_max], magnetisation sigma = B^2/rho log-uniform in
    [sigma_min, sigma_max], isotropic random directions for v and B.
    Returns prim[5, n] (rho, vx, vy, vz, p) and B[3, n]."""
    rng = np.random.Generator(np.random.PCG64(seed))

    def logu(lo, hi, size):
        return np.exp(rng.uniform(math.log(lo), math.log(hi), size))

    def unit(size):
        v = rng.normal(size=(3, size))
        return v / np.linalg.norm(v, axis=0)

    rho = logu(0.1, 10.0, n)
    p = rho * logu(theta_min, theta_max, n)
    lor = logu(1.0, lorentz_max, n)
    vmag = np.sqrt(1.0 - 1.0 / lor ** 2)
    v = unit(n) * vmag
    bmag = np.sqrt(rho * logu(sigma_min, sigma_max, n))
    B = unit(n) * bmag
    prim = np.vstack([rho[None], v, p[None]])
    return prim, B


def random_smooth_fields(nx, ny, nz, seed, amp=0.3, kmax=2, L=(1.0, 1.0, 1.0),
                         rho0=1.0, p0=1.0, B0=(0.7, 0.4, 0.3)):
    """A smooth random periodic state for parity tests: a few Fourier modes
    (|m| <= kmax) of random phase on rho, v, p at cell centres and on the edge
    vector potential.  Returns prim5[5], bface background [3] (uniform B0) and
    apot[3]."""
    rng = np.random.Generator(np.random.PCG64(seed))
    modes = [(a, b, c) for a in range(-kmax, kmax + 1) for b in range(-kmax, kmax + 1)
             for c in range(-kmax, kmax + 1) if 0 < a * a + b * b + c * c <= kmax * kmax]

    def field(off, scale, nmodes=6):
        x, y, z = _coords(nx, ny, nz, *L, off)
        f = np.zeros((nz, ny, nx))
        for q in rng.choice(len(modes), size=nmodes, replace=False):
            m = modes[q]
            ph = rng.uniform(0, 2 * math.pi)
            a = rng.uniform(-1, 1) * scale
            k = 2 * math.pi * np.array(m) / np.array(L)
            f = f + a * np.cos(k[0] * x + k[1] * y + k[2] * z + ph)
        return f / nmodes

    prim = np.empty((5, nz, ny, nx))
    prim[0] = rho0 * (1.0 + 0.5 * amp * field((0.5, 0.5, 0.5), 1.0))
    for d in range(3):
        prim[1 + d] = amp * field((0.5, 0.5, 0.5), 1.0)
    prim[4] = p0 * (1.0 + 0.5 * amp * field((0.5, 0.5, 0.5), 1.0))
    bg = np.empty((3, nz, ny, nx))
    for d in range(3):
        bg[d] = B0[d]
    offs = [(0.5, 1.0, 1.0), (1.0, 0.5, 1.0), (1.0, 1.0, 0.5)]
    apot = np.empty((3, nz, ny, nx))
    for c in range(3):
        apot[c] = amp * field(offs[c], 1.0) / (2 * math.pi)
    return prim, bg, apot


# ---------------------------------------------------------------------------
# Decaying relativistic Alfvenic turbulence (3-D extension of the Sec. 5 set-up)
# ---------------------------------------------------------------------------

def _modes(kmax):
    """Integer wave vectors with 1 <= |k| <= kmax, one of each +-k pair."""
    out = []
    r = int(kmax)
    for kz in range(-r, r + 1):
        for ky in range(-r, r + 1):
            for kx in range(0, r + 1):
                k2 = kx * kx + ky * ky + kz * kz
                if k2 == 0 or k2 > kmax * kmax:
                    continue
                # half space: kx > 0, or kx == 0 and (ky > 0, or ky == 0 and kz > 0)
                if kx == 0 and (ky < 0 or (ky == 0 and kz < 0)):
                    continue
                out.append((kx, ky, kz))
    return np.array(out, dtype=np.float64)


def _synth(n, modes, coef, phase, off, device=None):
    """Real periodic field sum_m coef[m] cos(k_m . x + phase[m]) on an n^3 grid of a
    2 pi box, sampled at (i + off) h per axis (h = 2 pi / n), by inverse real FFT
    (exact for integer wave vectors).  Returns [nz, ny, nx]: a numpy array, or a
    float64 torch tensor on ``device`` when one is given (the same sums, for grids
    whose synthesis would take minutes on the host)."""
    h = 2.0 * np.pi / n
    # the nonzero spectral coefficients (index, value), accumulated on the host
    entries = {}

    def put(idx, c):
        entries[idx] = entries.get(idx, 0.0) + c

    for m, k in enumerate(modes):
        kx, ky, kz = (int(round(q)) for q in k)
        shift = (kx * off[0] + ky * off[1] + kz * off[2]) * h
        c = coef[m] * np.exp(1j * (phase[m] + shift)) * n ** 3
        if kx > 0:
            put((kz % n, ky % n, kx), c)
        else:  # kx = 0 plane: put both members of the pair (irfftn needs Hermitian input)
            put((kz % n, ky % n, 0), 0.5 * c)
            put(((-kz) % n, (-ky) % n, 0), 0.5 * np.conj(c))
    idx = np.array(list(entries.keys()), dtype=np.int64).reshape(-1, 3)
    val = np.array(list(entries.values()), dtype=np.complex128)
    if device is None:
        spec = np.zeros((n, n, n // 2 + 1), dtype=np.complex128)
        spec[idx[:, 0], idx[:, 1], idx[:, 2]] = val
        return np.fft.irfftn(spec, s=(n, n, n), axes=(0, 1, 2))
    import torch
    spec = torch.zeros((n, n, n // 2 + 1), dtype=torch.complex128, device=device)
    ti = torch.from_numpy(idx).to(device)
    spec[ti[:, 0], ti[:, 1], ti[:, 2]] = torch.from_numpy(val).to(device)
    out = torch.fft.irfftn(spec, s=(n, n, n), dim=(0, 1, 2))
    del spec
    return out


class Turbulence:
    """3-D decaying relativistic Alfvenic turbulence on a periodic (2 pi)^3 box.

    Background (Sec. 5 with the magnetisation of the 3-D benchmark): rho0 = 1, a
    uniform field B0 along z with sigma0 = B0^2/rho0 (default 10) and
    beta0 = 2 p0/B0^2 = 1, at rest.  Fluctuations: all integer modes with
    1 <= |k| <= kmax (default 4), random phases and random unit vectors e(k)
    perpendicular to k, independent for the velocity and the field (Sec. 5 uses
    different phases for v and B), so both are divergence-free:
      delta B = curl A,  A = sum_k (a_B/|k|) e_B(k) sin(k.x + phi_B(k)),
      u = sum_k a_u (k x e_u(k))/|k| cos(k.x + phi_u(k))  (a 4-velocity),
      v = u / sqrt(1 + u^2).
    The amplitudes are set afterwards (as in Sec. 5): a_B so that the mean of
    |delta B| over the cell centres is eta_b B0, a_u so that the largest Lorentz
    factor on the grid is lorentz_max.  Seeded (PCG64)."""

    def __init__(self, n, seed, sigma0=10.0, beta0=1.0, rho0=1.0, eta_b=0.5, lorentz_max=5.0,
                 kmax=4.0, gam=GAMMA, device=None):
        self.n = n
        self.device = device  # None: numpy arrays; else float64 torch tensors there
        self.L = (2 * np.pi,) * 3
        self.rho0, self.gam = rho0, gam
        self.B0 = math.sqrt(sigma0 * rho0)
        self.p0 = 0.5 * beta0 * self.B0 ** 2
        rng = np.random.Generator(np.random.PCG64(seed))
        self.modes = _modes(kmax)
        nm = len(self.modes)
        kn = np.linalg.norm(self.modes, axis=1)

        def perp_units():
            e = rng.normal(size=(nm, 3))
            e -= (np.sum(e * self.modes, axis=1) / kn ** 2)[:, None] * self.modes
            return e / np.linalg.norm(e, axis=1)[:, None]

        self.eB = perp_units()
        self.phB = rng.uniform(0, 2 * np.pi, nm)
        self.eu = perp_units()
        self.phu = rng.uniform(0, 2 * np.pi, nm)
        kxe_B = np.cross(self.modes, self.eB) / kn[:, None]   # unit vectors (e perp k)
        kxe_u = np.cross(self.modes, self.eu) / kn[:, None]
        self._kn = kn
        # unit-amplitude delta B and u at cell centres, for the normalisation
        c = (0.5, 0.5, 0.5)
        if device is None:
            dB = np.array([_synth(n, self.modes, kxe_B[:, q], self.phB, c) for q in range(3)])
            self.aB = eta_b * self.B0 / np.mean(np.sqrt(np.sum(dB ** 2, axis=0)))
            self._dBc = dB * self.aB
            u = np.array([_synth(n, self.modes, kxe_u[:, q], self.phu, c) for q in range(3)])
            umax = np.max(np.sqrt(np.sum(u ** 2, axis=0)))
            self.au = math.sqrt(lorentz_max ** 2 - 1.0) / umax
            u *= self.au
            self._v = u / np.sqrt(1.0 + np.sum(u ** 2, axis=0))[None]
        else:
            import torch
            m2 = None
            for q in range(3):
                f = _synth(n, self.modes, kxe_B[:, q], self.phB, c, device)
                m2 = f * f if m2 is None else m2.add_(f * f)
                del f
            self.aB = eta_b * self.B0 / float(torch.sqrt(m2).mean())
            del m2
            self._dBc = None  # the cell-centred field is only needed without UCT
            u = torch.stack([_synth(n, self.modes, kxe_u[:, q], self.phu, c, device)
                             for q in range(3)])
            u2 = (u * u).sum(0)
            umax = float(torch.sqrt(u2.max()))
            self.au = math.sqrt(lorentz_max ** 2 - 1.0) / umax
            u *= self.au
            u2 *= self.au ** 2
            self._v = u.div_(torch.sqrt(1.0 + u2)[None])
            del u2

    def _empty(self, shape):
        if self.device is None:
            return np.empty(shape)
        import torch
        return torch.empty(shape, dtype=torch.float64, device=self.device)

    def prim5(self):
        n = self.n
        out = self._empty((5, n, n, n))
        out[0] = self.rho0
        out[1:4] = self._v
        out[4] = self.p0
        return out

    def bface_background(self):
        n = self.n
        out = self._empty((3, n, n, n))
        out[0:2] = 0.0
        out[2] = self.B0
        return out

    def bcell(self):
        """[3, n, n, n]: the field at cell centres (B0 z + delta B), for the cell-centred
        variant without constrained transport."""
        out = self._dBc.copy()
        out[2] += self.B0
        return np.ascontiguousarray(out)

    def apot(self):
        """Edge vector potential: A_x at (i, j+1/2, k+1/2) and cyclic."""
        n = self.n
        offs = [(0.5, 1.0, 1.0), (1.0, 0.5, 1.0), (1.0, 1.0, 0.5)]
        out = self._empty((3, n, n, n))
        for c in range(3):
            # sin(k.x + phi) = cos(k.x + phi - pi/2)
            coef = self.aB / self._kn * self.eB[:, c]
            out[c] = _synth(n, self.modes, coef, self.phB - 0.5 * np.pi, offs[c], self.device)
        return out

    def release(self):
        """Drop the stored velocity field (after prim5() has been taken)."""
        self._v = None


# ---------------------------------------------------------------------------
# Initial parameters of the learned Newton guess (random inputs of training)
# ---------------------------------------------------------------------------

MLP_SHAPES = [(64, 5), (64,), (64, 64), (64,), (64,), (1,)]  # W1, b1, W2, b2, w3, b3


def mlp_init(seed):
    """Glorot-uniform weights and zero biases, flattened in the order W1, b1, W2, b2,
    w3, b3 (4609 float32 values); seeded PCG64."""
    rng = np.random.Generator(np.random.PCG64(seed))
    parts = []
    for shape in MLP_SHAPES:
        if len(shape) == 2 or shape == (64,) and len(parts) == 4:
            fan_in = shape[1] if len(shape) == 2 else 64
            fan_out = shape[0] if len(shape) == 2 else 1
            lim = math.sqrt(6.0 / (fan_in + fan_out))
            parts.append(rng.uniform(-lim, lim, shape).ravel())
        else:
            parts.append(np.zeros(int(np.prod(shape))))
    return np.concatenate(parts).astype(np.float32)


# ---------------------------------------------------------------------------
# 2.5-D decaying relativistic turbulence (the Sec. 5 run)
# ---------------------------------------------------------------------------

class Turbulence2D:
    """The Sec. 5 set-up on an n x n x 1 grid of a (2 pi)^2 box: rho0 = 1, uniform B0
    along z with sigma0 = B0^2/rho0 = 100 and beta0 = 2 p0/B0^2 = 1 (B0 = 10,
    p0 = 50), fluid at rest, plus in-plane fluctuations
      dv = eta_v sum_k (k/|k|) x e_z cos(k.x + phi_v(k)),
      dB = eta_B sum_k (k/|k|) x e_z cos(k.x + phi_B(k)),
    over kx = 0..4, ky = -4..4 with 1 <= |k| <= 4, independent random phases for v and
    B (Sec. 5).  Both are divergence-free; dB enters as the curl of the edge potential
    A_z = eta_B sum_k sin(k.x + phi_B)/|k|.  The amplitudes are fixed afterwards so
    that the grid means of |dv|/v_A and |dB|/B0 equal eta_rms = 0.25, with
    v_A = B0/sqrt(rho0 + 4 p0 + B0^2) (Sec. 5).  Seeded PCG64."""

    def __init__(self, n, seed, sigma0=100.0, beta0=1.0, rho0=1.0, eta_rms=0.25, kmax=4,
                 gam=GAMMA):
        self.n = n
        self.L = (2 * np.pi, 2 * np.pi, 2 * np.pi / n)
        self.rho0, self.gam = rho0, gam
        self.B0 = math.sqrt(sigma0 * rho0)
        self.p0 = 0.5 * beta0 * self.B0 ** 2
        self.vA = self.B0 / math.sqrt(rho0 + gam / (gam - 1.0) * self.p0 + self.B0 ** 2)
        modes = [(kx, ky) for kx in range(0, kmax + 1) for ky in range(-kmax, kmax + 1)
                 if 0 < kx * kx + ky * ky <= kmax * kmax]
        self.modes = np.array(modes, dtype=np.float64)
        rng = np.random.Generator(np.random.PCG64(seed))
        self.phv = rng.uniform(0, 2 * np.pi, len(modes))
        self.phB = rng.uniform(0, 2 * np.pi, len(modes))
        self.kn = np.linalg.norm(self.modes, axis=1)
        x = (np.arange(n) + 0.5) * 2 * np.pi / n
        X, Y = np.meshgrid(x, x, indexing="xy")   # [y, x]
        self._X, self._Y = X, Y
        dv = self._field(self.phv, (0.5, 0.5))
        dB = self._field(self.phB, (0.5, 0.5))
        self.eta_v = eta_rms * self.vA / np.mean(np.sqrt(dv[0] ** 2 + dv[1] ** 2))
        self.eta_B = eta_rms * self.B0 / np.mean(np.sqrt(dB[0] ** 2 + dB[1] ** 2))
        self._dv = dv * self.eta_v

    def _field(self, ph, off):
        """unit-amplitude sum of (ky, -kx)/|k| cos(k.x + ph) at offset positions"""
        h = 2 * np.pi / self.n
        X = self._X + (off[0] - 0.5) * h
        Y = self._Y + (off[1] - 0.5) * h
        fx = np.zeros_like(X)
        fy = np.zeros_like(X)
        for q, (kx, ky) in enumerate(self.modes):
            c = np.cos(kx * X + ky * Y + ph[q])
            fx += ky / self.kn[q] * c
            fy -= kx / self.kn[q] * c
        return np.array([fx, fy])

    def prim5(self):
        n = self.n
        out = np.zeros((5, 1, n, n))
        out[0] = self.rho0
        out[1, 0] = self._dv[0]
        out[2, 0] = self._dv[1]
        out[4] = self.p0
        return out

    def bface_background(self):
        out = np.zeros((3, 1, self.n, self.n))
        out[2] = self.B0
        return out

    def bcell(self):
        """cell-centred B (the variant without UCT): B0 e_z plus the pointwise dB"""
        out = np.zeros((3, 1, self.n, self.n))
        dB = self._field(self.phB, (0.5, 0.5)) * self.eta_B
        out[0, 0], out[1, 0], out[2] = dB[0], dB[1], self.B0
        return out

    def apot(self):
        """A_z at the z-edges (i+1/2, j+1/2); A_x = A_y = 0."""
        n = self.n
        h = 2 * np.pi / n
        X = self._X + 0.5 * h
        Y = self._Y + 0.5 * h
        az = np.zeros_like(X)
        for q, (kx, ky) in enumerate(self.modes):
            az += np.sin(kx * X + ky * Y + self.phB[q]) / self.kn[q]
        out = np.zeros((3, 1, n, n))
        out[2, 0] = self.eta_B * az
        return out
