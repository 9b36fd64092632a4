"""Python side of the FP64 CPU oracle (ctypes over ``echo_oracle.c``).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this module.  It shares nothing with
the CUDA library; inputs come from the seeded generators in
``paper_2401_03008_gb300.workloads`` (which hold none of the method's arithmetic).

Every grid array is a C-contiguous float64 numpy array shaped
``[var, nz, ny, nx]`` (x fastest).
"""
import ctypes as C
import os

import numpy as np

from . import build_oracle

_dp = C.POINTER(C.c_double)
_ip = C.POINTER(C.c_int)


class Cfg(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int),
                ("lx", C.c_double), ("ly", C.c_double), ("lz", C.c_double),
                ("gam", C.c_double), ("cfl", C.c_double),
                ("uct", C.c_int), ("ho", C.c_int),
                ("tol", C.c_double), ("maxit", C.c_int),
                ("guess", C.c_int), ("nthreads", C.c_int), ("rec", C.c_int), ("rk", C.c_int)]


class Stats(C.Structure):
    _fields_ = [("cells", C.c_long), ("iters", C.c_long), ("itmax", C.c_int),
                ("failures", C.c_long), ("fallbacks", C.c_long),
                ("rec_fallbacks", C.c_long)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


GUESS_WARM, GUESS_COLD, GUESS_ARRAY = 0, 1, 2

_lib = None


def lib():
    global _lib
    if _lib is None:
        # a test may point at a deliberately broken copy (mutation tests)
        path = os.environ.get("ECHO_ORACLE_LIB") or build_oracle.build()
        L = C.CDLL(path)
        L.orc_prim2cons.argtypes = [_dp, _dp, C.c_double, _dp]
        L.orc_flux.argtypes = [_dp, _dp, C.c_double, C.c_int, _dp]
        L.orc_speeds.argtypes = [_dp, _dp, C.c_double, C.c_int, _dp, _dp]
        L.orc_hll.argtypes = [_dp, _dp, _dp, _dp, C.c_double, C.c_int, _dp, _dp, _dp]
        L.orc_mp5.argtypes = [_dp]
        L.orc_mp5.restype = C.c_double
        L.orc_mc.argtypes = [_dp]
        L.orc_mc.restype = C.c_double
        L.orc_int.argtypes = [_dp, C.c_int]
        L.orc_int.restype = C.c_double
        L.orc_der.argtypes = [_dp, C.c_double, C.c_int]
        L.orc_der.restype = C.c_double
        L.orc_c2p_fdf.argtypes = [_dp, _dp, C.c_double, C.c_double, _dp, _dp]
        L.orc_c2p.argtypes = [_dp, _dp, C.c_double, C.c_double, C.c_double, C.c_int,
                              _dp, _dp, _ip]
        L.orc_c2p.restype = C.c_int
        L.orc_c2p_batch.argtypes = [C.c_long, _dp, _dp, _dp, C.c_double, C.c_double,
                                    C.c_int, _dp, _dp, _ip]
        L.orc_c2p_batch.restype = C.c_long
        L.orc_uct_point.argtypes = [_dp, _dp, _dp, _dp, C.c_double, C.c_double,
                                    C.c_double, C.c_double]
        L.orc_uct_point.restype = C.c_double
        cp = C.POINTER(Cfg)
        sp = C.POINTER(Stats)
        L.orc_curl_apot.argtypes = [cp, _dp, _dp]
        L.orc_divb.argtypes = [cp, _dp, _dp]
        L.orc_rhs.argtypes = [cp, _dp, _dp, _dp, _dp, _dp, _dp, _dp, _dp, sp]
        L.orc_rhs.restype = C.c_int
        L.orc_set_state.argtypes = [cp, _dp, _dp, _dp, _dp]
        L.orc_step.argtypes = [cp, _dp, _dp, _dp, _dp, _dp, C.c_double, _dp, sp]
        L.orc_step.restype = C.c_int
        L.orc_primitives.argtypes = [cp, _dp, _dp, _dp, _dp, sp]
        L.orc_primitives.restype = C.c_int
        L.orc_totals.argtypes = [cp, _dp, _dp, _dp]
        _lib = L
    return _lib


def _p(a):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(_dp)


def _vec(x):
    return np.ascontiguousarray(np.asarray(x, dtype=np.float64))


# --------------------------------------------------------------------------
# point-wise functions
# --------------------------------------------------------------------------

def prim2cons(prim, B, gam):
    """(rho, vx, vy, vz, p), (Bx, By, Bz) -> (D, Sx, Sy, Sz, U)."""
    u = np.zeros(5)
    lib().orc_prim2cons(_p(_vec(prim)), _p(_vec(B)), gam, _p(u))
    return u


def flux(prim, B, gam, d):
    """Physical flux along d of (D, S, U, B): 8 values."""
    f = np.zeros(8)
    lib().orc_flux(_p(_vec(prim)), _p(_vec(B)), gam, d, _p(f))
    return f


def speeds(prim, B, gam, d):
    lm, lp = C.c_double(), C.c_double()
    lib().orc_speeds(_p(_vec(prim)), _p(_vec(B)), gam, d, C.byref(lm), C.byref(lp))
    return lm.value, lp.value


def hll(primL, BL, primR, BR, gam, d):
    f = np.zeros(8)
    ap, am = C.c_double(), C.c_double()
    lib().orc_hll(_p(_vec(primL)), _p(_vec(BL)), _p(_vec(primR)), _p(_vec(BR)), gam, d,
                  _p(f), C.byref(ap), C.byref(am))
    return f, ap.value, am.value


def mp5(s):
    return lib().orc_mp5(_p(_vec(s)))


def mc(s):
    """Linear (MC-limited) value at i+1/2 from (u_{i-1}, u_i, u_{i+1})."""
    return lib().orc_mc(_p(_vec(s)))


def interp(s, ho):
    return lib().orc_int(_p(_vec(s)), int(ho))


def der(s, h, ho):
    return lib().orc_der(_p(_vec(s)), h, int(ho))


def c2p_fdf(u, B, gam, W):
    f, df = C.c_double(), C.c_double()
    lib().orc_c2p_fdf(_p(_vec(u)), _p(_vec(B)), gam, W, C.byref(f), C.byref(df))
    return f.value, df.value


def c2p(u, B, gam, W0, tol=1e-6, maxit=100):
    prim = np.zeros(5)
    W = C.c_double()
    it = C.c_int()
    bad = lib().orc_c2p(_p(_vec(u)), _p(_vec(B)), gam, W0, tol, maxit, _p(prim),
                        C.byref(W), C.byref(it))
    return prim, W.value, it.value, bad


def c2p_batch(u, B, W0, gam, tol=1e-6, maxit=100):
    """u[5, n], B[3, n], W0[n] -> prim[5, n], W[n], iterations[n], failures."""
    u = _vec(u)
    B = _vec(B)
    W0 = _vec(W0)
    n = W0.shape[0]
    prim = np.zeros((5, n))
    W = np.zeros(n)
    it = np.zeros(n, dtype=np.int32)
    fails = lib().orc_c2p_batch(n, _p(u), _p(B), _p(W0), gam, tol, maxit, _p(prim),
                                _p(W), it.ctypes.data_as(_ip))
    return prim, W, it, fails


def uct_point(va, vb, Ba, Bb, apa, ama, apb, amb):
    return lib().orc_uct_point(_p(_vec(va)), _p(_vec(vb)), _p(_vec(Ba)), _p(_vec(Bb)),
                               apa, ama, apb, amb)


# --------------------------------------------------------------------------
# grid-level oracle
# --------------------------------------------------------------------------

class Grid:
    """Oracle state on a periodic nx*ny*nz grid: cons[5], face (or cell) B[3], W."""

    def __init__(self, nx, ny, nz, lx=1.0, ly=1.0, lz=1.0, gam=4.0 / 3.0, cfl=0.4,
                 uct=1, ho=1, tol=1e-6, maxit=100, guess=GUESS_WARM, nthreads=0, rec=0, rk=3):
        self.cfg = Cfg(nx, ny, nz, lx, ly, lz, gam, cfl, uct, ho, tol, maxit, guess,
                       nthreads or int(os.environ.get("ORACLE_THREADS", "0")), rec, rk)
        self.shape = (nz, ny, nx)
        self.n = nx * ny * nz
        self.cons = np.zeros((5,) + self.shape)
        self.bf = np.zeros((3,) + self.shape)
        self.W = np.zeros(self.shape)
        self.guessarr = None
        self.t = 0.0
        self.steps = 0
        self.stats = Stats()

    def set_state(self, prim5, bf=None, apot=None):
        """prim5[5]: rho, vx, vy, vz, p at cell centres; bf[3] face (or cell) field;
        apot[3] edge vector potential whose curl is added to bf."""
        b = np.zeros((3,) + self.shape) if bf is None else _vec(bf).copy()
        if apot is not None:
            lib().orc_curl_apot(C.byref(self.cfg), _p(_vec(apot)), _p(b))
        self.bf = np.ascontiguousarray(b)
        lib().orc_set_state(C.byref(self.cfg), _p(_vec(prim5)), _p(self.bf),
                            _p(self.cons), _p(self.W))
        self.t = 0.0
        self.steps = 0

    def _guess_ptr(self):
        """the caller's guess array (required when guess == GUESS_ARRAY)"""
        if self.cfg.guess == GUESS_ARRAY:
            if self.guessarr is None or self.guessarr.size != self.n:
                raise ValueError("guess = GUESS_ARRAY needs guessarr of %d values" % self.n)
            self.guessarr = np.ascontiguousarray(self.guessarr, dtype=np.float64)
            return _p(self.guessarr)
        return None

    def rhs(self, with_prims=False):
        rc = np.zeros((5,) + self.shape)
        rb = np.zeros((3,) + self.shape)
        prim = np.zeros((8,) + self.shape)
        amax = C.c_double()
        ga = self._guess_ptr()
        bad = lib().orc_rhs(C.byref(self.cfg), _p(self.cons), _p(self.bf), _p(self.W), ga,
                            _p(rc), _p(rb), _p(prim), C.byref(amax), C.byref(self.stats))
        if with_prims:
            return rc, rb, amax.value, bad, prim
        return rc, rb, amax.value, bad

    def step(self, nsteps=1, t_end=float("inf")):
        bad = 0
        dt = C.c_double()
        t = C.c_double(self.t)
        ga = self._guess_ptr()
        self.dts = []
        for _ in range(nsteps):
            if t.value >= t_end:
                break
            bad |= lib().orc_step(C.byref(self.cfg), _p(self.cons), _p(self.bf), _p(self.W),
                                  ga, C.byref(t), t_end, C.byref(dt), C.byref(self.stats))
            self.dts.append(dt.value)
            self.steps += 1
        self.t = t.value
        return bad

    def primitives(self):
        """[8, nz, ny, nx]: rho, vx, vy, vz, p, Bx, By, Bz (B at cell centres)."""
        out = np.zeros((8,) + self.shape)
        W = self.W.copy()
        lib().orc_primitives(C.byref(self.cfg), _p(self.cons), _p(self.bf), _p(W), _p(out),
                             C.byref(self.stats))
        return out

    def divb(self):
        out = np.zeros(self.shape)
        lib().orc_divb(C.byref(self.cfg), _p(self.bf), _p(out))
        return out

    def totals(self):
        tot = np.zeros(8)
        lib().orc_totals(C.byref(self.cfg), _p(self.cons), _p(self.bf), _p(tot))
        return tot
