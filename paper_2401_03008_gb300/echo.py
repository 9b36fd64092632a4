"""Thin ctypes binding of libecho (include/echo.h): argument marshalling only.

Every step of the computation runs in the CUDA library; this module converts
numpy arrays (host, ``ECHO_PTR_HOST``) and torch CUDA tensors (device,
``ECHO_PTR_DEVICE``) to pointers and status codes to exceptions.  If the library
cannot be built or loaded it raises: there is no fallback.
"""
import ctypes as C
import math
import os

import numpy as np

from . import build as _build

ECHO_OK, ECHO_ERR_ARG, ECHO_ERR_CUDA, ECHO_ERR_OOM = 0, -1, -2, -3
ECHO_ERR_C2P, ECHO_ERR_NONFINITE, ECHO_ERR_STATE = -4, -5, -6
PTR_HOST, PTR_DEVICE = 0, 1
FP64, MIXED = 0, 1
GUESS_PREV, GUESS_COLD, GUESS_MLP = 0, 1, 2
NKERNELS = 20

_STATUS = {0: "ECHO_OK", -1: "ECHO_ERR_ARG", -2: "ECHO_ERR_CUDA", -3: "ECHO_ERR_OOM",
           -4: "ECHO_ERR_C2P", -5: "ECHO_ERR_NONFINITE", -6: "ECHO_ERR_STATE"}

# every entry point declared in include/echo.h
EXPORTS = ["echo_config_default", "echo_create", "echo_destroy", "echo_set_state",
           "echo_step", "echo_rhs", "echo_get_primitives", "echo_get_state",
           "echo_set_conserved", "echo_diagnostics", "echo_l1_error", "echo_profile_enable",
           "echo_profile_read", "echo_launches", "echo_probe_fma_peak", "echo_stream",
           "echo_last_error", "echo_diagnostics_noalloc", "echo_mlp_load", "echo_mlp_forward",
           "echo_mlp_grad", "echo_mlp_train", "echo_mlp_harvest", "echo_mlp_guess",
           "echo_decomp_min_halo",
           "echo_decomp_create", "echo_decomp_destroy", "echo_decomp_set_state",
           "echo_decomp_step", "echo_decomp_get_state", "echo_decomp_get_primitives",
           "echo_decomp_counters", "echo_decomp_last_error"]
MLP_NPARAM = 4609


class EchoError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s: %s" % (_STATUS.get(status, status), msg))
        self.status = status


class Config(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int),
                ("lx", C.c_double), ("ly", C.c_double), ("lz", C.c_double),
                ("gamma_ad", C.c_double), ("cfl", C.c_double),
                ("uct", C.c_int), ("ho", C.c_int), ("rec", C.c_int),
                ("precision", C.c_int), ("c2p_guess", C.c_int),
                ("c2p_tol", C.c_double), ("c2p_maxit", C.c_int),
                ("device", C.c_int), ("stream", C.c_void_p), ("rk_order", C.c_int),
                ("sweeps", C.c_int)]


class TrainCfg(C.Structure):
    _fields_ = [("epochs", C.c_int), ("batch", C.c_int), ("lr", C.c_double),
                ("beta1", C.c_double), ("beta2", C.c_double), ("eps", C.c_double),
                ("lr_decay", C.c_double), ("seed", C.c_ulong)]


class Diag(C.Structure):
    _fields_ = [("t", C.c_double), ("dt", C.c_double), ("amax", C.c_double),
                ("divb_max", C.c_double), ("divb_l2", C.c_double),
                ("tot", C.c_double * 8), ("newton_it_mean", C.c_double),
                ("newton_it_max", C.c_int), ("c2p_calls", C.c_long),
                ("c2p_fallbacks", C.c_long), ("c2p_failures", C.c_long),
                ("nonfinite", C.c_long), ("step", C.c_long), ("newton_it32_mean", C.c_double)]

    def as_dict(self):
        d = {k: getattr(self, k) for k, _ in self._fields_}
        d["tot"] = list(self.tot)
        return d


_lib = None


def lib_path():
    return _build.LIB


def lib():
    """Load libecho.so (building it in-tree if it is missing or stale)."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.build()
    L = C.CDLL(path)
    vp, dp, ip = C.c_void_p, C.POINTER(C.c_double), C.c_int
    L.echo_config_default.argtypes = [C.POINTER(Config)]
    L.echo_create.argtypes = [C.POINTER(Config), C.POINTER(vp)]
    L.echo_destroy.argtypes = [vp]
    L.echo_set_state.argtypes = [vp, vp, vp, vp, ip]
    L.echo_step.argtypes = [vp, ip, C.c_double, C.POINTER(C.c_int), dp]
    L.echo_rhs.argtypes = [vp, vp, vp, dp, ip]
    L.echo_get_primitives.argtypes = [vp, vp, ip]
    L.echo_get_state.argtypes = [vp, vp, vp, vp, dp, C.POINTER(C.c_long), ip]
    L.echo_set_conserved.argtypes = [vp, vp, vp, vp, C.c_double, C.c_long, ip]
    L.echo_diagnostics.argtypes = [vp, C.POINTER(Diag), ip]
    L.echo_l1_error.argtypes = [vp, vp, ip, dp]
    L.echo_profile_enable.argtypes = [vp, ip]
    L.echo_profile_read.argtypes = [vp, ip, C.POINTER(C.c_long), dp, C.POINTER(C.c_char_p), ip]
    L.echo_launches.argtypes = [vp]
    L.echo_launches.restype = C.c_long
    L.echo_probe_fma_peak.argtypes = [vp, ip, dp]
    L.echo_stream.argtypes = [vp]
    L.echo_stream.restype = vp
    L.echo_last_error.argtypes = [vp]
    L.echo_last_error.restype = C.c_char_p
    L.echo_diagnostics_noalloc.argtypes = [vp, vp, ip, ip, ip, C.c_double, C.c_double,
                                           C.c_double, ip, vp, vp, ip]
    fp = C.POINTER(C.c_float)
    L.echo_mlp_load.argtypes = [vp, fp, C.c_long]
    L.echo_mlp_forward.argtypes = [fp, vp, C.c_long, vp, vp]
    L.echo_mlp_grad.argtypes = [fp, vp, vp, C.c_long, fp, fp, vp]
    L.echo_mlp_train.argtypes = [vp, vp, C.c_long, C.POINTER(TrainCfg), fp, fp, vp]
    L.echo_mlp_harvest.argtypes = [vp, ip, C.c_long, vp, vp, C.c_long, C.POINTER(C.c_long)]
    L.echo_mlp_guess.argtypes = [vp, vp, ip]
    L.echo_decomp_min_halo.argtypes = [C.POINTER(Config)]
    L.echo_decomp_create.argtypes = [C.POINTER(Config), ip, ip, ip, ip, C.POINTER(vp)]
    L.echo_decomp_destroy.argtypes = [vp]
    L.echo_decomp_set_state.argtypes = [vp, vp, vp, vp, ip]
    L.echo_decomp_step.argtypes = [vp, ip, C.c_double, C.POINTER(C.c_int), dp]
    L.echo_decomp_get_state.argtypes = [vp, vp, vp, vp, dp, C.POINTER(C.c_long), ip]
    L.echo_decomp_get_primitives.argtypes = [vp, vp, ip]
    L.echo_decomp_counters.argtypes = [vp, dp]
    L.echo_decomp_last_error.argtypes = [vp]
    L.echo_decomp_last_error.restype = C.c_char_p
    _lib = L
    return L


def _is_torch(x):
    return type(x).__module__.startswith("torch")


def _ptr(x, what, count):
    """(pointer, kind) of a float64 array with count elements; None passes through."""
    if x is None:
        return None, None
    if _is_torch(x):
        import torch
        if not (x.is_cuda and x.dtype == torch.float64 and x.is_contiguous()):
            raise ValueError("%s: need a contiguous float64 CUDA tensor" % what)
        if x.numel() != count:
            raise ValueError("%s: %d elements, expected %d" % (what, x.numel(), count))
        return C.c_void_p(x.data_ptr()), PTR_DEVICE
    if not (isinstance(x, np.ndarray) and x.dtype == np.float64 and x.flags.c_contiguous):
        raise ValueError("%s: need a C-contiguous float64 numpy array" % what)
    if x.size != count:
        raise ValueError("%s: %d elements, expected %d" % (what, x.size, count))
    return C.c_void_p(x.ctypes.data), PTR_HOST


def make_config(nx, ny, nz, L=(1.0, 1.0, 1.0), gamma=4.0 / 3.0, cfl=0.4, ho=1,
                precision="fp64", guess="prev", tol=1e-6, maxit=100, device=0, stream=None,
                uct=1, rec="mp5", rk_order=3, sweeps="auto"):
    """echo_config from keyword arguments (the defaults of echo_config_default)."""
    cfg = Config()
    lib().echo_config_default(C.byref(cfg))
    cfg.nx, cfg.ny, cfg.nz = nx, ny, nz
    cfg.lx, cfg.ly, cfg.lz = L
    cfg.gamma_ad = gamma
    cfg.cfl = cfl
    cfg.ho = ho
    cfg.uct = uct
    cfg.rec = {"mp5": 0, "linear": 1}[rec]
    cfg.rk_order = rk_order
    cfg.precision = {"fp64": FP64, "mixed": MIXED}[precision]
    cfg.c2p_guess = {"prev": GUESS_PREV, "cold": GUESS_COLD, "mlp": GUESS_MLP}[guess]
    cfg.c2p_tol = tol
    cfg.c2p_maxit = maxit
    cfg.device = device
    cfg.stream = stream
    cfg.sweeps = {"auto": 0, "fused": 1, "separate": 2}[sweeps]
    return cfg


class Solver:
    """One libecho context: a periodic grid with its state on the GPU."""

    def __init__(self, nx, ny, nz, L=(1.0, 1.0, 1.0), **kw):
        self.L = lib()
        cfg = make_config(nx, ny, nz, L, **kw)
        self.cfg = cfg
        self.shape = (nz, ny, nx)
        self.n = nx * ny * nz
        self._h = C.c_void_p()
        self._check(self.L.echo_create(C.byref(cfg), C.byref(self._h)), None)

    # ------------------------------------------------------------------
    def _check(self, st, h="self"):
        if st != ECHO_OK:
            handle = self._h if h == "self" else None
            raise EchoError(st, self.L.echo_last_error(handle).decode())

    def close(self):
        if getattr(self, "_h", None):
            self.L.echo_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    @staticmethod
    def _same_kind(*kinds):
        ks = {k for k in kinds if k is not None}
        if len(ks) > 1:
            raise ValueError("mix of host and device arrays in one call")
        return ks.pop() if ks else PTR_HOST

    @staticmethod
    def _sync_torch(kind):
        if kind == PTR_DEVICE:
            import torch
            torch.cuda.synchronize()

    # ------------------------------------------------------------------
    def set_state(self, prim, bface=None, apot=None):
        """Initial data (echo_set_state): prim [5][nz][ny][nx] = rho, v, p at cell
        centres; bface [3][nz][ny][nx] the face field (cell-centred with uct=0);
        apot [3][nz][ny][nx] an edge vector potential whose curl is added.  numpy
        arrays (host) or float64 CUDA tensors (device), all of one kind."""
        n = self.n
        p, kp = _ptr(prim, "prim", 5 * n)
        b, kb = _ptr(bface, "bface", 3 * n)
        a, ka = _ptr(apot, "apot", 3 * n)
        kind = self._same_kind(kp, kb, ka)
        self._sync_torch(kind)
        self._check(self.L.echo_set_state(self._h, p, b, a, kind))

    def step(self, max_steps=1, t_end=math.inf):
        """Advance up to max_steps Runge-Kutta steps, the last one shortened to land on
        t_end (echo_step); returns (steps taken, time reached).  Raises EchoError
        (status ECHO_ERR_C2P) after rolling back a step whose inversion failed."""
        done = C.c_int()
        t = C.c_double()
        st = self.L.echo_step(self._h, max_steps, t_end, C.byref(done), C.byref(t))
        self._check(st)
        return done.value, t.value

    def _out(self, count, shape, device):
        if device:
            import torch
            return torch.empty(shape, dtype=torch.float64, device="cuda")
        return np.empty(shape, dtype=np.float64)

    def rhs(self, device=False):
        """One evaluation of the right-hand side (echo_rhs): (d/dt of the 5 conserved
        cell variables, d/dt of the 3 face-field arrays, largest HLL speed)."""
        n = self.n
        rc = self._out(5 * n, (5,) + self.shape, device)
        rb = self._out(3 * n, (3,) + self.shape, device)
        amax = C.c_double()
        pc, kind = _ptr(rc, "rhs_cons", 5 * n)
        pb, _ = _ptr(rb, "rhs_face", 3 * n)
        self._sync_torch(kind)
        self._check(self.L.echo_rhs(self._h, pc, pb, C.byref(amax), kind))
        return rc, rb, amax.value

    def primitives(self, out=None, device=False):
        """[8][nz][ny][nx] = rho, vx, vy, vz, p, Bx, By, Bz with the field at cell
        centres (echo_get_primitives); into out if given (numpy or CUDA tensor)."""
        if out is None:
            out = self._out(8 * self.n, (8,) + self.shape, device)
        p, kind = _ptr(out, "out", 8 * self.n)
        self._sync_torch(kind)
        self._check(self.L.echo_get_primitives(self._h, p, kind))
        return out

    def get_state(self, cons=None, bface=None, w=None, device=False):
        """Checkpoint (echo_get_state): (cons [5][...], bface [3][...], Newton guess
        W [...], t, step)."""
        n = self.n
        cons = self._out(5 * n, (5,) + self.shape, device) if cons is None else cons
        bface = self._out(3 * n, (3,) + self.shape, device) if bface is None else bface
        w = self._out(n, self.shape, device) if w is None else w
        pc, kind = _ptr(cons, "cons", 5 * n)
        pb, _ = _ptr(bface, "bface", 3 * n)
        pw, _ = _ptr(w, "w", n)
        t = C.c_double()
        step = C.c_long()
        self._sync_torch(kind)
        self._check(self.L.echo_get_state(self._h, pc, pb, pw, C.byref(t), C.byref(step), kind))
        return cons, bface, w, t.value, step.value

    def set_conserved(self, cons, bface, w=None, t=0.0, step=0):
        """Resume from a checkpoint of get_state (echo_set_conserved); bit-identical
        to an uninterrupted run."""
        n = self.n
        pc, kc = _ptr(cons, "cons", 5 * n)
        pb, kb = _ptr(bface, "bface", 3 * n)
        pw, kw = _ptr(w, "w", n)
        kind = self._same_kind(kc, kb, kw)
        self._sync_torch(kind)
        self._check(self.L.echo_set_conserved(self._h, pc, pb, pw, t, step, kind))

    def diagnostics(self, reset=False):
        """Totals, div B, Newton statistics of the current state (echo_diagnostics) as
        a dict; reset=True clears the Newton counters afterwards."""
        d = Diag()
        self._check(self.L.echo_diagnostics(self._h, C.byref(d), int(reset)))
        return d.as_dict()

    def l1_error(self, ref):
        """Mean |primitives - ref| per variable (echo_l1_error), ref [8][nz][ny][nx]."""
        p, kind = _ptr(ref, "ref", 8 * self.n)
        out = (C.c_double * 8)()
        self._sync_torch(kind)
        self._check(self.L.echo_l1_error(self._h, p, kind, out))
        return np.array(out[:])

    def profile(self, on=True):
        self._check(self.L.echo_profile_enable(self._h, int(on)))

    def profile_read(self, reset=True):
        res = {}
        for k in range(NKERNELS):
            cnt = C.c_long()
            ms = C.c_double()
            name = C.c_char_p()
            self._check(self.L.echo_profile_read(self._h, k, C.byref(cnt), C.byref(ms),
                                                 C.byref(name), int(reset)))
            if cnt.value:
                res[name.value.decode()] = (cnt.value, ms.value)
        return res

    @property
    def launches(self):
        return self.L.echo_launches(self._h)

    def probe_fma_peak(self, precision="fp64"):
        f = C.c_double()
        self._check(self.L.echo_probe_fma_peak(self._h, {"fp64": FP64, "fp32": MIXED}[precision],
                                               C.byref(f)))
        return f.value

    @property
    def stream(self):
        return self.L.echo_stream(self._h)


class Decomp:
    """The grid split into px * py * pz blocks with a wide halo, all on one GPU
    (echo_decomp_*): one exchange of every variable per Runge-Kutta substep."""

    def __init__(self, nx, ny, nz, blocks, halo=None, L=(1.0, 1.0, 1.0), **kw):
        self.L = lib()
        self.cfg = make_config(nx, ny, nz, L, **kw)
        self.min_halo = self.L.echo_decomp_min_halo(C.byref(self.cfg))
        self.halo = self.min_halo if halo is None else halo
        self.shape = (nz, ny, nx)
        self.n = nx * ny * nz
        self._h = C.c_void_p()
        self._check(self.L.echo_decomp_create(C.byref(self.cfg), *blocks, self.halo,
                                              C.byref(self._h)), None)

    def _check(self, st, h="self"):
        if st != ECHO_OK:
            handle = self._h if h == "self" else None
            raise EchoError(st, self.L.echo_decomp_last_error(handle).decode())

    def close(self):
        if getattr(self, "_h", None):
            self.L.echo_decomp_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_state(self, prim, bface=None, apot=None):
        """Initial data (echo_set_state): prim [5][nz][ny][nx] = rho, v, p at cell
        centres; bface [3][nz][ny][nx] the face field (cell-centred with uct=0);
        apot [3][nz][ny][nx] an edge vector potential whose curl is added.  numpy
        arrays (host) or float64 CUDA tensors (device), all of one kind."""
        n = self.n
        p, kp = _ptr(prim, "prim", 5 * n)
        b, kb = _ptr(bface, "bface", 3 * n)
        a, ka = _ptr(apot, "apot", 3 * n)
        kind = Solver._same_kind(kp, kb, ka)
        Solver._sync_torch(kind)
        self._check(self.L.echo_decomp_set_state(self._h, p, b, a, kind))

    def step(self, max_steps=1, t_end=math.inf):
        done = C.c_int()
        t = C.c_double()
        self._check(self.L.echo_decomp_step(self._h, max_steps, t_end, C.byref(done),
                                            C.byref(t)))
        return done.value, t.value

    def primitives(self):
        out = np.empty((8,) + self.shape)
        p, kind = _ptr(out, "out", 8 * self.n)
        self._check(self.L.echo_decomp_get_primitives(self._h, p, kind))
        return out

    def get_state(self):
        n = self.n
        cons = np.empty((5,) + self.shape)
        bface = np.empty((3,) + self.shape)
        w = np.empty(self.shape)
        t = C.c_double()
        step = C.c_long()
        self._check(self.L.echo_decomp_get_state(
            self._h, _ptr(cons, "cons", 5 * n)[0], _ptr(bface, "bface", 3 * n)[0],
            _ptr(w, "w", n)[0], C.byref(t), C.byref(step), PTR_HOST))
        return cons, bface, w, t.value, step.value

    def counters(self):
        out = (C.c_double * 5)()
        self._check(self.L.echo_decomp_counters(self._h, out))
        return {"c2p_calls": int(out[0]), "newton_it_sum": int(out[1]),
                "newton_it_max": int(out[2]), "c2p_failures": int(out[3]),
                "rec_fallbacks": int(out[4])}


# ---------------------------------------------------------------------------
# the learned Newton starting guess
# ---------------------------------------------------------------------------

def _f32(w):
    w = np.ascontiguousarray(np.asarray(w, dtype=np.float32))
    if w.size != MLP_NPARAM:
        raise ValueError("need %d parameters" % MLP_NPARAM)
    return w


def _dev_f32(t, what, count):
    import torch
    if not (t.is_cuda and t.dtype == torch.float32 and t.is_contiguous() and t.numel() == count):
        raise ValueError("%s: need a contiguous float32 CUDA tensor of %d elements" % (what, count))
    return C.c_void_p(t.data_ptr())


def _chk(st, what):
    if st != ECHO_OK:
        raise EchoError(st, "%s: %s" % (what, lib().echo_last_error(None).decode()))


def mlp_forward(weights, feats):
    """y[n] (torch CUDA float32) for feats[n, 5] (torch CUDA float32)."""
    import torch
    n = feats.shape[0]
    y = torch.empty(n, dtype=torch.float32, device=feats.device)
    w = _f32(weights)
    torch.cuda.synchronize()
    _chk(lib().echo_mlp_forward(w.ctypes.data_as(C.POINTER(C.c_float)),
                                _dev_f32(feats, "feats", 5 * n), n, C.c_void_p(y.data_ptr()), None),
         "echo_mlp_forward")
    return y


def mlp_grad(weights, feats, target):
    """(mean squared loss, gradient[4609]) for one batch (n a multiple of 64)."""
    import torch
    n = feats.shape[0]
    w = _f32(weights)
    g = np.zeros(MLP_NPARAM, dtype=np.float32)
    loss = C.c_float()
    torch.cuda.synchronize()
    fp = C.POINTER(C.c_float)
    _chk(lib().echo_mlp_grad(w.ctypes.data_as(fp), _dev_f32(feats, "feats", 5 * n),
                             _dev_f32(target, "target", n), n, g.ctypes.data_as(fp),
                             C.byref(loss), None), "echo_mlp_grad")
    return loss.value, g


def mlp_train(feats, target, weights, epochs=5, batch=1024, lr=2e-3, beta1=0.9, beta2=0.999,
              eps=1e-8, lr_decay=0.7, seed=0):
    """Adam on the GPU; returns (trained weights, mean loss per epoch)."""
    import torch
    n = feats.shape[0]
    w = _f32(weights).copy()
    hist = np.zeros(epochs, dtype=np.float32)
    cfg = TrainCfg(epochs, batch, lr, beta1, beta2, eps, lr_decay, seed)
    torch.cuda.synchronize()
    fp = C.POINTER(C.c_float)
    _chk(lib().echo_mlp_train(_dev_f32(feats, "feats", 5 * n), _dev_f32(target, "target", n), n,
                              C.byref(cfg), w.ctypes.data_as(fp), hist.ctypes.data_as(fp), None),
         "echo_mlp_train")
    return w, hist


def _solver_mlp_load(self, weights):
    w = _f32(weights)
    self._check(self.L.echo_mlp_load(self._h, w.ctypes.data_as(C.POINTER(C.c_float)),
                                     MLP_NPARAM))


def _solver_mlp_harvest(self, nsteps, stride, feats, target):
    """Advance nsteps steps, collecting features and W/U after every inversion
    into feats[cap, 5], target[cap] (torch CUDA float32); returns the count."""
    import torch
    cap = target.shape[0]
    cnt = C.c_long()
    torch.cuda.synchronize()
    self._check(self.L.echo_mlp_harvest(self._h, nsteps, stride,
                                        _dev_f32(feats, "feats", 5 * cap),
                                        _dev_f32(target, "target", cap), cap, C.byref(cnt)))
    return cnt.value


def _solver_mlp_guess(self, out=None, device=False):
    """The learned starting guess W0 = U y of every cell for the current state
    (echo_mlp_guess), [nz][ny][nx]."""
    out = self._out(self.n, self.shape, device) if out is None else out
    p, kind = _ptr(out, "out", self.n)
    self._sync_torch(kind)
    self._check(self.L.echo_mlp_guess(self._h, p, kind))
    return out


Solver.mlp_load = _solver_mlp_load
Solver.mlp_guess = _solver_mlp_guess
Solver.mlp_harvest = _solver_mlp_harvest
