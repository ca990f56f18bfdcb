"""GB300-native space-time Vanka-multigrid GMRES solver (Python binding of libstg.so).

The solver (Anselmann & Bause, Sec. 3) preconditions flexible GMRES with one
geometric-multigrid V-cycle whose smoother is the local Vanka operator of
Eq. (3.4) applied through the averaging loop (S0)-(S3), for the Newton/Oseen
Jacobian (Eq. (3.3)) of the dG(k)-in-time, (Q2)^d x P1disc-in-space slab
problem of Eq. (2.2).  All arithmetic runs in the CUDA library (include/stg.h);
this module only marshals arguments: torch provides device memory and a
stream.  There is no CPU fallback: every call fails loudly when libstg.so is
missing or no CUDA device is present.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libstg.so")

STG_OK, STG_EINVAL, STG_ENOMEM, STG_ECUDA, STG_ESINGULAR, STG_ENOCONV, STG_ETIMEOUT = range(7)
STG_OSEEN, STG_NEWTON = 0, 1
STG_VANKA_AVERAGED, STG_VANKA_COLOURED = 0, 1
STG_F64, STG_F32, STG_BF16 = 0, 1, 2
PREC = {"f64": STG_F64, "f32": STG_F32, "bf16": STG_BF16}

EXPORTED = ("stg_options_default", "stg_setup", "stg_update_linearisation", "stg_set_slab_length",
            "stg_apply_jacobian",
            "stg_apply_level_jacobian", "stg_vcycle", "stg_smooth", "stg_prolongate", "stg_restrict",
            "stg_coarse_solve", "stg_gmres_solve", "stg_get_sizes", "stg_get_local_inverse", "stg_profile",
            "stg_profile_read", "stg_kernel_launches", "stg_invert_local_noalloc", "stg_newton_slab",
            "stg_slab_initial_guess", "stg_obstacle_forces", "stg_autotune", "stg_set_wait_limit", "stg_get_colour_variant",
            "stg_set_colour_variant",
            "stg_batch_create", "stg_batch_gmres_solve",
            "stg_batch_destroy", "stg_cnn_create", "stg_cnn_n_params", "stg_cnn_set_params",
            "stg_cnn_get_params", "stg_cnn_forward", "stg_cnn_gradients", "stg_cnn_adam_step", "stg_cnn_train",
            "stg_cnn_last_error", "stg_cnn_destroy", "stg_warm_features", "stg_warm_target", "stg_warm_start",
            "stg_warm_scales", "stg_last_error", "stg_destroy")


class StgError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"stg status {status}: {msg}")
        self.status = status


class stg_mesh(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int), ("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
                ("n_levels", ctypes.c_int), ("x0", ctypes.c_double), ("x1", ctypes.c_double),
                ("y0", ctypes.c_double), ("y1", ctypes.c_double), ("z0", ctypes.c_double),
                ("z1", ctypes.c_double), ("dirichlet_faces", ctypes.c_uint), ("obstacle", ctypes.c_int * 4),
                ("order", ctypes.c_int)]


class stg_options(ctypes.Structure):
    _fields_ = [("linearisation", ctypes.c_int), ("smoother", ctypes.c_int), ("nu1", ctypes.c_int),
                ("nu2", ctypes.c_int), ("omega", ctypes.c_double), ("gamma1", ctypes.c_double),
                ("gamma2", ctypes.c_double), ("factor_prec", ctypes.c_int), ("vcycle_prec", ctypes.c_int),
                ("gmres_restart", ctypes.c_int), ("gmres_maxit", ctypes.c_int), ("gmres_rtol", ctypes.c_double),
                ("gmres_atol", ctypes.c_double), ("use_graph", ctypes.c_int), ("coarse_refine", ctypes.c_int),
                ("coarse_prec", ctypes.c_int), ("overlap_launches", ctypes.c_int)]


class stg_cnn_desc(ctypes.Structure):
    _fields_ = [("n_layers", ctypes.c_int), ("channels", ctypes.c_int * 9), ("height", ctypes.c_int),
                ("width", ctypes.c_int), ("max_batch", ctypes.c_int)]


_lib = None


def load_library(path: str = LIB_PATH) -> ctypes.CDLL:
    """Loads libstg.so and declares the signatures of include/stg.h."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"{path} is missing: build it with `python -c 'import __graft_entry__ as g; g.build()'`")
    lib = ctypes.CDLL(path)
    P, D, I, LL = ctypes.c_void_p, ctypes.c_double, ctypes.c_int, ctypes.c_longlong
    sig = {
        "stg_options_default": (I, [ctypes.POINTER(stg_options)]),
        "stg_setup": (I, [ctypes.POINTER(stg_mesh), I, D, D, P, ctypes.POINTER(stg_options), P,
                          ctypes.POINTER(P)]),
        "stg_update_linearisation": (I, [P, P]),
        "stg_set_slab_length": (I, [P, D]),
        "stg_apply_jacobian": (I, [P, P, P]),
        "stg_apply_level_jacobian": (I, [P, I, P, P]),
        "stg_vcycle": (I, [P, P, P]),
        "stg_smooth": (I, [P, I, I, P, P]),
        "stg_prolongate": (I, [P, I, P, P]),
        "stg_restrict": (I, [P, I, P, P]),
        "stg_coarse_solve": (I, [P, P, P]),
        "stg_gmres_solve": (I, [P, P, P, ctypes.POINTER(I), ctypes.POINTER(D)]),
        "stg_get_sizes": (I, [P, I, ctypes.POINTER(LL), ctypes.POINTER(LL), ctypes.POINTER(I)]),
        "stg_get_local_inverse": (I, [P, I, LL, P]),
        "stg_profile": (I, [P, I]),
        "stg_profile_read": (I, [P, ctypes.POINTER(D), ctypes.POINTER(LL), ctypes.POINTER(LL)]),
        "stg_kernel_launches": (LL, []),
        "stg_invert_local_noalloc": (I, [I, LL, P, P, P]),
        "stg_newton_slab": (I, [P, P, P, P, P, D, D, I, ctypes.POINTER(I), ctypes.POINTER(I), ctypes.POINTER(D)]),
        "stg_slab_initial_guess": (I, [P, P, P]),
        "stg_obstacle_forces": (I, [P, P, P]),
        "stg_autotune": (I, [P, ctypes.POINTER(I), ctypes.POINTER(D)]),
        "stg_set_wait_limit": (I, [LL]),
        "stg_get_colour_variant": (I, [P, I, ctypes.POINTER(I)]),
        "stg_set_colour_variant": (I, [P, I, I]),
        "stg_batch_create": (I, [I, ctypes.POINTER(P), ctypes.POINTER(P)]),
        "stg_batch_gmres_solve": (I, [P, ctypes.POINTER(P), ctypes.POINTER(P), ctypes.POINTER(I),
                                      ctypes.POINTER(D)]),
        "stg_batch_destroy": (None, [P]),
        "stg_cnn_create": (I, [ctypes.POINTER(stg_cnn_desc), P, ctypes.POINTER(P)]),
        "stg_cnn_n_params": (I, [P, ctypes.POINTER(LL)]),
        "stg_cnn_set_params": (I, [P, P]),
        "stg_cnn_get_params": (I, [P, P]),
        "stg_cnn_forward": (I, [P, P, P, I]),
        "stg_cnn_gradients": (I, [P, P, P, I, P, ctypes.POINTER(D)]),
        "stg_cnn_adam_step": (I, [P, P, ctypes.c_float, ctypes.c_float, ctypes.c_float, ctypes.c_float]),
        "stg_cnn_train": (I, [P, P, P, I, P, I, I, ctypes.c_float, P]),
        "stg_cnn_last_error": (ctypes.c_char_p, [P]),
        "stg_cnn_destroy": (I, [P]),
        "stg_warm_features": (I, [P, P, P, ctypes.c_float, ctypes.c_float, P]),
        "stg_warm_target": (I, [P, P, P, P, ctypes.c_float, P]),
        "stg_warm_start": (I, [P, P, P, P, ctypes.c_float, ctypes.c_float, P]),
        "stg_warm_scales": (I, [P, P, P, ctypes.POINTER(D), ctypes.POINTER(D)]),
        "stg_last_error": (ctypes.c_char_p, [P]),
        "stg_destroy": (None, [P]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def make_mesh(spec) -> stg_mesh:
    """stg_mesh from a stg_inputs.MeshSpec-like object (dim, n, lo, hi, n_levels, dirichlet)."""
    n = list(spec.n) + [1] * (3 - len(spec.n))
    lo = list(spec.lo) + [0.0] * (3 - len(spec.lo))
    hi = list(spec.hi) + [1.0] * (3 - len(spec.hi))
    ob = tuple(getattr(spec, "obstacle", ()) or (0, 0, 0, 0))
    return stg_mesh(spec.dim, n[0], n[1], n[2], spec.n_levels, lo[0], hi[0], lo[1], hi[1], lo[2], hi[2],
                    spec.dirichlet, (ctypes.c_int * 4)(*ob), int(getattr(spec, "order", 2)))


def make_options(**kw) -> stg_options:
    lib = load_library()
    o = stg_options()
    lib.stg_options_default(ctypes.byref(o))
    for key, val in kw.items():
        if key in ("factor_prec", "vcycle_prec", "coarse_prec") and isinstance(val, str):
            val = PREC[val]
        if key == "smoother" and isinstance(val, str):
            val = {"averaged": STG_VANKA_AVERAGED, "coloured": STG_VANKA_COLOURED}[val]
        if key == "linearisation" and isinstance(val, str):
            val = {"oseen": STG_OSEEN, "newton": STG_NEWTON}[val]
        setattr(o, key, val)
    return o


def _check(lib, ctx, status: int):
    if status not in (STG_OK, STG_ENOCONV):
        msg = lib.stg_last_error(ctx)
        raise StgError(status, msg.decode() if msg else "")
    return status


def set_wait_limit(spins: int) -> None:
    """Iteration limit of the staged smoother's waits (fault injection; default 2**22)."""
    lib = load_library()
    st = lib.stg_set_wait_limit(int(spins))
    if st != STG_OK:
        raise StgError(st, "stg_set_wait_limit")


class Solver:
    """One slab problem on one GPU: wraps an stg_ctx and a private CUDA stream.

    All tensors are float64 CUDA tensors in the C-ABI order of X_n.  Each call
    orders itself after the caller's current stream and makes the caller's
    stream wait for it, so it composes with ordinary torch code.
    """

    def __init__(self, spec, k: int, nu: float, tau: float, w, **options):
        import torch

        if not torch.cuda.is_available():
            raise RuntimeError("paper_2210_02690_gb300 needs a CUDA device; there is no CPU path")
        self.torch = torch
        self.lib = load_library()
        self.spec, self.k, self.nu, self.tau = spec, k, nu, tau
        self.device = torch.device("cuda", torch.cuda.current_device())
        self.stream = torch.cuda.Stream(device=self.device)
        self.mesh = make_mesh(spec)
        self.opts = make_options(**options)
        w = self._dev(w)
        ctx = ctypes.c_void_p()
        self._enter()
        st = self.lib.stg_setup(ctypes.byref(self.mesh), k, nu, tau, ctypes.c_void_p(w.data_ptr()),
                                ctypes.byref(self.opts), ctypes.c_void_p(self.stream.cuda_stream),
                                ctypes.byref(ctx))
        self._leave()
        if st != STG_OK:
            msg = self.lib.stg_last_error(None)
            raise StgError(st, msg.decode() if msg else "")
        self.ctx = ctx

    # -- stream plumbing
    def _enter(self):
        self.stream.wait_stream(self.torch.cuda.current_stream(self.device))

    def _leave(self):
        self.torch.cuda.current_stream(self.device).wait_stream(self.stream)

    def _dev(self, a):
        t = self.torch
        if isinstance(a, np.ndarray):
            a = t.from_numpy(np.ascontiguousarray(a, dtype=np.float64))
        a = a.to(device=self.device, dtype=t.float64).contiguous()
        return a

    @staticmethod
    def _p(a):
        return ctypes.c_void_p(a.data_ptr())

    def _call(self, fn, *args):
        self._enter()
        try:
            return _check(self.lib, self.ctx, fn(self.ctx, *args))
        finally:
            self._leave()

    def sizes(self, level: int = -1):
        level = self.spec.n_levels - 1 if level < 0 else level
        nd, nc, npch = ctypes.c_longlong(), ctypes.c_longlong(), ctypes.c_int()
        _check(self.lib, self.ctx, self.lib.stg_get_sizes(self.ctx, level, ctypes.byref(nd), ctypes.byref(nc),
                                                          ctypes.byref(npch)))
        return nd.value, nc.value, npch.value

    def update_linearisation(self, w):
        w = self._dev(w)
        self._call(self.lib.stg_update_linearisation, self._p(w))

    def set_slab_length(self, tau: float):
        """New slab length tau; every level is re-assembled at the current linearisation velocity."""
        self._call(self.lib.stg_set_slab_length, float(tau))
        self.tau = tau

    def apply_jacobian(self, x, level: int = -1):
        level = self.spec.n_levels - 1 if level < 0 else level
        x = self._dev(x)
        y = self.torch.empty_like(x)
        self._call(self.lib.stg_apply_level_jacobian, level, self._p(x), self._p(y))
        return y

    def vcycle(self, b, out=None):
        b = self._dev(b)
        x = self.torch.empty_like(b) if out is None else out
        self._call(self.lib.stg_vcycle, self._p(b), self._p(x))
        return x

    def smooth(self, level: int, sweeps: int, b, x):
        b = self._dev(b)
        x = self._dev(x).clone()
        self._call(self.lib.stg_smooth, level, sweeps, self._p(b), self._p(x))
        return x

    def prolongate(self, level: int, xc, xf):
        xc = self._dev(xc)
        xf = self._dev(xf).clone()
        self._call(self.lib.stg_prolongate, level, self._p(xc), self._p(xf))
        return xf

    def restrict(self, level: int, rf):
        rf = self._dev(rf)
        nd, _, _ = self.sizes(level - 1)
        bc = self.torch.empty(nd, dtype=self.torch.float64, device=self.device)
        self._call(self.lib.stg_restrict, level, self._p(rf), self._p(bc))
        return bc

    def coarse_solve(self, b):
        b = self._dev(b)
        x = self.torch.empty_like(b)
        self._call(self.lib.stg_coarse_solve, self._p(b), self._p(x))
        return x

    def gmres_solve(self, b, x0=None, out=None):
        """Returns (x, total inner iterations, relative residual, converged)."""
        b = self._dev(b)
        if out is not None:
            x = out
            if x0 is None:
                x.zero_()
            else:
                x.copy_(self._dev(x0))
        else:
            x = self.torch.zeros_like(b) if x0 is None else self._dev(x0).clone()
        its, rel = ctypes.c_int(), ctypes.c_double()
        st = self._call(self.lib.stg_gmres_solve, self._p(b), self._p(x), ctypes.byref(its), ctypes.byref(rel))
        return x, its.value, rel.value, st == STG_OK

    def newton_slab(self, X0, v_prev=None, f=None, g=None, rtol=1e-8, atol=0.0, maxit=20):
        """Damped Newton for the slab; returns (X, Newton steps, GMRES iterations, final ||F||, converged)."""
        X = self._dev(X0).clone()
        opt = [self._dev(a) if a is not None else None for a in (v_prev, f, g)]
        ptr = [self._p(a) if a is not None else None for a in opt]
        steps, its, res = ctypes.c_int(), ctypes.c_int(), ctypes.c_double()
        st = self._call(self.lib.stg_newton_slab, ptr[0], ptr[1], ptr[2], self._p(X), rtol, atol, maxit,
                        ctypes.byref(steps), ctypes.byref(its), ctypes.byref(res))
        return X, steps.value, its.value, res.value, st == STG_OK

    def slab_initial_guess(self, X_prev):
        Xp = self._dev(X_prev)
        X0 = self.torch.empty_like(Xp)
        self._call(self.lib.stg_slab_initial_guess, self._p(Xp), self._p(X0))
        return X0

    def obstacle_forces(self, X) -> np.ndarray:
        """(k+1, 2) force of the fluid on the obstacle (drag, lift) at every Radau node of X."""
        Xd = self._dev(X)
        out = np.zeros((self.k + 1, 2))
        self._call(self.lib.stg_obstacle_forces, self._p(Xd), out.ctypes.data_as(ctypes.c_void_p))
        return out

    # -- learned warm start of the next slab (2D)
    def node_grid(self):
        """(height, width) of the finest level's Q2 node grid."""
        return 2 * self.spec.n[1] + 1, 2 * self.spec.n[0] + 1

    def warm_features(self, X_n, X_prev, scale_v: float, scale_d: float, out=None):
        Xn, Xp = self._dev(X_n), self._dev(X_prev)
        H, W = self.node_grid()
        f = out if out is not None else self.torch.empty((2 * self.spec.dim, H, W), dtype=self.torch.float32,
                                                         device=self.device)
        self._call(self.lib.stg_warm_features, self._p(Xn), self._p(Xp), scale_v, scale_d, self._p(f))
        return f

    def warm_target(self, X_n, X_prev, X_next, scale_d: float, out=None):
        Xn, Xp, Xx = self._dev(X_n), self._dev(X_prev), self._dev(X_next)
        H, W = self.node_grid()
        t = out if out is not None else self.torch.empty((self.spec.dim * (self.k + 1), H, W),
                                                         dtype=self.torch.float32, device=self.device)
        self._call(self.lib.stg_warm_target, self._p(Xn), self._p(Xp), self._p(Xx), scale_d, self._p(t))
        return t

    def warm_start(self, net, X_n, X_prev, scale_v: float, scale_d: float):
        """Initial guess for the next slab: linear extrapolation plus the network's correction
        (net None: linear extrapolation alone)."""
        Xn, Xp = self._dev(X_n), self._dev(X_prev)
        X0 = self.torch.empty_like(Xn)
        self._call(self.lib.stg_warm_start, net.handle if net is not None else None, self._p(Xn), self._p(Xp),
                   scale_v, scale_d, self._p(X0))
        return X0

    def warm_scales(self, X_n, X_prev):
        """(rms of v_n, rms of v_n - v_{n-1}) over the nodal velocity entries."""
        Xn, Xp = self._dev(X_n), self._dev(X_prev)
        a, b = ctypes.c_double(), ctypes.c_double()
        self._call(self.lib.stg_warm_scales, self._p(Xn), self._p(Xp), ctypes.byref(a), ctypes.byref(b))
        return a.value, b.value

    def local_inverse(self, level: int, cell: int) -> np.ndarray:
        n = self.sizes(level)[2]
        out = np.zeros((n, n))
        self.stream.synchronize()
        _check(self.lib, self.ctx, self.lib.stg_get_local_inverse(self.ctx, level, cell,
                                                                  out.ctypes.data_as(ctypes.c_void_p)))
        return out

    def profile(self, enable: bool):
        """Start (and reset) or stop CUDA-event timing of the finest-level colour kernels."""
        self._call(self.lib.stg_profile, 1 if enable else 0)

    def profile_read(self):
        """(device milliseconds, launches, patches) accumulated since profiling started."""
        ms, n, p = ctypes.c_double(), ctypes.c_longlong(), ctypes.c_longlong()
        self.lib.stg_profile_read(self.ctx, ctypes.byref(ms), ctypes.byref(n), ctypes.byref(p))
        return ms.value, n.value, p.value

    def autotune(self):
        """Picks the fastest colour-kernel variant per level; returns (finest variant, sweep ms)."""
        v, ms = ctypes.c_int(), ctypes.c_double()
        self._call(self.lib.stg_autotune, ctypes.byref(v), ctypes.byref(ms))
        return v.value, ms.value

    def colour_variants(self):
        """Colour-kernel variant of every level >= 1 (finest last)."""
        out = []
        for level in range(1, self.spec.n_levels):
            v = ctypes.c_int()
            _check(self.lib, self.ctx, self.lib.stg_get_colour_variant(self.ctx, level, ctypes.byref(v)))
            out.append(v.value)
        return out

    def set_colour_variants(self, variants):
        """Sets the colour-kernel variant of levels 1.. (as returned by colour_variants)."""
        for level, v in enumerate(variants, start=1):
            self._call(self.lib.stg_set_colour_variant, level, int(v))

    def kernel_launches(self) -> int:
        return int(self.lib.stg_kernel_launches())

    def close(self):
        if getattr(self, "ctx", None):
            self.lib.stg_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch:
    """Several independent Solvers solved together: one CUDA graph holds all V-cycles."""

    def __init__(self, solvers):
        self.solvers = list(solvers)
        self.lib = load_library()
        n = len(self.solvers)
        arr = (ctypes.c_void_p * n)(*[s.ctx for s in self.solvers])
        out = ctypes.c_void_p()
        for s in self.solvers:
            s.stream.synchronize()
        st = self.lib.stg_batch_create(n, arr, ctypes.byref(out))
        if st != STG_OK:
            msg = self.lib.stg_last_error(None)
            raise StgError(st, msg.decode() if msg else "")
        self.handle = out

    def gmres_solve(self, rhs, x0=None):
        import torch

        n = len(self.solvers)
        bs = [s._dev(b) for s, b in zip(self.solvers, rhs)]
        xs = [torch.zeros_like(b) if x0 is None else s._dev(x).clone() for s, b, x in
              zip(self.solvers, bs, x0 if x0 is not None else [None] * n)]
        for s in self.solvers:
            s._enter()
        pb = (ctypes.c_void_p * n)(*[b.data_ptr() for b in bs])
        px = (ctypes.c_void_p * n)(*[x.data_ptr() for x in xs])
        its = (ctypes.c_int * n)()
        rel = (ctypes.c_double * n)()
        st = self.lib.stg_batch_gmres_solve(self.handle, pb, px, its, rel)
        for s in self.solvers:
            s._leave()
        if st not in (STG_OK, STG_ENOCONV):
            msg = self.lib.stg_last_error(None)
            raise StgError(st, msg.decode() if msg else "")
        return xs, list(its), list(rel), st == STG_OK

    def close(self):
        if getattr(self, "handle", None):
            self.lib.stg_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Cnn:
    """The warm-start network (stg_cnn): 3x3 convolutions with tanh, trained with Adam.

    channels = [c_0, ..., c_L]; tensors are float32 CUDA tensors [batch][c][height][width].
    """

    def __init__(self, channels, height: int, width: int, max_batch: int):
        import torch

        if not torch.cuda.is_available():
            raise RuntimeError("paper_2210_02690_gb300 needs a CUDA device; there is no CPU path")
        self.torch = torch
        self.lib = load_library()
        self.channels = list(channels)
        self.height, self.width = height, width
        self.device = torch.device("cuda", torch.cuda.current_device())
        self.stream = torch.cuda.Stream(device=self.device)
        d = stg_cnn_desc()
        d.n_layers = len(channels) - 1
        for i, c in enumerate(channels):
            d.channels[i] = c
        d.height, d.width, d.max_batch = height, width, max_batch
        h = ctypes.c_void_p()
        st = self.lib.stg_cnn_create(ctypes.byref(d), ctypes.c_void_p(self.stream.cuda_stream), ctypes.byref(h))
        if st != STG_OK:
            msg = self.lib.stg_cnn_last_error(None) or self.lib.stg_last_error(None)
            raise StgError(st, msg.decode() if msg else "")
        self.handle = h
        n = ctypes.c_longlong()
        self.lib.stg_cnn_n_params(h, ctypes.byref(n))
        self.n_params = n.value

    def _enter(self):
        self.stream.wait_stream(self.torch.cuda.current_stream(self.device))

    def _leave(self):
        self.torch.cuda.current_stream(self.device).wait_stream(self.stream)

    def _call(self, fn, *args):
        self._enter()
        try:
            st = fn(self.handle, *args)
            if st != STG_OK:
                msg = self.lib.stg_cnn_last_error(self.handle)
                raise StgError(st, msg.decode() if msg else "")
        finally:
            self._leave()

    def _f32(self, a):
        t = self.torch
        if isinstance(a, np.ndarray):
            a = t.from_numpy(np.ascontiguousarray(a, dtype=np.float32))
        return a.to(device=self.device, dtype=t.float32).contiguous()

    def set_params(self, flat):
        a = np.ascontiguousarray(np.asarray(flat, dtype=np.float32))
        assert a.size == self.n_params
        self._call(self.lib.stg_cnn_set_params, a.ctypes.data_as(ctypes.c_void_p))

    def get_params(self) -> np.ndarray:
        a = np.zeros(self.n_params, dtype=np.float32)
        self._call(self.lib.stg_cnn_get_params, a.ctypes.data_as(ctypes.c_void_p))
        return a

    def forward(self, x):
        x = self._f32(x)
        y = self.torch.empty((x.shape[0], self.channels[-1], self.height, self.width), dtype=self.torch.float32,
                             device=self.device)
        self._call(self.lib.stg_cnn_forward, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(y.data_ptr()),
                   x.shape[0])
        return y

    def gradients(self, x, t):
        """(loss, flat gradient tensor)."""
        x, t = self._f32(x), self._f32(t)
        g = self.torch.empty(self.n_params, dtype=self.torch.float32, device=self.device)
        loss = ctypes.c_double()
        self._call(self.lib.stg_cnn_gradients, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(t.data_ptr()),
                   x.shape[0], ctypes.c_void_p(g.data_ptr()), ctypes.byref(loss))
        return loss.value, g

    def adam_step(self, grad, lr: float, beta1=0.9, beta2=0.999, eps=1e-8):
        g = self._f32(grad)
        self._call(self.lib.stg_cnn_adam_step, ctypes.c_void_p(g.data_ptr()), lr, beta1, beta2, eps)

    def train(self, x_all, t_all, order, batch: int, lr: float):
        """Adam steps over the sample indices `order` (len = steps * batch); returns the losses."""
        x, t = self._f32(x_all), self._f32(t_all)
        order = np.ascontiguousarray(np.asarray(order, dtype=np.int32))
        steps = order.size // batch
        losses = np.zeros(steps)
        self._call(self.lib.stg_cnn_train, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(t.data_ptr()),
                   x.shape[0], order.ctypes.data_as(ctypes.c_void_p), batch, steps, lr,
                   losses.ctypes.data_as(ctypes.c_void_p))
        return losses

    def close(self):
        if getattr(self, "handle", None):
            self.lib.stg_cnn_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
