"""ctypes binding of libfrost.so, the C-ABI declared in include/frost.h.

The module-level functions carry the C names and only marshal arguments (pointers, sizes,
the caller's CUDA stream); every step of the computation runs in the library's CUDA
kernels.  ``Frost`` is a small convenience wrapper over the same calls that allocates output
tensors with PyTorch.  There is no CPU fallback: if the library cannot be loaded the calls
raise.
"""

from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from . import build as _build

FROST_OK, FROST_EINVAL, FROST_ENOMEM, FROST_ECUDA = 0, 1, 2, 3
FROST_ENONFINITE, FROST_ECOINCIDENT, FROST_EDEPTH, FROST_ETIMEOUT = 4, 5, 6, 7
FROST_PREC_FP64, FROST_PREC_MIXED = 0, 1
FROST_SYM_HARMONIC, FROST_SYM_ARITHMETIC, FROST_SYM_NONE = 0, 1, 2
FROST_FLYBY_EXACT = 4  # or-ed into sym: exact fly-by derivative
FROST_HHS_FSI, FROST_HOLD2 = 0, 1  # frost_opts.integrator

_STATUS = {0: "FROST_OK", 1: "FROST_EINVAL", 2: "FROST_ENOMEM", 3: "FROST_ECUDA",
           4: "FROST_ENONFINITE", 5: "FROST_ECOINCIDENT", 6: "FROST_EDEPTH",
           7: "FROST_ETIMEOUT"}


class FrostError(RuntimeError):
    def __init__(self, code: int, where: str, msg: str):
        super().__init__(f"{where}: {_STATUS.get(code, code)}: {msg}")
        self.code = code


class frost_opts(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int32), ("sym", ctypes.c_int32),
                ("eps_soft", ctypes.c_double), ("max_depth", ctypes.c_int32),
                ("cuda_stream", ctypes.c_void_p), ("subtree_max", ctypes.c_int32),
                ("integrator", ctypes.c_int32), ("subtree_blocks", ctypes.c_int32),
                ("branch_streams", ctypes.c_int32), ("sym_cross", ctypes.c_int32)]


class frost_stats(ctypes.Structure):
    _fields_ = [("acc_pairs", ctypes.c_int64), ("grad_pairs", ctypes.c_int64),
                ("tstep_pairs", ctypes.c_int64), ("kernel_launches", ctypes.c_int64),
                ("hhs_calls", ctypes.c_int64), ("fsi_calls", ctypes.c_int64),
                ("max_depth_seen", ctypes.c_int32), ("timing_enabled", ctypes.c_int32),
                ("timed_launches", ctypes.c_int64 * 4), ("timed_ms", ctypes.c_double * 4),
                ("timed_pairs", ctypes.c_int64 * 4), ("subtree_launches", ctypes.c_int64),
                ("level_calls", ctypes.c_int64 * 48), ("level_particles", ctypes.c_int64 * 48),
                ("acc_pairs_reused", ctypes.c_int64), ("subtree_pairs", ctypes.c_int64 * 3),
                ("acc_pairs_symmetric", ctypes.c_int64), ("grad_pairs_symmetric", ctypes.c_int64),
                ("subtree_fsi_beside", ctypes.c_int64)]

    def as_dict(self) -> dict:
        d = {k: getattr(self, k) for k, _ in self._fields_}
        for k in ("timed_launches", "timed_ms", "timed_pairs", "level_calls", "level_particles", "subtree_pairs"):
            d[k] = list(d[k])
        return d


_lock = threading.Lock()
_lib = None

_P = ctypes.c_void_p
_I64 = ctypes.c_int64
_D = ctypes.c_double
_SIGS = {
    "frost_default_opts": (None, [ctypes.POINTER(frost_opts)]),
    "frost_init": (ctypes.c_int, [ctypes.POINTER(_P), _I64, _P, _P, _P, _D, _D,
                                  ctypes.POINTER(frost_opts)]),
    "frost_set_state": (ctypes.c_int, [_P, _P, _P, _D]),
    "frost_get_state": (ctypes.c_int, [_P, _P, _P, ctypes.POINTER(_D)]),
    "frost_accel_gradient": (ctypes.c_int, [_P, _P, _I64, _P, _I64, _D, _P, _P, _P]),
    "frost_timesteps": (ctypes.c_int, [_P, _P, _I64, _P]),
    "frost_accel_pairwise": (ctypes.c_int, [_P, _P, _I64, _P, _I64, _P, _P]),
    "frost_accel_gradient_pairwise": (ctypes.c_int, [_P, _P, _I64, _P, _I64, _D, _P, _P, _P, _P, _P, _P]),
    "frost_partition": (ctypes.c_int, [_P, _P, _I64, _P, _D, _P, _P, ctypes.POINTER(_I64),
                                       ctypes.POINTER(_I64)]),
    "frost_kick": (ctypes.c_int, [_P, _P, _I64, _P, _D]),
    "frost_drift": (ctypes.c_int, [_P, _P, _I64, _D]),
    "frost_fsi": (ctypes.c_int, [_P, _P, _I64, _D]),
    "frost_step": (ctypes.c_int, [_P, _D, _I64]),
    "frost_energy_momentum": (ctypes.c_int, [_P, ctypes.POINTER(_D), ctypes.POINTER(_D), _P, _P]),
    "frost_get_stats": (ctypes.c_int, [_P, ctypes.POINTER(frost_stats)]),
    "frost_reset_stats": (ctypes.c_int, [_P]),
    "frost_set_timing": (ctypes.c_int, [_P, ctypes.c_int32]),
    "frost_autotune": (ctypes.c_int, [_P, _P]),
    "frost_synchronize": (ctypes.c_int, [_P]),
    "frost_clear_error": (ctypes.c_int, [_P]),
    "frost_destroy": (None, [_P]),
    "frost_last_error": (ctypes.c_char_p, []),
    "frost_version": (ctypes.c_char_p, []),
    "frost_accel_noalloc": (ctypes.c_int, [_I64, _P, _P, _D, _D, _P, _P]),
    "frost_peak_probe": (ctypes.c_int, [_P, _P]),
    "frost_init_batch": (ctypes.c_int, [ctypes.POINTER(_P), ctypes.c_int32, _P, _P, _P, _P, _D, _D,
                                        ctypes.POINTER(frost_opts)]),
    "frost_energy_clusters": (ctypes.c_int, [_P, _P, _P, _P, _P]),
}


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load libfrost.so (building it with nvcc first if it is missing or stale)."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.build() if build_if_missing else _build.LIB
            if not os.path.exists(path):
                raise FileNotFoundError(f"libfrost.so not built: {path}")
            lib = ctypes.CDLL(path)
            for name, (res, args) in _SIGS.items():
                fn = getattr(lib, name)
                fn.restype = res
                fn.argtypes = args
            _lib = lib
    return _lib


def _check(code: int, where: str) -> None:
    if code != FROST_OK:
        raise FrostError(code, where, load().frost_last_error().decode())


def _ptr(a):
    """Data pointer of a torch tensor / numpy array, or None."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        assert a.flags.c_contiguous
        return a.ctypes.data
    assert a.is_contiguous()
    return a.data_ptr()


def current_stream_handle():
    import torch
    return torch.cuda.current_stream().cuda_stream


# ---- thin functions with the C names ---------------------------------------------------

def frost_default_opts() -> frost_opts:
    o = frost_opts()
    load().frost_default_opts(ctypes.byref(o))
    return o


def frost_init(m, x, v, G: float, eta: float, opts: frost_opts | None = None) -> ctypes.c_void_p:
    ctx = ctypes.c_void_p()
    n = int(m.shape[0])
    _check(load().frost_init(ctypes.byref(ctx), n, _ptr(m), _ptr(x), _ptr(v), float(G), float(eta),
                             ctypes.byref(opts) if opts is not None else None), "frost_init")
    return ctx


def frost_init_batch(offsets, m, x, v, G: float, eta: float,
                     opts: frost_opts | None = None) -> ctypes.c_void_p:
    ctx = ctypes.c_void_p()
    off = np.ascontiguousarray(offsets, dtype=np.int64)
    _check(load().frost_init_batch(ctypes.byref(ctx), int(off.size - 1), _ptr(off), _ptr(m), _ptr(x),
                                   _ptr(v), float(G), float(eta),
                                   ctypes.byref(opts) if opts is not None else None),
           "frost_init_batch")
    return ctx


def frost_energy_clusters(ctx, n_clusters: int) -> dict:
    T = np.zeros(n_clusters)
    U = np.zeros(n_clusters)
    P = np.zeros((n_clusters, 3))
    L = np.zeros((n_clusters, 3))
    _check(load().frost_energy_clusters(ctx, _ptr(T), _ptr(U), _ptr(P), _ptr(L)),
           "frost_energy_clusters")
    return {"T": T, "U": U, "E": T + U, "P": P, "L": L}


def frost_set_state(ctx, x, v, t: float) -> None:
    _check(load().frost_set_state(ctx, _ptr(x), _ptr(v), float(t)), "frost_set_state")


def frost_get_state(ctx, x, v) -> float:
    t = ctypes.c_double()
    _check(load().frost_get_state(ctx, _ptr(x), _ptr(v), ctypes.byref(t)), "frost_get_state")
    return t.value


def frost_accel_gradient(ctx, active, n_active, source, n_source, eps_grad, acc, acc_tilde,
                         grad) -> None:
    _check(load().frost_accel_gradient(ctx, _ptr(active), int(n_active), _ptr(source),
                                       int(n_source), float(eps_grad), _ptr(acc), _ptr(acc_tilde),
                                       _ptr(grad)), "frost_accel_gradient")


def frost_accel_pairwise(ctx, a, n_a, b, n_b, acc_a, acc_b) -> None:
    _check(load().frost_accel_pairwise(ctx, _ptr(a), int(n_a), _ptr(b), int(n_b), _ptr(acc_a), _ptr(acc_b)),
           "frost_accel_pairwise")


def frost_accel_gradient_pairwise(ctx, a, n_a, b, n_b, eps_grad, acc_a, acc_b, acc_tilde_a, acc_tilde_b,
                                  grad_a, grad_b) -> None:
    _check(load().frost_accel_gradient_pairwise(ctx, _ptr(a), int(n_a), _ptr(b), int(n_b), float(eps_grad),
                                                _ptr(acc_a), _ptr(acc_b), _ptr(acc_tilde_a), _ptr(acc_tilde_b),
                                                _ptr(grad_a), _ptr(grad_b)),
           "frost_accel_gradient_pairwise")


def frost_timesteps(ctx, set_, n_set, tau) -> None:
    _check(load().frost_timesteps(ctx, _ptr(set_), int(n_set), _ptr(tau)), "frost_timesteps")


def frost_partition(ctx, set_, n_set, tau, tau_pivot, S, F):
    ns, nf = ctypes.c_int64(), ctypes.c_int64()
    _check(load().frost_partition(ctx, _ptr(set_), int(n_set), _ptr(tau), float(tau_pivot), _ptr(S),
                                  _ptr(F), ctypes.byref(ns), ctypes.byref(nf)), "frost_partition")
    return ns.value, nf.value


def frost_kick(ctx, set_, n_set, a, dt) -> None:
    _check(load().frost_kick(ctx, _ptr(set_), int(n_set), _ptr(a), float(dt)), "frost_kick")


def frost_drift(ctx, set_, n_set, dt) -> None:
    _check(load().frost_drift(ctx, _ptr(set_), int(n_set), float(dt)), "frost_drift")


def frost_fsi(ctx, set_, n_set, dt) -> None:
    _check(load().frost_fsi(ctx, _ptr(set_), int(n_set), float(dt)), "frost_fsi")


def frost_step(ctx, dt_pivot, n_steps) -> None:
    _check(load().frost_step(ctx, float(dt_pivot), int(n_steps)), "frost_step")


def frost_energy_momentum(ctx):
    ek, ep = ctypes.c_double(), ctypes.c_double()
    P = np.zeros(3)
    L = np.zeros(3)
    _check(load().frost_energy_momentum(ctx, ctypes.byref(ek), ctypes.byref(ep), _ptr(P), _ptr(L)),
           "frost_energy_momentum")
    return ek.value, ep.value, P, L


def frost_get_stats(ctx) -> dict:
    s = frost_stats()
    _check(load().frost_get_stats(ctx, ctypes.byref(s)), "frost_get_stats")
    return s.as_dict()


def frost_reset_stats(ctx) -> None:
    _check(load().frost_reset_stats(ctx), "frost_reset_stats")


def frost_set_timing(ctx, enable: bool) -> None:
    _check(load().frost_set_timing(ctx, 1 if enable else 0), "frost_set_timing")


def frost_autotune(ctx):
    """Run the launch-shape autotuner; returns {kind: {size: waves}} of the choices made
    (negative waves: the small-tile kernel layout)."""
    out = (ctypes.c_int32 * 128)()
    _check(load().frost_autotune(ctx, out), "frost_autotune")
    kinds = ("acc", "grad", "tstep", "acc_feeding_grad")
    return {kinds[q]: {1 << k: int(out[q * 32 + k]) for k in range(32) if out[q * 32 + k] != 0}
            for q in range(4)}


def frost_synchronize(ctx) -> None:
    _check(load().frost_synchronize(ctx), "frost_synchronize")


def frost_clear_error(ctx) -> None:
    _check(load().frost_clear_error(ctx), "frost_clear_error")


def frost_destroy(ctx) -> None:
    load().frost_destroy(ctx)


def frost_last_error() -> str:
    return load().frost_last_error().decode()


def frost_version() -> str:
    return load().frost_version().decode()


def frost_peak_probe(stream=None) -> dict:
    """Measured throughput of the pipes the pair passes run on (see include/frost.h)."""
    out = np.zeros(6)
    _check(load().frost_peak_probe(_ptr(out), stream), "frost_peak_probe")
    return {"ffma_tflops": float(out[0]), "ffma2_tflops": float(out[1]), "dfma_tflops": float(out[2]),
            "mufu_rsqrt_per_s": float(out[3]), "sms": int(out[4]), "threads_per_sm": int(out[5])}


FROST_NOALLOC_MAX_N = 65536


def frost_accel_noalloc(n, m, x, G, eps_soft, acc, stream=None) -> None:
    """Newtonian accelerations of all n particles (device m[n], x[n][3] -> acc[n][3]) without
    any device allocation: the scratch is a static device array of FROST_NOALLOC_MAX_N
    particles shared by all calls (serialise calls whose GPU work could overlap)."""
    _check(load().frost_accel_noalloc(int(n), _ptr(m), _ptr(x), float(G), float(eps_soft),
                                      _ptr(acc), stream), "frost_accel_noalloc")


# ---- convenience wrapper ---------------------------------------------------------------

class Frost:
    """A frost_ctx on the current CUDA device and stream; outputs are torch tensors."""

    def __init__(self, m, x, v, G: float = 1.0, eta: float = 0.2, precision: str = "mixed",
                 sym: int = FROST_SYM_HARMONIC, eps_soft: float = 0.0, max_depth: int = 40,
                 stream=None, subtree_max: int = 0, offsets=None, integrator: int = FROST_HHS_FSI,
                 subtree_blocks: int = 0, branch_streams: int = 0, sym_cross: int = 0):
        import torch
        self.torch = torch
        o = frost_default_opts()
        o.precision = FROST_PREC_MIXED if precision == "mixed" else FROST_PREC_FP64
        o.sym = int(sym)
        o.eps_soft = float(eps_soft)
        o.max_depth = int(max_depth)
        o.cuda_stream = stream if stream is not None else current_stream_handle()
        o.subtree_max = int(subtree_max)
        o.integrator = int(integrator)
        o.subtree_blocks = int(subtree_blocks)
        o.branch_streams = int(branch_streams)
        o.sym_cross = int(sym_cross)
        self.n = int(np.asarray(m).shape[0]) if not hasattr(m, "shape") else int(m.shape[0])
        self.G = G
        self.eta = eta
        self.precision = precision
        mm = _as_f64(m)
        xx = _as_f64(x).reshape(-1, 3)
        vv = _as_f64(v).reshape(-1, 3)
        self.offsets = None
        if offsets is not None:
            self.offsets = np.ascontiguousarray(offsets, dtype=np.int64)
            self.ctx = frost_init_batch(self.offsets, mm, xx, vv, G, eta, o)
        else:
            self.ctx = frost_init(mm, xx, vv, G, eta, o)

    def close(self):
        if getattr(self, "ctx", None) is not None:
            frost_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _dev(self, a, dtype):
        t = self.torch
        if a is None:
            return None
        if not isinstance(a, t.Tensor):
            a = t.as_tensor(np.ascontiguousarray(a))
        return a.to(device="cuda", dtype=dtype).contiguous()

    def accel_gradient(self, active=None, source=None, eps_grad=0.0, n_active=None, n_source=None,
                       want=("acc", "acc_tilde", "grad")):
        t = self.torch
        A = self._dev(active, t.int32)
        B = self._dev(source, t.int32)
        na = int(A.numel()) if A is not None else (self.n if n_active is None else n_active)
        ns = int(B.numel()) if B is not None else (self.n if n_source is None else n_source)
        if active is not None and source is not None and active is source:
            B = A
        out = {k: t.empty((na, 3), dtype=t.float64, device="cuda") for k in want}
        frost_accel_gradient(self.ctx, A, na, B, ns, eps_grad, out.get("acc"), out.get("acc_tilde"),
                             out.get("grad"))
        return out

    def accel_pairwise(self, a, b):
        """Accelerations of the disjoint lists a and b due to each other, each pair once."""
        t = self.torch
        A = self._dev(a, t.int32)
        B = self._dev(b, t.int32)
        out_a = t.empty((int(A.numel()), 3), dtype=t.float64, device="cuda")
        out_b = t.empty((int(B.numel()), 3), dtype=t.float64, device="cuda")
        frost_accel_pairwise(self.ctx, A, int(A.numel()), B, int(B.numel()), out_a, out_b)
        return out_a, out_b

    def accel_gradient_pairwise(self, a, b, eps_grad):
        """The force-gradient kick of the disjoint lists a and b due to each other: per list
        the Newtonian acceleration, a~ and the gradient ({"acc", "acc_tilde", "grad"} x
        {"a", "b"}, [n][3] each); mixed mode: each pair once for both lists."""
        t = self.torch
        A = self._dev(a, t.int32)
        B = self._dev(b, t.int32)
        na, nb = int(A.numel()), int(B.numel())
        out = {k + "_" + s: t.empty((n, 3), dtype=t.float64, device="cuda")
               for k in ("acc", "acc_tilde", "grad") for s, n in (("a", na), ("b", nb))}
        frost_accel_gradient_pairwise(self.ctx, A, na, B, nb, eps_grad, out["acc_a"], out["acc_b"],
                                      out["acc_tilde_a"], out["acc_tilde_b"], out["grad_a"], out["grad_b"])
        return out

    def timesteps(self, set_=None, n_set=None):
        t = self.torch
        P = self._dev(set_, t.int32)
        n = int(P.numel()) if P is not None else (self.n if n_set is None else n_set)
        tau = t.empty(n, dtype=t.float64, device="cuda")
        frost_timesteps(self.ctx, P, n, tau)
        return tau

    def partition(self, set_, tau, tau_pivot):
        t = self.torch
        P = self._dev(set_, t.int32)
        tt = self._dev(tau, t.float64)
        n = int(tt.numel())
        S = t.empty(max(n, 1), dtype=t.int32, device="cuda")
        F = t.empty(max(n, 1), dtype=t.int32, device="cuda")
        ns, nf = frost_partition(self.ctx, P, n, tt, tau_pivot, S, F)
        return S[:ns], F[:nf]

    def kick(self, set_, a, dt):
        t = self.torch
        P = self._dev(set_, t.int32)
        aa = self._dev(a, t.float64)
        frost_kick(self.ctx, P, aa.shape[0], aa, dt)

    def drift(self, set_, dt, n_set=None):
        t = self.torch
        P = self._dev(set_, t.int32)
        n = int(P.numel()) if P is not None else (self.n if n_set is None else n_set)
        frost_drift(self.ctx, P, n, dt)

    def fsi(self, set_=None, dt=0.0, n_set=None):
        t = self.torch
        P = self._dev(set_, t.int32)
        n = int(P.numel()) if P is not None else (self.n if n_set is None else n_set)
        frost_fsi(self.ctx, P, n, dt)
        frost_synchronize(self.ctx)

    def step(self, dt_pivot, n_steps=1):
        frost_step(self.ctx, dt_pivot, n_steps)

    def state(self):
        x = np.zeros((self.n, 3))
        v = np.zeros((self.n, 3))
        tt = frost_get_state(self.ctx, x, v)
        return x, v, tt

    def set_state(self, x=None, v=None, t=0.0):
        frost_set_state(self.ctx, None if x is None else _as_f64(x).reshape(-1, 3),
                        None if v is None else _as_f64(v).reshape(-1, 3), t)

    def energy(self):
        ek, ep, P, L = frost_energy_momentum(self.ctx)
        return {"T": ek, "U": ep, "E": ek + ep, "P": P, "L": L}

    def cluster_energies(self):
        return frost_energy_clusters(self.ctx, self.offsets.size - 1)

    def stats(self):
        return frost_get_stats(self.ctx)

    def reset_stats(self):
        frost_reset_stats(self.ctx)

    def set_timing(self, on: bool):
        frost_set_timing(self.ctx, on)

    def autotune(self):
        """Launch shapes of the pair kernels ({kind: {size: waves}}); on a batch context the
        team split, {"team_min_n": ..., "team_blocks": ...}."""
        if self.offsets is not None:
            out = (ctypes.c_int32 * 128)()
            _check(load().frost_autotune(self.ctx, out), "frost_autotune")
            return {"team_min_n": int(out[0]), "team_blocks": int(out[1])}
        return frost_autotune(self.ctx)


def _as_f64(a):
    try:
        import torch
        if isinstance(a, torch.Tensor):
            return a.to(torch.float64).contiguous()
    except ImportError:
        pass
    return np.ascontiguousarray(a, dtype=np.float64)
