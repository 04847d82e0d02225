"""Plain FP64 CPU oracle for the HHS-FSI hot path -- test infrastructure only.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline leg may import
this package.  The computation lives in ``frost_oracle.c`` (plain C, FP64, one double loop
per pass, written from the paper's equations and algorithms); this module compiles it with
gcc and wraps it with ctypes and numpy.  It shares no code with the CUDA path.

Functions with their sources in the paper:
  acc, accel_gradient, grad  -- Eq. acc-newton, Eq. acc-gradient(-g), Eqs. force-*-inter
  pair_timescales            -- Eqs. dt-freefall, dt-flyby and their derivatives
  sym_harmonic, sym_arithmetic -- Eq. time-step-factor
  timesteps                  -- Sec. 4.3 (min over j of symmetrised pair timescales)
  partition                  -- Sec. 3.1 slow/fast split
  fsi, hhs_fsi, steps        -- Algorithms fsi, hhs-fsi and the main loop of frost
  energy                     -- E = T + U, P, L (Sec. 2.3)
"""

from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "frost_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

OK, EINVAL, ENOMEM, ENONFINITE, ECOINCIDENT, EDEPTH = 0, 1, 2, 4, 5, 6
SYM_HARMONIC, SYM_ARITHMETIC, SYM_NONE = 0, 1, 2
FLYBY_EXACT = 4  # or-ed into sym: exact fly-by derivative (first line of Eq. dt-flyby-derivative)


class OracleError(RuntimeError):
    def __init__(self, code: int, what: str):
        super().__init__(f"oracle {what} failed with status {code}")
        self.code = code


def build(force: bool = False) -> str:
    """Compile frost_oracle.c into oracle/_build/liboracle.so (gcc, -O2, OpenMP if present)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    base = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared", _SRC, "-lm"]
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    try:
        subprocess.run(base[:-1] + ["-fopenmp", "-o", tmp, "-lm"], check=True,
                       capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base[:-1] + ["-o", tmp, "-lm"], check=True, capture_output=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            P = ctypes.c_void_p
            i64 = ctypes.c_int64
            d = ctypes.c_double
            ci = ctypes.c_int
            lib.or_acc.argtypes = [P, P, P, i64, P, i64, d, d, P]
            lib.or_grad.argtypes = [P, P, P, i64, P, P, i64, P, d, d, P]
            lib.or_accel_gradient.argtypes = [i64, P, P, P, i64, P, i64, d, d, d, P, P]
            lib.or_pair_timescales.argtypes = [P, P, d, P, P, d, d, P]
            lib.or_pair_timescales.restype = None
            lib.or_pair_timescales_exact.argtypes = [P, P, P, d, P, P, P, d, d, P]
            lib.or_pair_timescales_exact.restype = None
            lib.or_sym_harmonic.argtypes = [d]
            lib.or_sym_harmonic.restype = d
            lib.or_sym_arithmetic.argtypes = [d]
            lib.or_sym_arithmetic.restype = d
            lib.or_timesteps.argtypes = [P, P, P, P, i64, d, d, ci, P]
            lib.or_timesteps_ex.argtypes = [P, P, P, P, i64, P, i64, d, d, d, ci, P]
            lib.or_steps_hold.argtypes = [i64, P, P, P, d, i64, d, d, d, ci, ci]
            lib.or_timesteps_of.argtypes = [P, P, P, P, i64, P, i64, d, d, ci, P]
            lib.or_partition.argtypes = [P, i64, P, d, P, P, P, P]
            lib.or_partition.restype = None
            lib.or_kick.argtypes = [P, i64, P, P, d]
            lib.or_kick.restype = None
            lib.or_drift.argtypes = [P, i64, P, P, d]
            lib.or_drift.restype = None
            lib.or_fsi.argtypes = [i64, P, P, P, P, i64, d, d, d]
            lib.or_hhs_fsi.argtypes = [i64, P, P, P, P, i64, d, d, d, d, ci, ci]
            lib.or_steps.argtypes = [i64, P, P, P, d, i64, d, d, d, ci, ci]
            lib.or_energy.argtypes = [i64, P, P, P, d, d, P]
            lib.or_get_counters.argtypes = [P]
            lib.or_get_counters.restype = None
            lib.or_reset_counters.argtypes = []
            lib.or_reset_counters.restype = None
            lib.or_num_threads.restype = ci
            lib.or_set_num_threads.argtypes = [ci]
            lib.or_set_num_threads.restype = None
            _lib = lib
    return _lib


def _f64(a, shape=None):
    a = np.ascontiguousarray(a, dtype=np.float64)
    if shape is not None:
        a = a.reshape(shape)
    return a


def _i32(a):
    return np.ascontiguousarray(a, dtype=np.int32)


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p) if a is not None else None


def _check(code, what):
    if code != OK:
        raise OracleError(code, what)


def num_threads() -> int:
    return _load().or_num_threads()


def set_num_threads(k: int) -> None:
    _load().or_set_num_threads(int(k))


def counters() -> dict:
    out = np.zeros(4, dtype=np.int64)
    _load().or_get_counters(_p(out))
    return {"acc": int(out[0]), "grad": int(out[1]), "tstep": int(out[2]),
            "max_depth": int(out[3])}


def reset_counters() -> None:
    _load().or_reset_counters()


def acc(m, x, A, B, G=1.0, eps2=0.0):
    """Newtonian accelerations of A due to B, [len(A), 3]."""
    m, x, A, B = _f64(m), _f64(x, (-1, 3)), _i32(A), _i32(B)
    out = np.zeros((A.size, 3))
    _check(_load().or_acc(_p(m), _p(x), _p(A), A.size, _p(B), B.size, G, eps2, _p(out)), "acc")
    return out


def grad(m, x, A, aA, B, aB, G=1.0, eps2=0.0):
    """Gradient accelerations g of A due to B given the accelerations aA, aB."""
    m, x, A, B = _f64(m), _f64(x, (-1, 3)), _i32(A), _i32(B)
    aA, aB = _f64(aA, (-1, 3)), _f64(aB, (-1, 3))
    out = np.zeros((A.size, 3))
    _check(_load().or_grad(_p(m), _p(x), _p(A), A.size, _p(aA), _p(B), B.size, _p(aB), G, eps2,
                           _p(out)), "grad")
    return out


def accel_gradient(m, x, A, B, eps_grad, G=1.0, eps2=0.0):
    """(a, a_tilde) for the active list A against the source list B (same set or disjoint)."""
    m, x, A, B = _f64(m), _f64(x, (-1, 3)), _i32(A), _i32(B)
    a = np.zeros((A.size, 3))
    at = np.zeros((A.size, 3))
    _check(_load().or_accel_gradient(m.size, _p(m), _p(x), _p(A), A.size, _p(B), B.size, G, eps2,
                                     eps_grad, _p(a), _p(at)), "accel_gradient")
    return a, at


def pair_timescales(xi, vi, mi, xj, vj, mj, G=1.0):
    """(t_ff, dt_ff/dt, t_fb, dt_fb/dt) of one pair."""
    xi, vi, xj, vj = _f64(xi), _f64(vi), _f64(xj), _f64(vj)
    out = np.zeros(4)
    _load().or_pair_timescales(_p(xi), _p(vi), float(mi), _p(xj), _p(vj), float(mj), G, _p(out))
    return tuple(out)


def pair_timescales_exact(xi, vi, ai, mi, xj, vj, aj, mj, G=1.0):
    """(t_ff, dt_ff/dt, t_fb, dt_fb/dt) of one pair with the exact fly-by derivative, given the
    accelerations a_i, a_j."""
    xi, vi, ai, xj, vj, aj = _f64(xi), _f64(vi), _f64(ai), _f64(xj), _f64(vj), _f64(aj)
    out = np.zeros(4)
    _load().or_pair_timescales_exact(_p(xi), _p(vi), _p(ai), float(mi), _p(xj), _p(vj), _p(aj), float(mj), G,
                                     _p(out))
    return tuple(out)


def sym_harmonic(d: float) -> float:
    return _load().or_sym_harmonic(float(d))


def sym_arithmetic(d: float) -> float:
    return _load().or_sym_arithmetic(float(d))


def timesteps(m, x, v, P, G=1.0, eta=0.2, sym=SYM_HARMONIC):
    """Symmetrised time-steps tau[len(P)] of the set P."""
    m, x, v, P = _f64(m), _f64(x, (-1, 3)), _f64(v, (-1, 3)), _i32(P)
    out = np.zeros(P.size)
    _check(_load().or_timesteps(_p(m), _p(x), _p(v), _p(P), P.size, G, eta, sym, _p(out)),
           "timesteps")
    return out


def timesteps_ex(m, x, v, A, P, G=1.0, eta=0.2, eps2=0.0, sym=SYM_HARMONIC):
    """Time-steps of the particles A over the set P; sym may carry FLYBY_EXACT (accelerations of
    the set due to itself, softened by eps2)."""
    m, x, v, A, P = _f64(m), _f64(x, (-1, 3)), _f64(v, (-1, 3)), _i32(A), _i32(P)
    out = np.zeros(A.size)
    _check(_load().or_timesteps_ex(_p(m), _p(x), _p(v), _p(A), A.size, _p(P), P.size, G, eta, eps2, int(sym),
                                   _p(out)), "timesteps_ex")
    return out


def timesteps_of(m, x, v, A, P, G=1.0, eta=0.2, sym=SYM_HARMONIC):
    """Symmetrised time-steps of the particles A (a sample of the set P) over the set P."""
    m, x, v, A, P = _f64(m), _f64(x, (-1, 3)), _f64(v, (-1, 3)), _i32(A), _i32(P)
    out = np.zeros(A.size)
    _check(_load().or_timesteps_of(_p(m), _p(x), _p(v), _p(A), A.size, _p(P), P.size, G, eta, sym,
                                   _p(out)), "timesteps_of")
    return out


def partition(P, tau, tau_pivot):
    """(S, F) index lists, in the order of P."""
    P, tau = _i32(P), _f64(tau)
    S = np.zeros(max(P.size, 1), dtype=np.int32)
    F = np.zeros(max(P.size, 1), dtype=np.int32)
    nS = ctypes.c_int64()
    nF = ctypes.c_int64()
    _load().or_partition(_p(P), P.size, _p(tau), float(tau_pivot), _p(S), ctypes.byref(nS),
                         _p(F), ctypes.byref(nF))
    return S[: nS.value].copy(), F[: nF.value].copy()


def kick(I, v, a, dt):
    I, a = _i32(I), _f64(a, (-1, 3))
    assert v.dtype == np.float64 and v.flags.c_contiguous
    _load().or_kick(_p(I), I.size, _p(v), _p(a), dt)


def drift(I, x, v, dt):
    I, v = _i32(I), _f64(v, (-1, 3))
    assert x.dtype == np.float64 and x.flags.c_contiguous
    _load().or_drift(_p(I), I.size, _p(x), _p(v), dt)


def fsi(m, x, v, S, dt, G=1.0, eps2=0.0):
    """One FSI step of the set S; returns updated copies (x, v)."""
    m = _f64(m)
    x = _f64(x, (-1, 3)).copy()
    v = _f64(v, (-1, 3)).copy()
    S = _i32(S)
    _check(_load().or_fsi(m.size, _p(m), _p(x), _p(v), _p(S), S.size, dt, G, eps2), "fsi")
    return x, v


def hhs_fsi(m, x, v, P, tau_pivot, G=1.0, eta=0.2, eps2=0.0, max_depth=40, sym=SYM_HARMONIC):
    """One hhs_fsi call on the set P; returns updated copies (x, v)."""
    m = _f64(m)
    x = _f64(x, (-1, 3)).copy()
    v = _f64(v, (-1, 3)).copy()
    P = _i32(P)
    _check(_load().or_hhs_fsi(m.size, _p(m), _p(x), _p(v), _p(P), P.size, tau_pivot, G, eta, eps2,
                              max_depth, sym), "hhs_fsi")
    return x, v


def steps_hold(m, x, v, dt, n_steps, G=1.0, eta=0.2, eps2=0.0, max_depth=40, sym=SYM_HARMONIC):
    """n_steps top-level steps of the second-order HOLD integrator (Eq. hhs2); returns (x, v)."""
    m = _f64(m)
    x = _f64(x, (-1, 3)).copy()
    v = _f64(v, (-1, 3)).copy()
    _check(_load().or_steps_hold(m.size, _p(m), _p(x), _p(v), dt, int(n_steps), G, eta, eps2, max_depth,
                                 int(sym)), "steps_hold")
    return x, v


def steps(m, x, v, dt, n_steps, G=1.0, eta=0.2, eps2=0.0, max_depth=40, sym=SYM_HARMONIC):
    """n_steps top-level hhs_fsi steps of size dt over all particles; returns (x, v)."""
    m = _f64(m)
    x = _f64(x, (-1, 3)).copy()
    v = _f64(v, (-1, 3)).copy()
    _check(_load().or_steps(m.size, _p(m), _p(x), _p(v), dt, int(n_steps), G, eta, eps2, max_depth,
                            sym), "steps")
    return x, v


def energy(m, x, v, G=1.0, eps2=0.0):
    """dict(T, U, E, P[3], L[3])."""
    m, x, v = _f64(m), _f64(x, (-1, 3)), _f64(v, (-1, 3))
    out = np.zeros(8)
    _check(_load().or_energy(m.size, _p(m), _p(x), _p(v), G, eps2, _p(out)), "energy")
    return {"T": out[0], "U": out[1], "E": out[0] + out[1], "P": out[2:5].copy(),
            "L": out[5:8].copy()}
