"""FP64 CPU oracle for TV-superiorized conjugate gradient (TEST INFRASTRUCTURE).

Only the test suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The CUDA library never calls it and it
never calls the CUDA library; they share only the seeded input generators.

The arithmetic lives in ``scg_oracle.c`` (plain C, FP64); this module compiles
it with gcc on first use (``build()``) and marshals numpy arrays through ctypes.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "scg_oracle.c")
_HDR = os.path.join(_HERE, "scg_oracle.h")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "liboracle.so")
_lock = threading.Lock()
_lib = None

# variant names follow the paper's algorithm names
VARIANTS = {"CG": 0, "PCG": 1, "S-CG": 2, "S-CG-CD": 3, "S-CG-K": 4, "S-PCG": 5, "S-PCG-K": 6}
PERTURB = {"none": 0, "gamma": 1, "eta": 2, "prox": 3}
STATUS = {0: "ok", 1: "max_iter", -1: "invalid", -4: "breakdown"}
TRACE_FIELDS = ("k", "f_test", "tv_before", "tv_after", "trials", "accepted", "ell",
                "gamma", "alpha", "beta", "margin", "f_after")


class Params(ctypes.Structure):
    _fields_ = [
        ("variant", ctypes.c_int),
        ("eps", ctypes.c_double),
        ("perturb", ctypes.c_int),
        ("gamma0", ctypes.c_double),
        ("gamma0_rel", ctypes.c_double),
        ("a", ctypes.c_double),
        ("max_trials", ctypes.c_int),
        ("eta0", ctypes.c_double),
        ("K", ctypes.c_int),
        ("k_inclusive", ctypes.c_int),
        ("mu", ctypes.c_double),
        ("filter_gain", ctypes.c_double),
        ("filter_identity", ctypes.c_int),
        ("max_iter", ctypes.c_int),
        ("prox_iters", ctypes.c_int),
        ("perturb_steps", ctypes.c_int),
    ]


_DP = ctypes.POINTER(ctypes.c_double)


class State(ctypes.Structure):
    _fields_ = [
        ("valid", ctypes.c_int),
        ("k", ctypes.c_int),
        ("ell", ctypes.c_longlong),
        ("gamma0", ctypes.c_double),
        ("gamma_fixed", ctypes.c_int),
        ("delta", ctypes.c_double),
        ("x", _DP),
        ("x_half", _DP),
        ("p", _DP),
        ("h", _DP),
        ("g", _DP),
    ]


STATE_VECTORS = ("x", "x_half", "p", "h", "g")


class Result(ctypes.Structure):
    _fields_ = [
        ("iters", ctypes.c_int),
        ("k_final", ctypes.c_int),
        ("status", ctypes.c_int),
        ("f_final", ctypes.c_double),
        ("tv_final", ctypes.c_double),
        ("ell", ctypes.c_longlong),
        ("gamma0_used", ctypes.c_double),
    ]


ITER_CB = ctypes.CFUNCTYPE(None, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p,
                           ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p)


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (OpenMP if available).  Returns the .so path."""
    with _lock:
        stale = (not os.path.exists(_LIB_PATH) or
                 os.path.getmtime(_LIB_PATH) < max(os.path.getmtime(_SRC), os.path.getmtime(_HDR)))
        if force or stale:
            os.makedirs(_OUT_DIR, exist_ok=True)
            tmp = _LIB_PATH + f".tmp{os.getpid()}"
            base = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
                    "-Wall", _SRC, "-o", tmp, "-lm"]
            try:
                subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True,
                               capture_output=True, text=True)
            except subprocess.CalledProcessError:
                subprocess.run(base, check=True, capture_output=True, text=True)
            os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    if _lib is None:
        path = build()
        L = ctypes.CDLL(path)
        dp = ctypes.POINTER(ctypes.c_double)
        ip = ctypes.POINTER(ctypes.c_int)
        i = ctypes.c_int
        d = ctypes.c_double
        L.orc_num_threads.restype = i
        L.orc_angle.argtypes = [i, i, dp, dp]
        L.orc_weight_trap.argtypes = [d, d, d]
        L.orc_weight_trap.restype = d
        L.orc_weight_clip.argtypes = [d, d, d, d, d]
        L.orc_weight_clip.restype = d
        for name in ("orc_project", "orc_backproject"):
            getattr(L, name).argtypes = [i, i, i, dp, dp]
        for name in ("orc_project_dense", "orc_backproject_dense"):
            getattr(L, name).argtypes = [i, i, i, i, dp, dp]
        L.orc_project_rays.argtypes = [i, i, i, dp, i, ip, ip, dp]
        L.orc_backproject_pixels.argtypes = [i, i, i, dp, i, ip, ip, dp]
        L.orc_tv.argtypes = [i, dp]
        L.orc_tv.restype = d
        L.orc_tv_grad.argtypes = [i, dp, dp]
        L.orc_tv_grad.restype = d
        L.orc_filter_length.argtypes = [i]
        L.orc_filter_length.restype = i
        L.orc_filter_factor.argtypes = [d, d]
        L.orc_filter_factor.restype = d
        L.orc_filter_rows.argtypes = [i, i, d, d, dp, dp]
        L.orc_fbp.argtypes = [i, i, i, dp, dp]
        L.orc_norm_A.argtypes = [i, i, i, i]
        L.orc_norm_A.restype = d
        L.orc_perturb_gamma.argtypes = [i, dp, d, d, i, ctypes.POINTER(ctypes.c_longlong), dp, dp, ip]
        L.orc_perturb_gamma.restype = i
        L.orc_perturb_prox.argtypes = [i, dp, d, d, i, ctypes.POINTER(ctypes.c_longlong), dp, dp]
        L.orc_perturb_prox.restype = i
        L.orc_tv_prox.argtypes = [i, dp, d, i, i, dp, dp, dp]
        L.orc_fista.argtypes = [i, i, i, dp, dp, d, d, d, i, i, i, dp, ctypes.POINTER(Result), dp, i]
        L.orc_fista.restype = i
        L.orc_solve.argtypes = [i, i, i, dp, dp, ctypes.POINTER(Params), dp,
                                ctypes.POINTER(Result), dp, i, ITER_CB, ctypes.c_void_p,
                                ctypes.POINTER(State), ctypes.POINTER(State)]
        L.orc_solve.restype = i
        _lib = L
    return _lib


def _dp(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _ip(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int))


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def num_threads() -> int:
    return int(lib().orc_num_threads())


def angle(a: int, n_angles: int):
    c, s = ctypes.c_double(), ctypes.c_double()
    lib().orc_angle(a, n_angles, ctypes.byref(c), ctypes.byref(s))
    return c.value, s.value


def weight_trap(d: float, c: float, s: float) -> float:
    return float(lib().orc_weight_trap(d, c, s))


def weight_clip(xc: float, yc: float, c: float, s: float, sb: float) -> float:
    return float(lib().orc_weight_clip(xc, yc, c, s, sb))


def project(x: np.ndarray, n_angles: int, n_bins: int) -> np.ndarray:
    x = _f64(x)
    n = x.shape[0]
    y = np.zeros((n_angles, n_bins))
    lib().orc_project(n, n_angles, n_bins, _dp(x), _dp(y))
    return y


def backproject(r: np.ndarray, n: int) -> np.ndarray:
    r = _f64(r)
    na, nb = r.shape
    x = np.zeros((n, n))
    lib().orc_backproject(n, na, nb, _dp(r), _dp(x))
    return x


def project_dense(x: np.ndarray, n_angles: int, n_bins: int, clip: bool = False) -> np.ndarray:
    x = _f64(x)
    y = np.zeros((n_angles, n_bins))
    lib().orc_project_dense(x.shape[0], n_angles, n_bins, int(clip), _dp(x), _dp(y))
    return y


def backproject_dense(r: np.ndarray, n: int, clip: bool = False) -> np.ndarray:
    r = _f64(r)
    x = np.zeros((n, n))
    lib().orc_backproject_dense(n, r.shape[0], r.shape[1], int(clip), _dp(r), _dp(x))
    return x


def project_rays(x: np.ndarray, n_angles: int, n_bins: int, a_idx, b_idx) -> np.ndarray:
    x = _f64(x)
    a_idx = np.ascontiguousarray(a_idx, dtype=np.int32)
    b_idx = np.ascontiguousarray(b_idx, dtype=np.int32)
    out = np.zeros(len(a_idx))
    lib().orc_project_rays(x.shape[0], n_angles, n_bins, _dp(x), len(a_idx),
                           _ip(a_idx), _ip(b_idx), _dp(out))
    return out


def backproject_pixels(r: np.ndarray, n: int, i_idx, j_idx) -> np.ndarray:
    r = _f64(r)
    i_idx = np.ascontiguousarray(i_idx, dtype=np.int32)
    j_idx = np.ascontiguousarray(j_idx, dtype=np.int32)
    out = np.zeros(len(i_idx))
    lib().orc_backproject_pixels(n, r.shape[0], r.shape[1], _dp(r), len(i_idx),
                                 _ip(i_idx), _ip(j_idx), _dp(out))
    return out


def tv(x: np.ndarray) -> float:
    x = _f64(x)
    return float(lib().orc_tv(x.shape[0], _dp(x)))


def tv_grad(x: np.ndarray):
    x = _f64(x)
    g = np.zeros_like(x)
    t = lib().orc_tv_grad(x.shape[0], _dp(x), _dp(g))
    return float(t), g


def filter_length(n_bins: int) -> int:
    return int(lib().orc_filter_length(n_bins))


def filter_factor(omega: float, mu: float) -> float:
    return float(lib().orc_filter_factor(omega, mu))


def filter_rows(r: np.ndarray, mu: float = 0.0, gain: float = 1.0) -> np.ndarray:
    r = _f64(r)
    out = np.zeros_like(r)
    lib().orc_filter_rows(r.shape[0], r.shape[1], mu, gain, _dp(r), _dp(out))
    return out


def fbp(y: np.ndarray, n: int) -> np.ndarray:
    """Filtered backprojection: A^T of the ramp-filtered (Hamming-windowed) rows,
    gain 1/(2 n_angles)."""
    y = _f64(y)
    na, nb = y.shape
    x = np.zeros((n, n))
    lib().orc_fbp(n, na, nb, _dp(y), _dp(x))
    return x


def norm_A(n: int, n_angles: int, n_bins: int, iters: int = 50) -> float:
    return float(lib().orc_norm_A(n, n_angles, n_bins, iters))


def perturb_gamma(x: np.ndarray, gamma0: float, a: float, max_trials: int, ell: int = 0):
    """One perturbation of the gamma rule from global index ``ell``: returns
    (x_half, ell after, accepted gamma or 0, trials, outcome) with outcome 1
    accepted, 0 every trial rejected (x kept), -1 zero subgradient."""
    x = _f64(x)
    n = x.shape[0]
    xh = np.zeros_like(x)
    e = ctypes.c_longlong(int(ell))
    g = ctypes.c_double(0.0)
    t = ctypes.c_int(0)
    rc = lib().orc_perturb_gamma(n, _dp(x), float(gamma0), float(a), int(max_trials), ctypes.byref(e),
                                 _dp(xh), ctypes.byref(g), ctypes.byref(t))
    return xh, int(e.value), float(g.value), int(t.value), int(rc)


def perturb_prox(x: np.ndarray, gamma0: float, a: float, prox_iters: int, ell: int = 0):
    """One perturbation of the prox rule from global index ``ell``: returns
    (x_half, ell after, lambda or 0, outcome) with outcome 1 perturbed, -1 zero
    subgradient (x kept)."""
    x = _f64(x)
    n = x.shape[0]
    xh = np.zeros_like(x)
    e = ctypes.c_longlong(int(ell))
    lam = np.zeros(1)
    rc = lib().orc_perturb_prox(n, _dp(x), float(gamma0), float(a), int(prox_iters), ctypes.byref(e),
                                _dp(xh), _dp(lam))
    return xh, int(e.value), float(lam[0]), int(rc)


def tv_prox(b: np.ndarray, alpha: float, iters: int, accel: bool = True, want_dual: bool = False):
    """prox of alpha TV at b by ``iters`` FGP steps (plain gradient projection
    with ``accel=False``); with ``want_dual`` also the dual field (p, q) on the
    (N-1)^2 interior terms."""
    b = _f64(b)
    n = b.shape[0]
    x = np.zeros_like(b)
    p = np.zeros((n - 1, n - 1))
    q = np.zeros((n - 1, n - 1))
    lib().orc_tv_prox(n, _dp(b), float(alpha), int(iters), int(bool(accel)), _dp(x), _dp(p), _dp(q))
    return (x, p, q) if want_dual else x


def fista(y: np.ndarray, n: int, eps: float, lam: float, c2: float, prox_iters: int = 20,
          accel: bool = True, max_iter: int = 100, x0=None):
    """FISTA (ISTA with ``accel=False``) with the TV prox; returns (x, result
    dict, trace [iters, 12]: k, -, -, TV(x_k), -, -, -, -, t_k, beta)."""
    y = _f64(y)
    na, nb = y.shape
    x = np.zeros((n, n))
    res = Result()
    rows = max(int(max_iter), 1)
    trace = np.zeros((rows, len(TRACE_FIELDS)))
    x0p = _dp(_f64(x0)) if x0 is not None else None
    keep = _f64(x0) if x0 is not None else None
    if keep is not None:
        x0p = _dp(keep)
    rc = lib().orc_fista(n, na, nb, _dp(y), x0p, float(eps), float(lam), float(c2), int(prox_iters),
                         int(bool(accel)), int(max_iter), _dp(x), ctypes.byref(res), _dp(trace), rows)
    out = dict(iters=res.iters, status=STATUS.get(res.status, res.status), f_final=res.f_final,
               tv_final=res.tv_final, rc=rc)
    return x, out, trace[: min(res.iters, rows)].copy()


def default_params(**kw) -> dict:
    p = dict(variant="S-CG", eps=1.0, perturb="gamma", gamma0=0.0, gamma0_rel=0.05,
             a=0.975, max_trials=32, eta0=0.0, K=2, k_inclusive=0, mu=0.0,
             filter_gain=1.0, filter_identity=0, max_iter=100, prox_iters=20, perturb_steps=1)
    p.update(kw)
    return p


def _state_in(st: dict, J: int, keep: list):
    S = State()
    S.valid = 1
    S.k = int(st["k"])
    S.ell = int(st["ell"])
    S.gamma0 = float(st["gamma0"])
    S.gamma_fixed = int(st["gamma_fixed"])
    S.delta = float(st.get("delta", 0.0))
    for name in STATE_VECTORS:
        v = st.get(name)
        if v is not None:
            a = _f64(np.asarray(v).reshape(J))
            keep.append(a)
            setattr(S, name, _dp(a))
    return S


def solve(y: np.ndarray, n: int, x0=None, callback=None, resume: dict | None = None,
          want_state: bool = False, **kw):
    """Run one solver.

    Returns (x, result dict, trace array [iters, 12]) and, with
    ``want_state``, the exit state as a dict (vectors as N x N arrays)."""
    p = default_params(**kw)
    y = _f64(y)
    na, nb = y.shape
    prm = Params(VARIANTS[p["variant"]], p["eps"], PERTURB[p["perturb"]], p["gamma0"],
                 p["gamma0_rel"], p["a"], p["max_trials"], p["eta0"], p["K"],
                 p["k_inclusive"], p["mu"], p["filter_gain"], p["filter_identity"],
                 p["max_iter"], p["prox_iters"], p["perturb_steps"])
    res = Result()
    x = np.zeros((n, n))
    rows = max(int(p["max_iter"]), 1)
    trace = np.zeros((rows, len(TRACE_FIELDS)))
    J = n * n
    if callback is not None:
        def _cb(it, xn, xh, pp, hh, gg, user):
            def arr(ptr):
                if not ptr:
                    return None
                return np.ctypeslib.as_array(ctypes.cast(ptr, _DP), shape=(J,)).reshape(n, n).copy()
            callback(it, arr(xn), arr(xh), arr(pp), arr(hh), arr(gg))
        cb = ITER_CB(_cb)
    else:
        cb = ITER_CB()
    x0p = None
    if x0 is not None:
        x0a = _f64(x0)
        x0p = _dp(x0a)
    keep: list = []
    rs = ctypes.byref(_state_in(resume, J, keep)) if resume is not None else None
    fs_arrays = {}
    fs = None
    if want_state:
        F = State()
        for name in STATE_VECTORS:
            fs_arrays[name] = np.zeros(J)
            setattr(F, name, _dp(fs_arrays[name]))
        fs = F
    st = lib().orc_solve(n, na, nb, _dp(y), x0p, ctypes.byref(prm), _dp(x), ctypes.byref(res),
                         _dp(trace), rows, cb, None, rs,
                         ctypes.byref(fs) if fs is not None else None)
    out = dict(iters=res.iters, k_final=res.k_final, status=STATUS.get(res.status, res.status),
               status_code=res.status, f_final=res.f_final, tv_final=res.tv_final,
               ell=res.ell, gamma0_used=res.gamma0_used, rc=st)
    tr = trace[: min(res.iters, rows)].copy()
    if not want_state:
        return x, out, tr
    state = dict(k=fs.k, ell=fs.ell, gamma0=fs.gamma0, gamma_fixed=fs.gamma_fixed, delta=fs.delta)
    for name in STATE_VECTORS:
        state[name] = fs_arrays[name].reshape(n, n)
    return x, out, tr, state
