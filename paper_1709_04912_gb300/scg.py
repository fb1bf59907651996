"""Thin ctypes binding of libscg (``include/scg.h``), with the same entry-point
names.  It only marshals arguments: tensors must already live on a CUDA
device, workspaces are allocated through PyTorch, and every step of the
method runs in the library's CUDA kernels.  There is no CPU fallback: if the
library cannot be loaded every call raises.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import torch

from . import build as _build

F64, F32, F16, BF16 = 0, 1, 2, 3
VARIANTS = {"CG": 0, "PCG": 1, "S-CG": 2, "S-CG-CD": 3, "S-CG-K": 4, "S-PCG": 5, "S-PCG-K": 6, "FISTA": 7}
PERTURB = {"none": 0, "gamma": 1, "eta": 2, "prox": 3}
STATUS = {0: "ok", 1: "max_iter", -1: "invalid", -2: "cuda", -3: "workspace", -4: "breakdown",
          -5: "unsupported"}
TRACE_FIELDS = ("k", "f_test", "tv_before", "tv_after", "trials", "accepted", "ell",
                "gamma", "alpha", "beta", "margin", "f_after")


class ScgError(RuntimeError):
    pass


class Geometry(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int), ("n_angles", ctypes.c_int), ("n_bins", ctypes.c_int)]


class Params(ctypes.Structure):
    _fields_ = [("perturb", ctypes.c_int), ("gamma0", ctypes.c_double),
                ("gamma0_rel", ctypes.c_double), ("a", ctypes.c_double),
                ("max_trials", ctypes.c_int), ("K", ctypes.c_int), ("k_inclusive", ctypes.c_int),
                ("mu", ctypes.c_double), ("filter_gain", ctypes.c_double),
                ("max_iter", ctypes.c_int), ("host_loop", ctypes.c_int), ("eta0", ctypes.c_double),
                ("lambda_", ctypes.c_double), ("prox_iters", ctypes.c_int), ("lipschitz", ctypes.c_double),
                ("proj_shape", ctypes.c_int), ("perturb_steps", ctypes.c_int)]


class Result(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int), ("k_final", ctypes.c_int), ("status", ctypes.c_int),
                ("f_final", ctypes.c_double), ("tv_final", ctypes.c_double),
                ("ell", ctypes.c_longlong), ("gamma0_used", ctypes.c_double),
                ("kernel_launches", ctypes.c_int), ("body_launches", ctypes.c_int),
                ("device_loop", ctypes.c_int), ("lipschitz_used", ctypes.c_double)]


class Problem(ctypes.Structure):
    _fields_ = [("geometry", Geometry), ("eps", ctypes.c_double), ("y", ctypes.c_void_p),
                ("x0", ctypes.c_void_p), ("x_out", ctypes.c_void_p)]


class ServerConfig(ctypes.Structure):
    _fields_ = [("variant", ctypes.c_int), ("precision", ctypes.c_int), ("params", Params),
                ("pool", ctypes.c_void_p), ("pool_bytes", ctypes.c_size_t),
                ("max_active", ctypes.c_int), ("bodies_per_step", ctypes.c_int)]


class Completion(ctypes.Structure):
    _fields_ = [("tag", ctypes.c_ulonglong), ("result", Result)]


class State(ctypes.Structure):
    _fields_ = [("valid", ctypes.c_int), ("k", ctypes.c_int), ("ell", ctypes.c_longlong),
                ("gamma0", ctypes.c_double), ("gamma_fixed", ctypes.c_int),
                ("delta", ctypes.c_double), ("x", ctypes.c_void_p), ("x_half", ctypes.c_void_p),
                ("p", ctypes.c_void_p), ("h", ctypes.c_void_p), ("g", ctypes.c_void_p)]


STATE_VECTORS = ("x", "x_half", "p", "h", "g")
_lib = None


def library_path() -> str:
    return _build.LIB


def load(build_if_needed: bool = True):
    """Load libscg.so (building it first when sources are newer)."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.build() if build_if_needed else _build.LIB
    if not os.path.exists(path):
        raise ScgError(f"libscg not built: {path}")
    L = ctypes.CDLL(path)
    vp, sz, i, d = ctypes.c_void_p, ctypes.c_size_t, ctypes.c_int, ctypes.c_double
    gp = ctypes.POINTER(Geometry)
    L.scg_strerror.restype = ctypes.c_char_p
    L.scg_strerror.argtypes = [i]
    L.scg_default_params.argtypes = [ctypes.POINTER(Params)]
    L.scg_op_workspace_bytes.restype = sz
    L.scg_op_workspace_bytes.argtypes = [gp, i]
    L.scg_solve_workspace_bytes.restype = sz
    L.scg_solve_workspace_bytes.argtypes = [gp, i, i]
    L.scg_solve_workspace_bytes_p.restype = sz
    L.scg_solve_workspace_bytes_p.argtypes = [gp, i, i, ctypes.POINTER(Params)]
    L.scg_project.argtypes = [gp, i, vp, vp, vp, sz, vp]
    L.scg_backproject.argtypes = [gp, i, vp, vp, vp, sz, vp]
    L.scg_tv.argtypes = [i, i, vp, vp, vp, sz, vp]
    L.scg_tv_grad.argtypes = [i, i, vp, vp, vp, vp, sz, vp]
    L.scg_filter.argtypes = [gp, i, d, d, vp, vp, vp, sz, vp]
    L.scg_fbp.argtypes = [gp, i, vp, vp, vp, sz, vp]
    L.scg_solve.argtypes = [gp, i, i, ctypes.POINTER(Params), d, vp, vp, vp, vp, sz,
                            ctypes.POINTER(Result), ctypes.POINTER(ctypes.c_double), i,
                            ctypes.POINTER(State), ctypes.POINTER(State), vp]
    L.scg_solve_async.argtypes = [gp, i, i, ctypes.POINTER(Params), d, vp, vp, vp, vp, sz, vp,
                                  ctypes.POINTER(State), vp]
    L.scg_solve_async.restype = i
    pp = ctypes.POINTER(Problem)
    L.scg_batch_workspace_bytes.restype = sz
    L.scg_batch_workspace_bytes.argtypes = [pp, i, i, i]
    L.scg_solve_batch.argtypes = [pp, i, i, i, ctypes.POINTER(Params), vp, sz, ctypes.POINTER(Result), vp]
    L.scg_release.argtypes = []
    L.scg_release.restype = i
    L.scg_test_stall_copies.argtypes = [i]
    L.scg_test_stall_copies.restype = i
    L.scg_operator_create.argtypes = [gp, i, vp, sz, vp, ctypes.POINTER(vp)]
    L.scg_operator_create_angles.argtypes = [gp, i, i, i, vp, sz, vp, ctypes.POINTER(vp)]
    L.scg_operator_create_angles.restype = i
    L.scg_operator_project.argtypes = [vp, vp, vp, vp]
    L.scg_operator_backproject.argtypes = [vp, vp, vp, vp]
    L.scg_operator_destroy.argtypes = [vp]
    L.scg_operator_kernel_ms.argtypes = [vp, ctypes.POINTER(ctypes.c_float), ctypes.POINTER(ctypes.c_float)]
    L.scg_operator_kernel_ms.restype = i
    L.scg_operator_timing.argtypes = [vp, i]
    L.scg_operator_timing.restype = i
    for name in ("scg_operator_create", "scg_operator_project", "scg_operator_backproject",
                 "scg_operator_destroy"):
        getattr(L, name).restype = i
    L.scg_server_footprint.restype = sz
    L.scg_server_footprint.argtypes = [gp, i, i]
    L.scg_server_create.argtypes = [ctypes.POINTER(ServerConfig), ctypes.POINTER(vp)]
    L.scg_server_submit.argtypes = [vp, pp, ctypes.c_ulonglong]
    L.scg_server_step.argtypes = [vp, vp, ctypes.POINTER(Completion), i, ctypes.POINTER(i)]
    L.scg_server_pending.argtypes = [vp, ctypes.POINTER(i), ctypes.POINTER(i)]
    L.scg_server_destroy.argtypes = [vp]
    for name in ("scg_project", "scg_backproject", "scg_tv", "scg_tv_grad", "scg_filter", "scg_fbp", "scg_solve",
                 "scg_solve_batch", "scg_server_create", "scg_server_submit", "scg_server_step",
                 "scg_server_pending", "scg_server_destroy"):
        getattr(L, name).restype = i
    _lib = L
    return L


def _check(rc: int, what: str, ok=(0,)):
    if rc not in ok:
        msg = load().scg_strerror(rc).decode()
        raise ScgError(f"{what} failed: {rc} ({msg})")


def _prec_of(dtype) -> int:
    p = {torch.float64: F64, torch.float32: F32, torch.float16: F16, torch.bfloat16: BF16}.get(dtype)
    if p is None:
        raise ScgError(f"unsupported dtype {dtype}")
    return p


def _prec(t: torch.Tensor) -> int:
    return _prec_of(t.dtype)


def _dev_ptr(t: torch.Tensor, name: str) -> int:
    if not t.is_cuda:
        raise ScgError(f"{name} must be a CUDA tensor")
    if not t.is_contiguous():
        raise ScgError(f"{name} must be contiguous")
    return t.data_ptr()


def _stream(device) -> int:
    return torch.cuda.current_stream(device).cuda_stream


_workspaces: dict = {}


def workspace(nbytes: int, device, tag: str) -> torch.Tensor:
    """Cached device workspace (one per tag and device)."""
    key = (tag, str(device))
    w = _workspaces.get(key)
    if w is None or w.numel() < nbytes:
        w = torch.empty(max(nbytes, 256), dtype=torch.uint8, device=device)
        _workspaces[key] = w
    return w


def geometry(n: int, n_angles: int, n_bins: int) -> Geometry:
    return Geometry(int(n), int(n_angles), int(n_bins))


def op_workspace_bytes(n: int, n_angles: int, n_bins: int, precision: int) -> int:
    g = geometry(n, n_angles, n_bins)
    return int(load().scg_op_workspace_bytes(ctypes.byref(g), precision))


def solve_workspace_bytes(n: int, n_angles: int, n_bins: int, variant: str, precision: int, **params) -> int:
    """Workspace bytes of scg_solve for this geometry, variant, precision and
    parameters (scg_solve_workspace_bytes_p; the proximal perturbation needs
    more than the defaults)."""
    g = geometry(n, n_angles, n_bins)
    p = _params(default_params(**params))
    return int(load().scg_solve_workspace_bytes_p(ctypes.byref(g), VARIANTS[variant], precision, ctypes.byref(p)))


def scg_project(x: torch.Tensor, n_angles: int, n_bins: int, out: torch.Tensor | None = None):
    """y = A x on the device (x: N x N)."""
    n = x.shape[-1]
    prec = _prec(x)
    if out is None:
        out = torch.empty((n_angles, n_bins), dtype=x.dtype, device=x.device)
    g = geometry(n, n_angles, n_bins)
    nb = load().scg_op_workspace_bytes(ctypes.byref(g), prec)
    w = workspace(nb, x.device, "op")
    rc = load().scg_project(ctypes.byref(g), prec, _dev_ptr(x, "x"), _dev_ptr(out, "y"),
                            w.data_ptr(), w.numel(), _stream(x.device))
    _check(rc, "scg_project")
    return out


def scg_backproject(r: torch.Tensor, n: int, out: torch.Tensor | None = None):
    """x = A^T r on the device (r: n_angles x n_bins)."""
    na, nbins = r.shape
    prec = _prec(r)
    if out is None:
        out = torch.empty((n, n), dtype=r.dtype, device=r.device)
    g = geometry(n, na, nbins)
    nb = load().scg_op_workspace_bytes(ctypes.byref(g), prec)
    w = workspace(nb, r.device, "op")
    rc = load().scg_backproject(ctypes.byref(g), prec, _dev_ptr(r, "r"), _dev_ptr(out, "x"),
                                w.data_ptr(), w.numel(), _stream(r.device))
    _check(rc, "scg_backproject")
    return out


def scg_tv(x: torch.Tensor) -> torch.Tensor:
    """TV(x) as a 0-d float64 device tensor."""
    n = x.shape[-1]
    prec = _prec(x)
    out = torch.zeros((), dtype=torch.float64, device=x.device)
    g = geometry(n, 1, 1)
    nb = load().scg_op_workspace_bytes(ctypes.byref(g), prec)
    w = workspace(nb, x.device, "op")
    rc = load().scg_tv(n, prec, _dev_ptr(x, "x"), out.data_ptr(), w.data_ptr(), w.numel(),
                       _stream(x.device))
    _check(rc, "scg_tv")
    return out


def scg_tv_grad(x: torch.Tensor):
    """(subgradient of TV at x, TV(x) as a 0-d float64 device tensor)."""
    n = x.shape[-1]
    prec = _prec(x)
    out = torch.zeros((), dtype=torch.float64, device=x.device)
    grad = torch.empty_like(x)
    g = geometry(n, 1, 1)
    nb = load().scg_op_workspace_bytes(ctypes.byref(g), prec)
    w = workspace(nb, x.device, "op")
    rc = load().scg_tv_grad(n, prec, _dev_ptr(x, "x"), grad.data_ptr(), out.data_ptr(),
                            w.data_ptr(), w.numel(), _stream(x.device))
    _check(rc, "scg_tv_grad")
    return grad, out


def scg_filter(r: torch.Tensor, mu: float = 0.0, gain: float = 1.0) -> torch.Tensor:
    """Row filter F^T C F r of the preconditioner."""
    na, nbins = r.shape
    prec = _prec(r)
    out = torch.empty_like(r)
    g = geometry(2, na, nbins)
    nb = load().scg_op_workspace_bytes(ctypes.byref(g), prec)
    w = workspace(nb, r.device, "op")
    rc = load().scg_filter(ctypes.byref(g), prec, float(mu), float(gain), _dev_ptr(r, "r"),
                           out.data_ptr(), w.data_ptr(), w.numel(), _stream(r.device))
    _check(rc, "scg_filter")
    return out


def scg_fbp(y: torch.Tensor, n: int, out: torch.Tensor | None = None) -> torch.Tensor:
    """Filtered backprojection of the n_angles x n_bins sinogram ``y`` (N x N image)."""
    na, nbins = y.shape
    prec = _prec(y)
    if out is None:
        out = torch.empty((n, n), dtype=y.dtype, device=y.device)
    g = geometry(n, na, nbins)
    nb = load().scg_op_workspace_bytes(ctypes.byref(g), prec)
    w = workspace(nb, y.device, "op")
    rc = load().scg_fbp(ctypes.byref(g), prec, _dev_ptr(y, "y"), _dev_ptr(out, "x"), w.data_ptr(), w.numel(),
                        _stream(y.device))
    _check(rc, "scg_fbp")
    return out


def default_params(**kw) -> dict:
    p = Params()
    load().scg_default_params(ctypes.byref(p))
    d = {name: getattr(p, name) for name, _ in Params._fields_}
    d["perturb"] = {v: k for k, v in PERTURB.items()}[d["perturb"]]
    d.update(kw)
    return d


def _params(d: dict) -> Params:
    return Params(PERTURB[d["perturb"]], float(d["gamma0"]), float(d["gamma0_rel"]), float(d["a"]),
                  int(d["max_trials"]), int(d["K"]), int(d["k_inclusive"]), float(d["mu"]),
                  float(d["filter_gain"]), int(d["max_iter"]), int(d["host_loop"]), float(d["eta0"]),
                  float(d["lambda_"]), int(d["prox_iters"]), float(d["lipschitz"]), int(d["proj_shape"]),
                  int(d["perturb_steps"]))


@dataclass
class SolveResult:
    x: torch.Tensor
    iters: int
    k_final: int
    status: str
    status_code: int
    f_final: float
    tv_final: float
    ell: int
    gamma0_used: float
    kernel_launches: int = 0
    body_launches: int = 0
    device_loop: int = 0
    lipschitz_used: float = 0.0
    trace: object = None
    state: dict | None = None


def scg_solve(y: torch.Tensor, n: int, variant: str = "S-CG", eps: float = 1.0, x0=None,
              trace: bool = False, resume: dict | None = None, want_state: bool = False,
              out: torch.Tensor | None = None, work: torch.Tensor | None = None, **params):
    """Run one solver on the device.  ``y`` is the n_angles x n_bins sinogram.

    ``resume``/``want_state`` carry the state dict of ``include/scg.h``'s
    scg_state (vectors as N x N device tensors)."""
    import numpy as np

    L = load()
    na, nbins = y.shape
    prec = _prec(y)
    g = geometry(n, na, nbins)
    p = _params(default_params(**params))
    nbytes = L.scg_solve_workspace_bytes_p(ctypes.byref(g), VARIANTS[variant], prec, ctypes.byref(p))
    if work is None:
        work = workspace(nbytes, y.device, "solve")
    if out is None:
        out = torch.empty((n, n), dtype=y.dtype, device=y.device)
    x0p = None
    if x0 is not None:
        x0 = x0.to(dtype=y.dtype).contiguous()
        x0p = _dev_ptr(x0, "x0")
    res = Result()
    rows = max(int(p.max_iter), 1)
    tr = np.zeros((rows, len(TRACE_FIELDS))) if trace else None
    trp = tr.ctypes.data_as(ctypes.POINTER(ctypes.c_double)) if trace else None
    keep = []
    rs = None
    if resume is not None:
        R = State()
        R.valid = 1
        R.k = int(resume["k"])
        R.ell = int(resume["ell"])
        R.gamma0 = float(resume["gamma0"])
        R.gamma_fixed = int(resume["gamma_fixed"])
        R.delta = float(resume.get("delta", 0.0))
        for name in STATE_VECTORS:
            v = resume.get(name)
            if v is not None:
                v = v.to(device=y.device, dtype=y.dtype).contiguous()
                keep.append(v)
                setattr(R, name, v.data_ptr())
        rs = ctypes.byref(R)
    fs = None
    fs_t = {}
    if want_state:
        F = State()
        for name in STATE_VECTORS:
            fs_t[name] = torch.zeros((n, n), dtype=y.dtype, device=y.device)
            setattr(F, name, fs_t[name].data_ptr())
        fs = F
    rc = L.scg_solve(ctypes.byref(g), VARIANTS[variant], prec, ctypes.byref(p), float(eps),
                     _dev_ptr(y, "y"), x0p, _dev_ptr(out, "x_out"), work.data_ptr(), work.numel(),
                     ctypes.byref(res), trp, rows if trace else 0, rs,
                     ctypes.byref(fs) if fs is not None else None, _stream(y.device))
    _check(rc, "scg_solve", ok=(0, 1, -4))
    out_res = SolveResult(out, res.iters, res.k_final, STATUS.get(res.status, str(res.status)),
                          res.status, res.f_final, res.tv_final, res.ell, res.gamma0_used,
                          res.kernel_launches, res.body_launches, res.device_loop, res.lipschitz_used)
    if trace:
        out_res.trace = tr[: min(res.iters, rows)].copy()
    if want_state:
        st = dict(k=fs.k, ell=fs.ell, gamma0=fs.gamma0, gamma_fixed=fs.gamma_fixed, delta=fs.delta)
        st.update(fs_t)
        out_res.state = st
    return out_res


class AsyncSolve:
    """A solve enqueued by scg_solve_async: ``x`` is ordered before later work
    on the stream; :meth:`result` waits for the stream and reads the result the
    device wrote into pinned host memory."""

    def __init__(self, x, res_buf, stream):
        self.x, self._buf, self._stream = x, res_buf, stream

    def result(self) -> SolveResult:
        self._stream.synchronize()
        r = Result.from_address(self._buf.data_ptr())
        return SolveResult(self.x, r.iters, r.k_final, STATUS.get(r.status, str(r.status)), r.status,
                           r.f_final, r.tv_final, r.ell, r.gamma0_used, r.kernel_launches, r.body_launches,
                           r.device_loop, r.lipschitz_used)


def scg_solve_async(y: torch.Tensor, n: int, variant: str = "S-CG", eps: float = 1.0, x0=None,
                    out: torch.Tensor | None = None, work: torch.Tensor | None = None, **params) -> AsyncSolve:
    """Enqueue one solve on the current stream (scg_solve_async) and return at once."""
    L = load()
    na, nbins = y.shape
    prec = _prec(y)
    g = geometry(n, na, nbins)
    p = _params(default_params(**params))
    nbytes = L.scg_solve_workspace_bytes_p(ctypes.byref(g), VARIANTS[variant], prec, ctypes.byref(p))
    if work is None:
        work = workspace(nbytes, y.device, "solve")
    if out is None:
        out = torch.empty((n, n), dtype=y.dtype, device=y.device)
    x0p = None
    if x0 is not None:
        x0 = x0.to(dtype=y.dtype).contiguous()
        x0p = _dev_ptr(x0, "x0")
    buf = torch.zeros(ctypes.sizeof(Result), dtype=torch.uint8).pin_memory()
    stream = torch.cuda.current_stream(y.device)
    rc = L.scg_solve_async(ctypes.byref(g), VARIANTS[variant], prec, ctypes.byref(p), float(eps),
                           _dev_ptr(y, "y"), x0p, _dev_ptr(out, "x_out"), work.data_ptr(), work.numel(),
                           buf.data_ptr(), None, stream.cuda_stream)
    _check(rc, "scg_solve_async")
    return AsyncSolve(out, buf, stream)


def _problems(ys, ns, eps, x0s, outs):
    arr = (Problem * len(ys))()
    for q, (y, n, e, x0, out) in enumerate(zip(ys, ns, eps, x0s, outs)):
        na, nbins = y.shape
        arr[q].geometry = geometry(n, na, nbins)
        arr[q].eps = float(e)
        arr[q].y = _dev_ptr(y, "y")
        arr[q].x0 = _dev_ptr(x0, "x0") if x0 is not None else None
        arr[q].x_out = _dev_ptr(out, "x_out")
    return arr


def batch_workspace_bytes(shapes, variant: str = "S-CG", dtype=torch.float32) -> int:
    """Workspace bytes of scg_solve_batch for problems of shapes (n, n_angles, n_bins)."""
    arr = (Problem * len(shapes))()
    for q, (n, na, nbins) in enumerate(shapes):
        arr[q].geometry = geometry(n, na, nbins)
    prec = _prec_of(dtype)
    return int(load().scg_batch_workspace_bytes(arr, len(shapes), VARIANTS[variant], prec))


def scg_solve_batch(ys, ns, variant: str = "S-CG", eps=1.0, x0s=None, outs=None,
                    work: torch.Tensor | None = None, **params):
    """Solve independent problems together (scg_solve_batch).  ``ys``: list of
    n_angles x n_bins device sinograms of one dtype; ``ns``: image sides;
    ``eps``: one threshold or one per problem.  Returns one SolveResult each."""
    L = load()
    count = len(ys)
    if count == 0:
        return []
    dev, dt = ys[0].device, ys[0].dtype
    prec = _prec(ys[0])
    if any(y.dtype != dt or y.device != dev for y in ys):
        raise ScgError("all sinograms must share one dtype and device")
    eps = list(eps) if isinstance(eps, (list, tuple)) else [eps] * count
    x0s = [None] * count if x0s is None else [None if x is None else x.to(dtype=dt).contiguous()
                                              for x in x0s]
    if outs is None:
        outs = [torch.empty((n, n), dtype=dt, device=dev) for n in ns]
    arr = _problems(ys, ns, eps, x0s, outs)
    nbytes = L.scg_batch_workspace_bytes(arr, count, VARIANTS[variant], prec)
    if nbytes == 0:
        raise ScgError("scg_batch_workspace_bytes rejected the problems")
    if work is None or work.numel() < nbytes:
        work = workspace(nbytes, dev, "batch")
    p = _params(default_params(**params))
    res = (Result * count)()
    rc = L.scg_solve_batch(arr, count, VARIANTS[variant], prec, ctypes.byref(p), work.data_ptr(),
                           work.numel(), res, _stream(dev))
    _check(rc, "scg_solve_batch", ok=(0, 1, -4))
    return [SolveResult(outs[q], r.iters, r.k_final, STATUS.get(r.status, str(r.status)), r.status,
                        r.f_final, r.tv_final, r.ell, r.gamma0_used, r.kernel_launches,
                        r.body_launches, r.device_loop) for q, r in enumerate(res)]


def server_footprint(n: int, n_angles: int, n_bins: int, variant: str = "S-CG",
                     dtype=torch.float32) -> int:
    """Pool bytes one resident request of this geometry holds (scg_server_footprint)."""
    g = geometry(n, n_angles, n_bins)
    prec = _prec_of(dtype)
    return int(load().scg_server_footprint(ctypes.byref(g), VARIANTS[variant], prec))


def _result(r: Result, x) -> SolveResult:
    return SolveResult(x, r.iters, r.k_final, STATUS.get(r.status, str(r.status)), r.status, r.f_final,
                       r.tv_final, r.ell, r.gamma0_used, r.kernel_launches, r.body_launches,
                       r.device_loop)


class Server:
    """Continuous-batching request server (scg_server_*).  The pool is one
    device tensor of ``pool_bytes``; submitted tensors are kept alive until
    their completion is returned by :meth:`step`."""

    def __init__(self, variant: str = "S-CG", dtype=torch.float32, pool_bytes: int = 1 << 30,
                 max_active: int = 64, bodies_per_step: int = 1, device="cuda:0", **params):
        L = load()
        self.variant, self.dtype, self.device = variant, dtype, torch.device(device)
        self.pool = torch.empty(int(pool_bytes), dtype=torch.uint8, device=self.device)
        cfg = ServerConfig(VARIANTS[variant], _prec_of(dtype),
                           _params(default_params(**params)), self.pool.data_ptr(), self.pool.numel(),
                           int(max_active), int(bodies_per_step))
        h = ctypes.c_void_p()
        _check(L.scg_server_create(ctypes.byref(cfg), ctypes.byref(h)), "scg_server_create")
        self._h = h
        self._live = {}
        self._next = 0
        self._buf = (Completion * int(max_active))()   # a step finishes at most max_active

    def submit(self, y: torch.Tensor, n: int, eps: float, x0=None, out=None, tag=None) -> int:
        if y.dtype != self.dtype:
            raise ScgError("sinogram dtype differs from the server's")
        if x0 is not None:
            x0 = x0.to(dtype=self.dtype).contiguous()
        if out is None:
            out = torch.empty((n, n), dtype=self.dtype, device=y.device)
        if tag is None:
            tag = self._next
        self._next = max(self._next, int(tag)) + 1
        arr = _problems([y], [n], [eps], [x0], [out])
        _check(load().scg_server_submit(self._h, arr, int(tag)), "scg_server_submit")
        self._live[int(tag)] = (y, x0, out)
        return int(tag)

    def step(self) -> list:
        """Advance the server one step; returns [(tag, SolveResult)] of the
        requests that finished."""
        nd = ctypes.c_int(0)
        rc = load().scg_server_step(self._h, _stream(self.device), self._buf, len(self._buf), ctypes.byref(nd))
        _check(rc, "scg_server_step")
        got = []
        for q in range(nd.value):
            c = self._buf[q]
            _, _, out = self._live.pop(int(c.tag))
            got.append((int(c.tag), _result(c.result, out)))
        return got

    def pending(self):
        q, a = ctypes.c_int(0), ctypes.c_int(0)
        _check(load().scg_server_pending(self._h, ctypes.byref(q), ctypes.byref(a)), "scg_server_pending")
        return q.value, a.value

    def close(self):
        if self._h:
            load().scg_server_destroy(self._h)
            self._h = None
            self._live.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Operator:
    """Prepared A / A^T pair for one geometry and precision (scg_operator_*):
    each application is device work only, so it is asynchronous and can be
    captured in a CUDA graph."""

    def __init__(self, n: int, n_angles: int, n_bins: int, dtype=torch.float32, device="cuda:0",
                 angles: tuple | None = None, timing: bool = False):
        """``angles=(a_begin, a_count)``: the operator of that block of the
        scan's angles (scg_operator_create_angles); sinograms are then
        a_count x n_bins.  ``timing``: record the kernels' own device times
        for kernel_ms() (scg_operator_timing; costs a few microseconds per
        application)."""
        L = load()
        a0, na_loc = (0, int(n_angles)) if angles is None else (int(angles[0]), int(angles[1]))
        self.n, self.na, self.nb = int(n), na_loc, int(n_bins)
        self.dtype, self.device = dtype, torch.device(device)
        prec = _prec_of(dtype)
        g = geometry(n, n_angles, n_bins)
        gl = geometry(n, na_loc, n_bins)
        nbytes = L.scg_op_workspace_bytes(ctypes.byref(gl), prec)
        self.work = torch.empty(max(int(nbytes), 256), dtype=torch.uint8, device=self.device)
        h = ctypes.c_void_p()
        _check(L.scg_operator_create_angles(ctypes.byref(g), a0, na_loc, prec, self.work.data_ptr(),
                                            self.work.numel(), _stream(self.device), ctypes.byref(h)),
               "scg_operator_create_angles")
        self._h = h
        if timing:
            self.set_timing(True)

    def set_timing(self, enable: bool):
        _check(load().scg_operator_timing(self._h, int(bool(enable))), "scg_operator_timing")

    def project(self, x: torch.Tensor, out: torch.Tensor | None = None) -> torch.Tensor:
        if out is None:
            out = torch.empty((self.na, self.nb), dtype=self.dtype, device=self.device)
        _check(load().scg_operator_project(self._h, _dev_ptr(x, "x"), _dev_ptr(out, "y"),
                                           _stream(self.device)), "scg_operator_project")
        return out

    def backproject(self, r: torch.Tensor, out: torch.Tensor | None = None) -> torch.Tensor:
        if out is None:
            out = torch.empty((self.n, self.n), dtype=self.dtype, device=self.device)
        _check(load().scg_operator_backproject(self._h, _dev_ptr(r, "r"), _dev_ptr(out, "x"),
                                               _stream(self.device)), "scg_operator_backproject")
        return out

    def kernel_ms(self):
        """(projector, gather) kernel device times of the last timed project /
        backproject calls (scg_operator_kernel_ms); None for a kernel not yet
        timed."""
        out = []
        for which in (0, 1):
            f = ctypes.c_float(0.0)
            args = (ctypes.byref(f), None) if which == 0 else (None, ctypes.byref(f))
            rc = load().scg_operator_kernel_ms(self._h, *args)
            out.append(float(f.value) if rc == 0 else None)
        return tuple(out)

    def close(self):
        if self._h:
            load().scg_operator_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def set_copy_stall(stall: bool) -> None:
    """Test hook (scg_test_stall_copies): while set, the gathers of problems set
    up afterwards wait for bytes that never arrive, so their bounded waits run
    out and solves report SCG_ERR_CUDA."""
    _check(load().scg_test_stall_copies(int(bool(stall))), "scg_test_stall_copies")


def release() -> None:
    """Free the library's cached graphs, side streams and pinned flags (scg_release)."""
    _check(load().scg_release(), "scg_release")
