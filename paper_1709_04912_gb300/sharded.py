"""Angle-sharded S-CG: one reconstruction spread over several GPUs.

Rank r of W holds a block of consecutive projection angles (``angle_blocks``),
its rows y_r of the data and the local operator pair A_r, A_r^T of that block
(the library's ``scg_operator_create_angles`` on its own GPU).  The loop is
S-CG (Algorithm 7 with CG-PR-STEP, Algorithm 8), with the sums over angle
blocks taken by all-reduces:

* f(x) = sum_r 1/2 ||A_r x - y_r||^2 -- one scalar all-reduce per body, from
  the residual the gradient also uses;
* g' = sum_r A_r^T (A_r x_{k+1/2} - y_r) -- one all-reduce of J values;
* h' = sum_r A_r^T A_r p' -- one all-reduce of J values.

Every image-space step (TV and its subgradient, the gamma trials, beta, alpha,
the vector updates) is replicated: each rank computes it from the same
all-reduced inputs, so all ranks hold the same iterate with no further
exchange.  A residual sinogram never leaves its rank.

The driver is written against a small array interface (numpy arrays on the
host, torch tensors on a device) and takes the local operators, TV, its
subgradient and the all-reduce as callables; ``device_operators`` builds them
from the library for one GPU.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import Callable


def angle_blocks(n_angles: int, world: int) -> list[tuple[int, int]]:
    """Contiguous angle blocks (a_begin, a_count) of one scan over ``world``
    ranks; block sizes differ by at most one.  A rank may get no angles only
    when there are more ranks than angles."""
    base, extra = divmod(int(n_angles), int(world))
    out, a0 = [], 0
    for r in range(world):
        cnt = base + (1 if r < extra else 0)
        out.append((a0, cnt))
        a0 += cnt
    return out


def _dot(u, v) -> float:
    return float((u * v).sum())


@dataclass
class ShardedResult:
    x: object
    iters: int
    k_final: int
    status: str
    f_final: float
    tv_final: float
    ell: int
    gamma0_used: float
    trace: list = field(default_factory=list)      # per body: (k, f tested, trials, accepted, l, gamma)
    exchanges: int = 0                             # all-reduces issued


class ShardedSCG:
    """S-CG over angle blocks.

    project_local(x) -> this rank's rows of A x;
    backproject_local(r) -> this rank's share A_r^T r;
    tv(x) -> TV(x); tv_grad(x) -> (subgradient, TV(x));
    allreduce(a) -> the elementwise sum of ``a`` over ranks (a float or an
    image array); for one rank the identity."""

    def __init__(self, project_local: Callable, backproject_local: Callable, tv: Callable, tv_grad: Callable,
                 allreduce: Callable):
        self.A = project_local
        self.AT = backproject_local
        self.tv = tv
        self.tv_grad = tv_grad
        self._allreduce = allreduce
        self.exchanges = 0

    def _sum(self, a):
        self.exchanges += 1
        return self._allreduce(a)

    def _gradient(self, x, y_local):
        """(f(x), A^T (A x - y)) with one scalar and one image exchange."""
        r = self.A(x) - y_local
        f = 0.5 * self._sum(_dot(r, r))
        return f, self._sum(self.AT(r))

    def _AtA(self, p):
        return self._sum(self.AT(self.A(p)))

    def solve(self, y_local, x0, eps: float, gamma0: float = 0.0, gamma0_rel: float = 0.05, a: float = 0.975,
              max_trials: int = 32, max_iter: int = 100, perturb: bool = True) -> ShardedResult:
        """Algorithm 7 from x0 (an image of the array type to work in) to the
        first f(x_{k-1/2}) <= eps; the gamma rule of Sec. 3 as the library
        reads it (one global l, gamma_0 a^l, l + 1 after every trial, accept
        on TV(z) <= TV(x), x kept after max_trials rejections)."""
        self.exchanges = 0
        ell = 0
        gamma_fixed = gamma0 > 0.0
        xh = x0.clone() if hasattr(x0, "clone") else x0.copy()     # x_{1/2} = x0
        f_half, g = self._gradient(xh, y_local)                    # g0 = A^T (A x0 - y)
        p = -g
        h = self._AtA(p)                                           # h0 = A^T A p0
        pth = _dot(p, h)
        alpha0 = -_dot(g, p) / pth if pth > 0.0 and math.isfinite(pth) else 0.0
        x = xh + alpha0 * p                                        # x1 = x0 + alpha p0
        k, it, status, trace = 1, 0, "ok", []
        if not (pth > 0.0) and _dot(g, g) != 0.0:
            status = "breakdown"
        while status == "ok":
            if not (f_half > eps):                                 # while f(x_{k-1/2}) > eps
                break
            if it >= max_iter:
                status = "max_iter"
                break
            row = [k, f_half, 0, -1, ell, 0.0]
            # x_{k+1/2} = perturbed(x_k)
            d, tvx = self.tv_grad(x)
            gn_tv = math.sqrt(_dot(d, d))
            xh = x
            if perturb and gn_tv > 0.0:
                if not gamma_fixed:
                    gamma0 = gamma0_rel * math.sqrt(_dot(x, x))
                    gamma_fixed = True
                v = -d / gn_tv
                row[3] = 0
                for t in range(max_trials):
                    gamma = gamma0 * a ** ell
                    z = x + gamma * v
                    ell += 1
                    row[2] = t + 1
                    if self.tv(z) <= tvx:
                        xh, row[3], row[5] = z, 1, gamma
                        break
            row[4] = ell
            # CG-PR-STEP from x_{k+1/2}
            f_half, gn = self._gradient(xh, y_local)               # g' and f(x_{k+1/2})
            beta = _dot(gn, h) / _dot(p, h)                        # beta = g'^T h / p^T h
            pn = -gn + beta * p                                    # p' = -g' + beta p
            hn = self._AtA(pn)                                     # h' = A^T A p'
            pnh = _dot(pn, hn)
            if pnh > 0.0 and math.isfinite(pnh):
                alpha = -_dot(gn, pn) / pnh                        # alpha = -g'^T p' / p'^T h'
            elif _dot(gn, gn) == 0.0:
                alpha = 0.0
            else:
                status = "breakdown"
                it += 1
                k += 1
                trace.append(row)
                break
            x = xh + alpha * pn                                    # x' = x + alpha p'
            p, h = pn, hn
            trace.append(row)
            k += 1
            it += 1
        return ShardedResult(xh, it, k, status, f_half, self.tv(xh), ell, gamma0 if gamma_fixed else 0.0,
                             trace, self.exchanges)


def torch_allreduce(value):
    """Sum over the default process group of a float, a numpy array or a torch
    tensor (FP64 for floats and host arrays; tensors keep their dtype)."""
    import numpy as np
    import torch
    import torch.distributed as dist

    if not dist.is_available() or not dist.is_initialized() or dist.get_world_size() == 1:
        return value
    if isinstance(value, float):
        t = torch.tensor([value], dtype=torch.float64)
        dist.all_reduce(t)
        return float(t.item())
    if isinstance(value, np.ndarray):
        t = torch.from_numpy(np.ascontiguousarray(value))
        dist.all_reduce(t)
        return t.numpy()
    dist.all_reduce(value)
    return value


def device_operators(n: int, n_angles: int, n_bins: int, block: tuple[int, int], dtype, device):
    """The library's operators for one rank's angle block on its GPU, and its
    TV entry points: (project_local, backproject_local, tv, tv_grad)."""
    from . import scg

    op = scg.Operator(n, n_angles, n_bins, dtype, device, angles=block)

    def tv(x):
        return float(scg.scg_tv(x))

    def tv_grad(x):
        g, t = scg.scg_tv_grad(x)
        return g, float(t)

    return op.project, op.backproject, tv, tv_grad
