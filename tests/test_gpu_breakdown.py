"""Non-finite data ends a solve with SCG_ERR_BREAKDOWN, never a hang or a
false convergence, and in a batch it stops only its own problem.

Fault injection on the host: one sinogram value is NaN.  The residual, f and
the gradient then carry the NaN, so the first step size's denominator p^T h is
not a finite positive number while ||g||^2 is not zero: the solver must stop
with the breakdown status (the CG denominators of Algorithms 1-14 are checked
on the device), within max_iter bodies.  In a batch, the neighbour's result
must still equal its solo solve bit for bit.
"""
import math

import pytest
import torch

import oracle
from paper_1709_04912_gb300 import inputs, scg

pytestmark = pytest.mark.gpu
DEV = "cuda:0"
BREAKDOWN = -4


@pytest.fixture(scope="module", autouse=True)
def lib():
    assert torch.cuda.is_available()
    return scg.load()


@pytest.fixture(scope="module")
def problem():
    prob = inputs.make_problem(inputs.SMALL_FP64, 0, oracle.project)
    return prob, torch.tensor(prob.y, dtype=torch.float32, device=DEV)


def poisoned(y):
    z = y.clone()
    z[y.shape[0] // 3, y.shape[1] // 2] = float("nan")
    return z


@pytest.mark.parametrize("variant", ["S-CG", "CG", "S-PCG", "S-CG-K"])
@pytest.mark.parametrize("dtype", [torch.float32, torch.float64])
def test_nan_data_reports_breakdown(problem, variant, dtype):
    prob, y = problem
    kw = dict(gamma0_rel=0.05) if variant != "CG" else dict(perturb="none")
    r = scg.scg_solve(poisoned(y).to(dtype), prob.work.n, variant, prob.eps, **kw)
    assert r.status_code == BREAKDOWN, (r.status, r.iters)
    assert r.iters <= prob.work.max_iter


def test_breakdown_stays_in_its_problem_in_a_batch(problem):
    prob, y = problem
    n = prob.work.n
    solo = scg.scg_solve(y, n, "S-CG", prob.eps, gamma0_rel=0.05)
    res = scg.scg_solve_batch([poisoned(y), y], [n, n], "S-CG", [prob.eps, prob.eps], gamma0_rel=0.05)
    assert res[0].status_code == BREAKDOWN
    assert res[1].status_code == solo.status_code and res[1].iters == solo.iters
    assert torch.equal(res[1].x, solo.x) and res[1].f_final == solo.f_final
    assert math.isfinite(res[1].tv_final)
