"""The oracle's reading of the loop test "while f(x) > eps" (Algorithms 1-14)
for non-finite data: a NaN f neither continues nor converges -- the solve ends
with the breakdown status, at its first test, for every variant and for FISTA.
Clean data reaches f <= eps with status ok."""
import numpy as np
import pytest

import oracle
from paper_1709_04912_gb300 import inputs


@pytest.fixture(scope="module")
def problem():
    return inputs.make_problem(inputs.SMALL_FP64, 0, oracle.project)


@pytest.mark.parametrize("variant", ["CG", "PCG", "S-CG", "S-CG-CD", "S-CG-K", "S-PCG", "S-PCG-K"])
def test_nan_data_is_a_breakdown(problem, variant):
    y = problem.y.copy()
    y[y.shape[0] // 3, y.shape[1] // 2] = np.nan
    kw = dict(perturb="none") if variant in ("CG", "PCG") else dict(gamma0_rel=0.05)
    _, r, _ = oracle.solve(y, problem.work.n, variant=variant, eps=problem.eps, **kw)
    assert r["status"] == "breakdown" and r["iters"] <= 1
    _, r, _ = oracle.solve(problem.y, problem.work.n, variant=variant, eps=problem.eps, **kw)
    assert r["status"] == "ok" and r["f_final"] <= problem.eps


def test_nan_data_is_a_breakdown_in_fista(problem):
    y = problem.y.copy()
    y[1, 1] = np.nan
    n = problem.work.n
    c2 = oracle.norm_A(n, y.shape[0], y.shape[1], 50) ** 2
    _, r, _ = oracle.fista(y, n, problem.eps, 1.0, c2, prox_iters=5, max_iter=20)
    assert r["status"] == "breakdown" and r["iters"] == 0
