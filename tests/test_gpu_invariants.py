"""The Appendix's invariants on states exported by the GPU solver (FP64),
checked with the GPU's own A and A^T -- properties the paper proves, so they
pin the device path independently of the oracle.

For S-CG / S-PCG the exported state after k bodies is x = x_k,
x_half = x_{k-1/2}, p = p_{k-1}, h = h_{k-1} (include/scg.h):
  * h_{k-1} = A^T A p_{k-1};
  * the step from x_{k-1/2} to x_k is along p_{k-1}, and the gradient at x_k
    is orthogonal to it (exact line search: <A x_k - y, A p_{k-1}> = 0);
  * consecutive directions are A-conjugate: <A p_k, A p_{k-1}> = 0 (S-CG; for
    plain CG likewise <A p_{k+1}, A p_k> = 0).
"""
import numpy as np
import pytest
import torch

import oracle
from paper_1709_04912_gb300 import inputs, scg

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


@pytest.fixture(scope="module", autouse=True)
def lib():
    assert torch.cuda.is_available()
    return scg.load()


@pytest.fixture(scope="module")
def small():
    return inputs.make_problem(inputs.SMALL_FP64, 1, oracle.project)


def state_after(prob, variant, k, **kw):
    y = torch.tensor(prob.y, dtype=torch.float64, device=DEV)
    r = scg.scg_solve(y, prob.work.n, variant, prob.eps * 1e-6, max_iter=k, want_state=True,
                      gamma0_rel=0.05, **kw)
    assert r.status == "max_iter" and r.iters == k
    return y, r.state


def A(v, work):
    return scg.scg_project(v, work.n_angles, work.n_bins)


def AT(r, work):
    return scg.scg_backproject(r, work.n)


def dot(a, b):
    return float((a * b).sum())


@pytest.mark.parametrize("variant", ["S-CG", "S-PCG"])
@pytest.mark.parametrize("k", [2, 5])
def test_h_is_AtA_p_and_the_step_is_an_exact_line_search(small, variant, k):
    w = small.work
    y, st = state_after(small, variant, k)
    p, h, x, xh = st["p"], st["h"], st["x"], st["x_half"]
    ath = AT(A(p, w), w)
    assert float((h - ath).norm()) <= 1e-11 * float(ath.norm())
    d = x - xh                                  # x_k - x_{k-1/2} = alpha p_{k-1}
    alpha = dot(d, p) / dot(p, p)
    assert float((d - alpha * p).norm()) <= 1e-11 * float(d.norm())
    g = AT(A(x, w) - y, w)                      # gradient of f at x_k
    assert abs(dot(g, p)) <= 1e-10 * float(g.norm()) * float(p.norm())


def test_s_cg_directions_are_A_conjugate(small):
    w = small.work
    _, s3 = state_after(small, "S-CG", 3)       # p_2
    _, s4 = state_after(small, "S-CG", 4)       # p_3
    a2, a3 = A(s3["p"], w), A(s4["p"], w)
    assert abs(dot(a2, a3)) <= 1e-10 * float(a2.norm()) * float(a3.norm())


def test_cg_directions_are_A_conjugate_and_g_is_the_gradient(small):
    w = small.work
    y, s3 = state_after(small, "CG", 3, perturb="none")
    _, s4 = state_after(small, "CG", 4, perturb="none")
    a3, a4 = A(s3["p"], w), A(s4["p"], w)
    assert abs(dot(a3, a4)) <= 1e-10 * float(a3.norm()) * float(a4.norm())
    g = AT(A(s4["x"], w) - y, w)                # the recursive g_k equals A^T (A x_k - y)
    assert float((s4["g"] - g).norm()) <= 1e-10 * float(g.norm())
