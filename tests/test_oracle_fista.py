"""Pins of the oracle's FISTA (Sec. 2, Eqs. FISTA, FISTA-u) and of its TV prox
(Eq. prox, computed by Beck and Teboulle's fast gradient projection on the
dual), against things the oracle does not compute itself:

* the prox of a 2 x 2 image in closed form: TV has one term, and for
  b = [[0, d], [d, *]] the prox shrinks both differences to
  e = max(0, d - 3 alpha / sqrt 2) and moves b[0,0] up by 2 (d - e) / 3
  (minimise (e - d)^2 / 3 + alpha sqrt(2) e after eliminating x[0,0]);
* the duality gap of a long FGP run: primal 1/2||x - b||^2 + alpha TV(x)
  (TV and L^T written out here in numpy) against the dual value
  1/2||b||^2 - 1/2||b - alpha L^T w||^2, with |w| <= 1 at every term;
* plain gradient projection (no momentum) reaching the same prox;
* ISTA (FISTA without momentum) lowering f + lambda TV at every step, and
  FISTA's objective gap within Beck and Teboulle's 2 c^2 ||x0 - x*||^2/(k+1)^2;
* lambda = 0: FISTA reaches the least-squares residual of a dense solve.
"""
import math

import numpy as np
import pytest

import oracle
from paper_1709_04912_gb300 import inputs


def tv_np(x):
    du = x[1:, :-1] - x[:-1, :-1]
    dv = x[:-1, 1:] - x[:-1, :-1]
    return float(np.sum(np.sqrt(du * du + dv * dv)))


def lt_np(p, q):
    n = p.shape[0] + 1
    out = np.zeros((n, n))
    out[:-1, :-1] -= p + q
    out[1:, :-1] += p
    out[:-1, 1:] += q
    return out


@pytest.mark.parametrize("d,alpha", [(1.0, 0.1), (2.0, 0.4), (1.0, 0.5), (0.3, 0.05)])
def test_prox_2x2_closed_form(d, alpha):
    b = np.array([[0.0, d], [d, 5.0]])
    x = oracle.tv_prox(b, alpha, 2000)
    e = max(0.0, d - 3.0 * alpha / math.sqrt(2.0))
    z = 2.0 * (d - e) / 3.0
    expect = np.array([[z, z + e], [z + e, 5.0]])
    np.testing.assert_allclose(x, expect, rtol=0, atol=1e-9)


def test_prox_duality_gap_closes():
    rng = np.random.default_rng(3)
    b = rng.standard_normal((10, 10)) + np.outer(np.arange(10) > 4, np.ones(10))
    alpha = 0.3
    x, p, q = oracle.tv_prox(b, alpha, 4000, want_dual=True)
    assert np.all(p * p + q * q <= 1.0 + 1e-12)
    np.testing.assert_allclose(x, b - alpha * lt_np(p, q), rtol=0, atol=1e-12)
    primal = 0.5 * np.sum((x - b) ** 2) + alpha * tv_np(x)
    dual = 0.5 * np.sum(b * b) - 0.5 * np.sum((b - alpha * lt_np(p, q)) ** 2)
    assert dual <= primal + 1e-12
    assert primal - dual <= 1e-7 * primal


def test_plain_gradient_projection_reaches_the_same_prox():
    rng = np.random.default_rng(4)
    b = rng.standard_normal((7, 7))
    fast = oracle.tv_prox(b, 0.2, 3000)
    slow = oracle.tv_prox(b, 0.2, 60000, accel=False)
    np.testing.assert_allclose(fast, slow, rtol=0, atol=1e-6)


def test_prox_of_constant_is_itself():
    b = np.full((6, 6), 1.7)
    np.testing.assert_array_equal(oracle.tv_prox(b, 0.5, 50), b)


@pytest.fixture(scope="module")
def tiny():
    w = inputs.Workload("f8", 8, 12, 13, 4, 0.02, 1.05, 100)
    prob = inputs.make_problem(w, 2, oracle.project)
    c = oracle.norm_A(w.n, w.n_angles, w.n_bins, 400)
    return prob, c


def objective(prob, x, lam):
    r = oracle.project(x, prob.work.n_angles, prob.work.n_bins) - prob.y
    return 0.5 * float(np.sum(r * r)) + lam * tv_np(x)


def test_ista_decreases_the_objective_every_step(tiny):
    prob, c = tiny
    lam = 0.5
    fs = []
    for k in range(1, 16):
        x, _, _ = oracle.fista(prob.y, prob.work.n, 1e-12, lam, c * c, prox_iters=400, accel=False, max_iter=k)
        fs.append(objective(prob, x, lam))
    assert all(b <= a * (1 + 1e-9) for a, b in zip(fs[:-1], fs[1:]))


def test_fista_objective_within_the_accelerated_bound(tiny):
    prob, c = tiny
    lam = 0.5
    x_star, _, _ = oracle.fista(prob.y, prob.work.n, 1e-12, lam, c * c, prox_iters=400, max_iter=3000)
    f_star = objective(prob, x_star, lam)
    r2 = float(np.sum(x_star ** 2))                   # x0 = 0
    for k in (2, 5, 10, 20):
        x, _, _ = oracle.fista(prob.y, prob.work.n, 1e-12, lam, c * c, prox_iters=400, max_iter=k)
        gap = objective(prob, x, lam) - f_star
        assert gap <= 2.0 * c * c * r2 / (k + 1) ** 2 + 1e-8 * f_star


def test_fista_without_regularisation_reaches_least_squares(tiny):
    prob, c = tiny
    w = prob.work
    A = np.stack([oracle.project(np.eye(w.J)[k].reshape(w.n, w.n), w.n_angles, w.n_bins).ravel()
                  for k in range(w.J)], axis=1)
    x_ls = np.linalg.lstsq(A, prob.y.ravel(), rcond=None)[0]
    f_ls = 0.5 * float(np.sum((A @ x_ls - prob.y.ravel()) ** 2))
    eps = f_ls * 1.001 + 1e-12
    x, res, tr = oracle.fista(prob.y, w.n, eps, 0.0, c * c, prox_iters=5, max_iter=20000)
    assert res["status"] == "ok" and res["f_final"] <= eps
    # t_k grows like (k+1)/2 and beta_k = (t_k - 1)/t_{k+1}
    t = tr[:, 8]
    assert t[0] == 1.0 and np.all(np.diff(t) > 0)
    np.testing.assert_allclose(tr[:-1, 9], (t[:-1] - 1.0) / t[1:], rtol=1e-14)
