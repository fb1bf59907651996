"""Pins of the oracle's solvers against facts the paper and linear algebra fix.

* CG run long enough equals the dense least-squares solution (Eq. LS2), and
  its directions are A^T A-conjugate (Sec. 2).
* Without perturbations S-CG and S-CG-CD reproduce CG's iterates and S-PCG
  reproduces PCG's (Sec. 3, "Perturbation Resilient CG"), while restarted
  CG-K does not (same section).
* S-CG keeps the Appendix invariants <g_{n+1}, p_n> = 0, h_{k-1} = A^T A p_{k-1}
  and <A p_k, A p_{k-1}> = 0, obeys the descent bound of the Appendix Lemma
  under the eta rule, and terminates with f <= eps for eps > eps0 (Theorem).
* PCG is invariant to scaling the filter (alpha absorbs the scale).
Dense matrices and numpy's lstsq/SVD provide the independent side.
"""
import math

import numpy as np
import pytest

import oracle
from paper_1709_04912_gb300 import inputs


def dense_A(n, na, nb):
    J = n * n
    A = np.zeros((na * nb, J))
    for q in range(J):
        e = np.zeros(J)
        e[q] = 1.0
        A[:, q] = oracle.project(e.reshape(n, n), na, nb).ravel()
    return A


TINY = inputs.Workload("tiny8", 8, 12, 12, 4, 0.02, 1.05, 100)


@pytest.fixture(scope="module")
def tiny():
    prob = inputs.make_problem(TINY, 11, oracle.project)
    A = dense_A(TINY.n, TINY.n_angles, TINY.n_bins)
    x_ls, *_ = np.linalg.lstsq(A, prob.y.ravel(), rcond=None)
    eps0 = 0.5 * np.sum((prob.y.ravel() - A @ x_ls) ** 2)
    return prob, A, x_ls, eps0


def f_dense(A, y, x):
    return 0.5 * float(np.sum((y.ravel() - A @ x.ravel()) ** 2))


def test_cg_reaches_dense_least_squares(tiny):
    prob, A, x_ls, eps0 = tiny
    n = TINY.n
    x, res, _ = oracle.solve(prob.y, n, variant="CG", eps=eps0 * (1 + 1e-13) + 1e-300,
                             perturb="none", max_iter=4 * n * n)
    rel = np.linalg.norm(x.ravel() - x_ls) / np.linalg.norm(x_ls)
    assert rel < 1e-8, rel


def test_cg_directions_are_conjugate(tiny):
    prob, A, x_ls, eps0 = tiny
    ps = []
    oracle.solve(prob.y, TINY.n, variant="CG", eps=eps0 * 1.0001, perturb="none", max_iter=12,
                 callback=lambda it, xn, xh, p, h, g: ps.append(p.ravel()))
    for p0, p1 in zip(ps[:-1], ps[1:]):
        a0, a1 = A @ p0, A @ p1
        assert abs(a0 @ a1) <= 1e-9 * np.linalg.norm(a0) * np.linalg.norm(a1)


def collect_x(variant, y, n, **kw):
    xs = []
    oracle.solve(y, n, variant=variant, callback=lambda it, xn, xh, p, h, g: xs.append(xn.ravel()), **kw)
    return xs


@pytest.mark.parametrize("variant", ["S-CG", "S-CG-CD"])
def test_unperturbed_s_cg_reproduces_cg(tiny, variant):
    prob, A, x_ls, eps0 = tiny
    kw = dict(eps=eps0 * (1 + 1e-13) + 1e-300, perturb="none", max_iter=20)
    cg = collect_x("CG", prob.y, TINY.n, **kw)
    sx = collect_x(variant, prob.y, TINY.n, **kw)
    # S-CG's first loop body yields x_2; CG's yields x_1.  The two recursions
    # are equal in exact arithmetic; their rounding differences grow about
    # tenfold per step on this problem, so the first six iterates are compared.
    assert min(len(sx), len(cg) - 1) >= 6
    for k in range(6):
        scale = np.linalg.norm(cg[k + 1])
        assert np.linalg.norm(sx[k] - cg[k + 1]) <= 1e-10 * scale, k


@pytest.mark.parametrize("gain", [1.0, 2.5])
def test_identity_filter_reduces_preconditioned_variants(tiny, gain):
    # With c(w) = gain for all w the filter is gain * identity, so
    # z = A^T(gain * (Ax - y)) = gain * g: PCG must reproduce CG exactly (the
    # scale cancels in alpha), S-PCG must reproduce S-CG and S-PCG-K S-CG-K.
    prob, A, x_ls, eps0 = tiny
    kw = dict(eps=eps0 * (1 + 1e-13) + 1e-300, max_iter=8, filter_identity=1, filter_gain=gain)
    for plain, pre, extra in (("CG", "PCG", dict(perturb="none")),
                              ("S-CG", "S-PCG", dict(gamma0_rel=0.05)),
                              ("S-CG-K", "S-PCG-K", dict(gamma0_rel=0.05))):
        a = collect_x(plain, prob.y, TINY.n, **kw, **extra)
        b = collect_x(pre, prob.y, TINY.n, **kw, **extra)
        assert len(a) == len(b) == 8
        for k in range(5):
            assert np.linalg.norm(a[k] - b[k]) <= 1e-10 * np.linalg.norm(a[k]), (plain, k)


def test_real_filter_changes_preconditioned_variants(tiny):
    # the filter of Sec. 3 acts on the residual, so S-PCG is not S-CG
    prob, A, x_ls, eps0 = tiny
    kw = dict(eps=eps0 * 1.001, perturb="none", max_iter=3)
    a = collect_x("S-CG", prob.y, TINY.n, **kw)
    b = collect_x("S-PCG", prob.y, TINY.n, **kw)
    assert np.linalg.norm(a[0] - b[0]) > 1e-3 * np.linalg.norm(a[0])


@pytest.mark.parametrize("variant", ["S-PCG", "S-CG-CD"])
def test_exact_line_search_invariant_holds_for_other_variants(tiny, variant):
    # alpha = -g'^T p' / p'^T h' makes <g_{k+1}, p_k> = 0 whatever p' is
    prob, A, x_ls, eps0 = tiny
    y = prob.y.ravel()
    rec = []
    oracle.solve(prob.y, TINY.n, variant=variant, eps=eps0 * 1.0001, gamma0_rel=0.05, max_iter=15,
                 callback=lambda it, xn, xh, p, h, g: rec.append((xn.ravel(), p.ravel())))
    for xn, p in rec:
        g_next = A.T @ (A @ xn - y)
        assert abs(g_next @ p) <= 1e-9 * np.linalg.norm(g_next) * np.linalg.norm(p) + 1e-14


@pytest.mark.parametrize("variant", ["CG", "PCG", "S-CG", "S-CG-CD", "S-PCG", "S-CG-K", "S-PCG-K"])
def test_resume_from_exported_state_is_exact(tiny, variant):
    # a run split at any loop body continues bit-for-bit
    prob, A, x_ls, eps0 = tiny
    kw = dict(variant=variant, eps=eps0 * 1.0001, gamma0_rel=0.05)
    x_full, r_full, _ = oracle.solve(prob.y, TINY.n, max_iter=9, **kw)
    _, r1, _, st = oracle.solve(prob.y, TINY.n, max_iter=4, want_state=True, **kw)
    x2, r2, _ = oracle.solve(prob.y, TINY.n, max_iter=5, resume=st, **kw)
    assert r1["iters"] + r2["iters"] == r_full["iters"]
    assert r2["ell"] == r_full["ell"]
    np.testing.assert_array_equal(x2, x_full)


def test_restarted_cg_k_is_not_cg(tiny):
    prob, A, x_ls, eps0 = tiny
    kw = dict(eps=eps0 * (1 + 1e-13) + 1e-300, perturb="none", max_iter=6)
    cg = collect_x("CG", prob.y, TINY.n, **kw)
    sk = collect_x("S-CG-K", prob.y, TINY.n, K=2, **kw)
    # first CG-2 call from x0 is exactly two CG steps ...
    assert np.linalg.norm(sk[0] - cg[1]) <= 1e-12 * np.linalg.norm(cg[1])
    # ... but the restart loses conjugacy with the earlier directions
    assert np.linalg.norm(sk[1] - cg[3]) > 1e-6 * np.linalg.norm(cg[3])


def test_cg_k_literal_loop_takes_one_more_step(tiny):
    prob, A, x_ls, eps0 = tiny
    kw = dict(eps=eps0 * (1 + 1e-13) + 1e-300, perturb="none", max_iter=2)
    cg = collect_x("CG", prob.y, TINY.n, max_iter=4, eps=kw["eps"], perturb="none")
    sk = collect_x("S-CG-K", prob.y, TINY.n, K=2, k_inclusive=1, **kw)
    assert np.linalg.norm(sk[0] - cg[2]) <= 1e-12 * np.linalg.norm(cg[2])


def test_s_cg_appendix_invariants(tiny):
    prob, A, x_ls, eps0 = tiny
    y = prob.y.ravel()
    rec = []
    oracle.solve(prob.y, TINY.n, variant="S-CG", eps=eps0 * 1.0001, perturb="gamma",
                 gamma0_rel=0.05, max_iter=25,
                 callback=lambda it, xn, xh, p, h, g: rec.append((xn.ravel(), p.ravel(), h.ravel())))
    assert len(rec) >= 10
    for k, (xn, p, h) in enumerate(rec):
        g_next = A.T @ (A @ xn - y)                  # g_{k+1} at x_{k+1}
        assert abs(g_next @ p) <= 1e-9 * np.linalg.norm(g_next) * np.linalg.norm(p) + 1e-14
        np.testing.assert_allclose(h, A.T @ (A @ p), rtol=0, atol=1e-10 * np.linalg.norm(h))
        if k > 0:
            ap, ap0 = A @ p, A @ rec[k - 1][1]
            assert abs(ap @ ap0) <= 1e-9 * np.linalg.norm(ap) * np.linalg.norm(ap0)


def test_oracle_norm_of_A_matches_svd(tiny):
    _, A, _, _ = tiny
    assert oracle.norm_A(TINY.n, TINY.n_angles, TINY.n_bins, 300) == pytest.approx(
        np.linalg.norm(A, 2), rel=1e-8)


def test_eta_rule_descent_bound(tiny):
    prob, A, x_ls, eps0 = tiny
    y = prob.y.ravel()
    c = np.linalg.norm(A, 2)
    eta1 = 1 / (4 * c * c)
    eta2 = (-1 + math.sqrt(1 + 1 / 32)) / (c * c)   # (2 + c^2 eta) eta = 1/(32 c^2)
    eta0 = min(eta1, eta2)
    xs = []
    oracle.solve(prob.y, TINY.n, variant="S-CG", eps=eps0 * 1.0001, perturb="eta", eta0=eta0,
                 max_iter=30, callback=lambda it, xn, xh, p, h, g: xs.append(xn.ravel()))
    assert len(xs) >= 5
    for xk, xk1 in zip(xs[:-1], xs[1:]):
        gk = A.T @ (A @ xk - y)
        drop = 2 * f_dense(A, prob.y, xk) - 2 * f_dense(A, prob.y, xk1)
        bound = (gk @ gk) / (32 * c * c)
        assert drop >= bound - 1e-12 * abs(2 * f_dense(A, prob.y, xk))


@pytest.mark.parametrize("variant", ["S-CG", "S-CG-CD", "S-PCG", "S-CG-K", "S-PCG-K"])
@pytest.mark.parametrize("rel", [0.3, 0.02])
def test_superiorized_variants_terminate_with_f_below_eps(tiny, variant, rel):
    prob, A, x_ls, eps0 = tiny
    f0 = f_dense(A, prob.y, np.zeros(TINY.J))
    eps = eps0 + rel * (f0 - eps0)
    x, res, tr = oracle.solve(prob.y, TINY.n, variant=variant, eps=eps, gamma0_rel=0.1,
                              max_iter=500)
    assert res["status"] == "ok", res
    assert f_dense(A, prob.y, x) <= eps
    assert res["f_final"] == pytest.approx(f_dense(A, prob.y, x), rel=1e-10)
    acc = tr[:, 5] == 1
    assert np.all(tr[acc, 3] <= tr[acc, 2])          # accepted: TV(z) <= TV(x)


def test_pcg_invariant_to_filter_scale(tiny):
    prob, A, x_ls, eps0 = tiny
    kw = dict(eps=eps0 * 1.001, perturb="none", max_iter=8)
    x1, r1, _ = oracle.solve(prob.y, TINY.n, variant="PCG", filter_gain=1.0, **kw)
    x2, r2, _ = oracle.solve(prob.y, TINY.n, variant="PCG", filter_gain=3.7, **kw)
    assert r1["iters"] == r2["iters"]
    np.testing.assert_allclose(x1, x2, rtol=0, atol=1e-10 * np.linalg.norm(x1))


def test_superiorization_lowers_tv_at_same_eps():
    # Abstract / Fig. 3: lower TV than CG at the same eps (empirical, checked
    # over seeds; not a theorem)
    work = inputs.Workload("small32", 32, 45, 46, 6, 0.01, 1.05, 200)
    wins = 0
    for seed in range(6):
        prob = inputs.make_problem(work, seed, oracle.project)
        _, rc, _ = oracle.solve(prob.y, work.n, variant="CG", eps=prob.eps, perturb="none",
                                max_iter=200)
        _, rs, _ = oracle.solve(prob.y, work.n, variant="S-CG", eps=prob.eps, gamma0_rel=0.05,
                                max_iter=200)
        assert rc["status"] == "ok" and rs["status"] == "ok"
        wins += rs["tv_final"] < rc["tv_final"]
    assert wins >= 5
