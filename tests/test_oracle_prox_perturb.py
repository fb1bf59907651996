"""Pins of the oracle's proximal perturbation (footnote to Eq. superiorized:
the proximal operator of Eq. prox may define the perturbed vector).

Reading of the paper (it gives no step for the prox): perturbed(x_k) =
prox_{lambda TV}(x_k) with lambda = gamma_0 a^l / ||dTV(x_k)||, the implicit
(proximal) counterpart of the gamma rule's explicit step x_k + gamma v =
x_k - (gamma / ||dTV||) dTV; gamma_0 is fixed as in the gamma rule; a prox step
cannot raise TV, so no trial is taken and l grows by one per perturbed step;
a zero subgradient leaves x_k as it is.

The checks below use a TV and a subgradient restated here in numpy (isotropic
forward differences over the interior terms, the reading of the paper's TV
that the library and the oracle follow), not the oracle's own routines: lambda against gamma_0 a^l, the
prox optimality of the result by brute force (no random nearby point has a
lower lambda TV(z) + ||z - x||^2 / 2), TV not raised, the index, and the
special cases.
"""
import numpy as np
import pytest

import oracle


def tv_np(x):
    dx = x[:-1, 1:] - x[:-1, :-1]
    dy = x[1:, :-1] - x[:-1, :-1]
    return float(np.sqrt(dx * dx + dy * dy).sum())


def tv_subgrad_np(x):
    # d/dx of sum_t sqrt(dx_t^2 + dy_t^2), dx_t = x[i, j+1] - x[i, j],
    # dy_t = x[i+1, j] - x[i, j], terms with zero norm contributing 0
    g = np.zeros_like(x)
    dx = x[:-1, 1:] - x[:-1, :-1]
    dy = x[1:, :-1] - x[:-1, :-1]
    nrm = np.sqrt(dx * dx + dy * dy)
    safe = np.where(nrm > 0, nrm, 1.0)
    ux = np.where(nrm > 0, dx / safe, 0.0)
    uy = np.where(nrm > 0, dy / safe, 0.0)
    g[:-1, :-1] -= ux + uy
    g[:-1, 1:] += ux
    g[1:, :-1] += uy
    return g


def image(seed, n=12):
    rng = np.random.default_rng(seed)
    x = np.zeros((n, n))
    x[3:9, 2:7] = 1.0
    x[6:11, 5:10] += 0.5
    return x + 0.05 * rng.standard_normal((n, n))


@pytest.mark.parametrize("seed,ell", [(0, 0), (1, 3), (2, 10)])
def test_lambda_follows_the_gamma_sequence(seed, ell):
    x = image(seed)
    g0, a = 0.4, 0.9
    xh, ell_after, lam, outcome = oracle.perturb_prox(x, g0, a, 50, ell)
    assert outcome == 1 and ell_after == ell + 1
    gn = np.linalg.norm(tv_subgrad_np(x))
    assert lam == pytest.approx(g0 * a ** ell / gn, rel=1e-12)


@pytest.mark.parametrize("seed", [0, 1])
def test_result_is_the_prox_by_brute_force(seed):
    # with enough FGP steps the result minimises lambda TV(z) + ||z - x||^2 / 2:
    # no random nearby point does better
    x = image(seed, 8)
    xh, _, lam, _ = oracle.perturb_prox(x, 0.5, 0.9, 3000, 0)
    F = lambda z: lam * tv_np(z) + 0.5 * float(((z - x) ** 2).sum())
    f0 = F(xh)
    rng = np.random.default_rng(seed + 10)
    for scale in (1e-2, 1e-3):
        for _ in range(200):
            assert F(xh + scale * rng.standard_normal(x.shape)) >= f0 - 1e-9
    assert tv_np(xh) <= tv_np(x)


def test_tv_not_raised_and_step_bounded():
    x = image(3)
    for ell in range(0, 40, 7):
        xh, _, lam, _ = oracle.perturb_prox(x, 0.6, 0.95, 100, ell)
        assert tv_np(xh) <= tv_np(x) + 1e-12
        # x - x_half = lambda L^T w with |w_t| <= 1: each pixel lies in at most
        # three terms, each adding at most sqrt 2 -> |x - x_half| <= 3 sqrt(2) lambda
        assert np.abs(x - xh).max() <= 3.0 * np.sqrt(2.0) * lam + 1e-12


def test_constant_image_is_kept():
    x = np.full((6, 6), 2.5)
    xh, ell_after, lam, outcome = oracle.perturb_prox(x, 1.0, 0.9, 20, 4)
    assert outcome == -1 and ell_after == 4 and lam == 0.0
    assert np.array_equal(xh, x)


def test_vanishing_gamma_leaves_x():
    x = image(4)
    xh, _, lam, _ = oracle.perturb_prox(x, 1e-12, 0.9, 20, 0)
    assert np.abs(xh - x).max() < 1e-11


def test_solver_with_the_prox_rule():
    # whole S-CG and S-CG-K solves: every perturbed step lowers (or keeps) TV,
    # l advances once per perturbed step, the solve stops below eps, and it ends
    # with a lower TV than plain CG at the same eps (the paper's invariant)
    from paper_1709_04912_gb300 import inputs
    prob = inputs.make_problem(inputs.SMALL_FP64, 0, oracle.project)
    n = prob.work.n
    xc, rc, _ = oracle.solve(prob.y, n, variant="CG", eps=prob.eps, perturb="none")
    for variant in ("S-CG", "S-CG-K"):
        x, r, tr = oracle.solve(prob.y, n, variant=variant, eps=prob.eps, perturb="prox", gamma0_rel=0.05,
                                prox_iters=20)
        assert r["status"] == "ok" and r["f_final"] <= prob.eps
        rows = tr[: r["iters"]]
        pert = rows[rows[:, oracle.TRACE_FIELDS.index("accepted")] == 1]
        assert len(pert) > 0
        assert np.all(pert[:, oracle.TRACE_FIELDS.index("tv_after")]
                      <= pert[:, oracle.TRACE_FIELDS.index("tv_before")] + 1e-9)
        ells = rows[:, oracle.TRACE_FIELDS.index("ell")]
        assert int(ells[-1]) == len(pert)
        assert r["tv_final"] < rc["tv_final"]
