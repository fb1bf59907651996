"""Pins of the oracle's several perturbations per step.

Reading (the printed algorithms take one perturbation per step; the
superiorization scheme they follow allows N nonascending steps per
iteration): perturbed(x_k) applies the rule perturb_steps times in
succession, each from the current point with its own subgradient; the
gamma rule's index l runs on across the sub-steps and each sub-step has its
own trial budget; a zero subgradient ends the sequence.  The trace row keeps
TV(x_k) from the first sub-step and the other fields of the last.

Checked against the single-step rule, which test_oracle_gamma.py pins by hand:
a whole solve's first perturbation equals the single-step gamma rule applied
three times in sequence; one sub-step reproduces the printed algorithm
exactly; every sub-step lowers TV; the solve still stops below eps with a TV
below plain CG's.
"""
import numpy as np
import pytest

import oracle
from paper_1709_04912_gb300 import inputs

F = oracle.TRACE_FIELDS


@pytest.fixture(scope="module")
def problem():
    return inputs.make_problem(inputs.SMALL_FP64, 0, oracle.project)


def test_one_sub_step_is_the_printed_algorithm(problem):
    n = problem.work.n
    xa, ra, ta = oracle.solve(problem.y, n, variant="S-CG", eps=problem.eps, gamma0_rel=0.05)
    xb, rb, tb = oracle.solve(problem.y, n, variant="S-CG", eps=problem.eps, gamma0_rel=0.05, perturb_steps=1)
    assert np.array_equal(xa, xb) and np.array_equal(ta, tb) and ra == rb


def test_first_step_is_the_single_rule_three_times(problem):
    # stop after the first perturbation: max_iter = 1 with a tiny eps; the
    # exported state holds x_{1/2}; the set-up gives x_1 = x_0 + alpha p_0
    n = problem.work.n
    x0 = oracle.solve(problem.y, n, variant="S-CG", eps=problem.eps * 1e-9, gamma0_rel=0.05, max_iter=0,
                      want_state=True)[3]["x"]
    _, r, tr, st = oracle.solve(problem.y, n, variant="S-CG", eps=problem.eps * 1e-9, gamma0_rel=0.05,
                                perturb_steps=3, max_iter=1, want_state=True)
    g0 = r["gamma0_used"]
    x, ell, outcomes = x0, 0, []
    for _ in range(3):
        x, ell, _, _, outcome = oracle.perturb_gamma(x, g0, 0.975, 32, ell)
        outcomes.append(outcome)
    # (at x_1 the first sub-step rejects all 32 trials -- gamma_0 is large this
    # early -- and a later one, from a smaller gamma, is accepted)
    assert 1 in outcomes
    np.testing.assert_array_equal(st["x_half"], x)
    assert int(tr[0, F.index("ell")]) == ell
    assert tr[0, F.index("tv_after")] < tr[0, F.index("tv_before")]


def test_solve_with_several_perturbations(problem):
    n = problem.work.n
    _, rc, _ = oracle.solve(problem.y, n, variant="CG", eps=problem.eps, perturb="none")
    _, r1, t1 = oracle.solve(problem.y, n, variant="S-CG", eps=problem.eps, gamma0_rel=0.05)
    for rule in ("gamma", "prox"):
        for variant in ("S-CG", "S-CG-K"):
            _, r, tr = oracle.solve(problem.y, n, variant=variant, eps=problem.eps, gamma0_rel=0.05,
                                    perturb=rule, perturb_steps=3, prox_iters=20)
            assert r["status"] == "ok" and r["f_final"] <= problem.eps
            rows = tr[: r["iters"]]
            acc = rows[:, F.index("accepted")] == 1
            assert np.all(rows[acc, F.index("tv_after")] <= rows[acc, F.index("tv_before")] + 1e-9)
            assert r["tv_final"] < rc["tv_final"]
    _, r3, _ = oracle.solve(problem.y, n, variant="S-CG", eps=problem.eps, gamma0_rel=0.05, perturb_steps=3)
    assert r3["ell"] > r1["ell"]
