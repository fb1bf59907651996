"""Pins of the oracle's gamma schedule (Sec. 3, Eq. gamma_sequence) against
hand-worked cases, independent of the oracle's own arithmetic.

Reading of the paper (it only says the gamma_k are "a subsequence of"
gamma_l = gamma_0 a^l and that each perturbation must not raise TV): one
global index l, starting at 0; trial t of a step uses gamma_0 a^l with the
current l, and l grows by one after every trial, accepted or not; the first
trial with TV(x + gamma v) <= TV(x) is taken; after max_trials rejections
x is kept; l is never reset between steps.

The hand-worked image is 2 x 2, x = [[0, 1], [1, 5]].  Its TV has a single
term (the interior grid is 1 x 1): TV(x) = sqrt(1^2 + 1^2) = sqrt 2.  The
subgradient of that term, on pixels (0,0), (1,0), (0,1), (1,1), is
(-sqrt 2, 1/sqrt 2, 1/sqrt 2, 0), of norm sqrt 3, so the nonascending
direction is v = (sqrt(2/3), -1/sqrt 6, -1/sqrt 6, 0).  Along it both
differences become 1 - gamma (1/sqrt 6 + 2/sqrt 6) = 1 - gamma sqrt(6)/2,
so TV(x + gamma v) = sqrt 2 |1 - gamma sqrt(6)/2|, which is <= TV(x)
exactly when 0 <= gamma <= 4/sqrt 6 = 1.63299...  With gamma_0 = 2 and
a = 0.9 the sequence is 2, 1.8, 1.62, 1.458, ...: the first two are
rejected and the third accepted.
"""
import math

import numpy as np
import pytest

import oracle

X = np.array([[0.0, 1.0], [1.0, 5.0]])
V = np.array([[math.sqrt(2.0 / 3.0), -1.0 / math.sqrt(6.0)], [-1.0 / math.sqrt(6.0), 0.0]])
G0, A = 2.0, 0.9
GAMMA_MAX = 4.0 / math.sqrt(6.0)


def tv_hand(gamma):
    return math.sqrt(2.0) * abs(1.0 - gamma * math.sqrt(6.0) / 2.0)


def test_hand_worked_boundary():
    # the closed form above, checked at the sequence's first values
    assert G0 > GAMMA_MAX and G0 * A > GAMMA_MAX and G0 * A * A < GAMMA_MAX
    assert tv_hand(G0 * A * A) < math.sqrt(2.0) < tv_hand(G0 * A)
    assert oracle.tv(X) == pytest.approx(math.sqrt(2.0), rel=1e-15)
    assert oracle.tv(X + G0 * A * A * V) == pytest.approx(tv_hand(G0 * A * A), rel=1e-13)


def test_third_trial_accepted_from_l0():
    xh, ell, gamma, trials, outcome = oracle.perturb_gamma(X, G0, A, 31, ell=0)
    assert outcome == 1 and trials == 3
    assert gamma == pytest.approx(G0 * A ** 2, rel=1e-15)      # gamma_0 a^2, not a^3
    assert ell == 3                                            # l advanced on the accepted trial too
    np.testing.assert_allclose(xh, X + G0 * A ** 2 * V, rtol=0, atol=1e-14)


def test_all_rejected_keeps_x():
    xh, ell, gamma, trials, outcome = oracle.perturb_gamma(X, G0, A, 2, ell=0)
    assert outcome == 0 and trials == 2 and ell == 2 and gamma == 0.0
    np.testing.assert_array_equal(xh, X)


@pytest.mark.parametrize("ell_in,trials,gamma_exp", [(1, 2, G0 * A ** 2), (3, 1, G0 * A ** 3),
                                                      (2, 1, G0 * A ** 2)])
def test_global_index_carries_over(ell_in, trials, gamma_exp):
    # a later step starts from the l the earlier steps left: its first trial
    # uses gamma_0 a^l with that l (not a^(l+1), not a^0)
    xh, ell, gamma, t, outcome = oracle.perturb_gamma(X, G0, A, 31, ell=ell_in)
    assert outcome == 1 and t == trials and ell == ell_in + trials
    assert gamma == pytest.approx(gamma_exp, rel=1e-15)
    np.testing.assert_allclose(xh, X + gamma_exp * V, rtol=0, atol=1e-14)


def test_zero_subgradient_leaves_l_unchanged():
    xh, ell, gamma, t, outcome = oracle.perturb_gamma(np.full((3, 3), 2.5), G0, A, 31, ell=7)
    assert outcome == -1 and ell == 7 and t == 0
    np.testing.assert_array_equal(xh, np.full((3, 3), 2.5))


def test_solve_trace_follows_one_global_index():
    # in a whole solve, l after step k = l after step k-1 + trials of step k
    # (never reset), and every accepted gamma is gamma_0 a^(l_after - 1)
    from paper_1709_04912_gb300 import inputs
    prob = inputs.make_problem(inputs.Workload("t24", 24, 30, 35, 5, 0.01, 1.05, 40), 3, oracle.project)
    for g0rel, a in ((0.05, 0.975), (0.5, 0.9)):
        _, res, tr = oracle.solve(prob.y, 24, variant="S-CG", eps=prob.eps, gamma0_rel=g0rel, a=a)
        g0 = res["gamma0_used"]
        prev = 0
        for row in tr:
            trials, accepted, ell, gamma = int(row[4]), row[5], int(row[6]), row[7]
            assert ell == prev + trials
            if accepted == 1:
                assert gamma == pytest.approx(g0 * a ** (ell - 1), rel=1e-12)
            prev = ell
        assert res["ell"] == prev
        assert any(r[4] > 1 for r in tr) or g0rel == 0.05
