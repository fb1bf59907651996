"""The Appendix's perturbation rule on the device (SCG_PERTURB_ETA), through the
C ABI: x_{k+1/2} = x_k + u_k with ||u_k|| = eta0 ||g_k||, g_k = A^T(A x_k - y),
along v_k = -dTV/||dTV|| (Eq. up bnd u_k; direction as in the gamma rule).

* Whole solves of every superiorized variant against the oracle's eta rule
  (FP64: same iterations, same perturbation sizes ||u_k||, x within 1e-9;
  FP32: the same iterations, x within a bound ~3x the measured error).
* The Lemma on states the device exports: with 0 < eta0 <= min(eta1, eta2)
  (eta1 = 1/(4c^2), eta2 the positive root of (2 + c^2 eta) eta = 1/(32 c^2),
  c = ||A||_2), every S-CG step satisfies
  2 f(x_k) - 2 f(x_{k+1}) >= ||g_k||^2 / (32 c^2), checked with the oracle's A.
"""
import math

import numpy as np
import pytest
import torch

import oracle
from paper_1709_04912_gb300 import inputs, scg

pytestmark = pytest.mark.gpu
DEV = "cuda:0"
S_VARIANTS = ["S-CG", "S-CG-CD", "S-CG-K", "S-PCG", "S-PCG-K"]


def rel(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


@pytest.fixture(scope="module")
def small():
    return inputs.make_problem(inputs.SMALL_FP64, 0, oracle.project)


@pytest.fixture(scope="module")
def eta(small):
    w = small.work
    c = oracle.norm_A(w.n, w.n_angles, w.n_bins, 200)
    eta1 = 1.0 / (4.0 * c * c)
    eta2 = (-1.0 + math.sqrt(1.0 + 1.0 / 32.0)) / (c * c)
    return c, min(eta1, eta2)


def gpu(prob, dtype, variant, **kw):
    y = torch.tensor(prob.y, dtype=dtype, device=DEV)
    return scg.scg_solve(y, prob.work.n, variant, kw.pop("eps", prob.eps), trace=True, **kw)


@pytest.mark.parametrize("variant", S_VARIANTS)
def test_eta_rule_matches_the_oracle_fp64(small, eta, variant):
    _, e0 = eta
    xo, ro, to = oracle.solve(small.y, small.work.n, variant=variant, eps=small.eps, perturb="eta", eta0=e0)
    r = gpu(small, torch.float64, variant, perturb="eta", eta0=e0)
    assert r.status == ro["status"] == "ok" and r.iters == ro["iters"] and r.ell == ro["ell"] == 0
    np.testing.assert_array_equal(r.trace[:, [4, 5, 6]], to[:, [4, 5, 6]])
    assert np.all(to[1:, 5] == 1)                       # a perturbation in every step (S-CG-K and
                                                        # S-PCG-K start from x_0 = 0: no dTV to follow)
    np.testing.assert_allclose(r.trace[:, 7], to[:, 7], rtol=1e-9)   # ||u_k||
    assert rel(r.x.cpu().numpy(), xo) <= 1e-9


@pytest.mark.parametrize("variant", ["S-CG", "S-PCG"])
def test_eta_rule_fp32(small, eta, variant):
    _, e0 = eta
    xo, ro, _ = oracle.solve(small.y, small.work.n, variant=variant, eps=small.eps, perturb="eta", eta0=e0)
    r = gpu(small, torch.float32, variant, perturb="eta", eta0=e0)
    err = rel(r.x.cpu().numpy(), xo)
    print(f"eta rule {variant} FP32: iters {r.iters}/{ro['iters']} rel L2 {err:.2e}")
    assert r.status == "ok" and r.iters == ro["iters"]
    assert err <= 2e-5


def test_lemma_descent_bound_on_device_states(small, eta):
    c, e0 = eta
    w = small.work
    y = torch.tensor(small.y, dtype=torch.float64, device=DEV)
    xs = []
    for k in range(1, 9):
        r = scg.scg_solve(y, w.n, "S-CG", small.eps * 1e-6, perturb="eta", eta0=e0, max_iter=k,
                          want_state=True)
        assert r.status == "max_iter" and r.iters == k
        xs.append(r.state["x"].cpu().numpy())          # x_{k+1} after k bodies (x_1 comes from the set-up)

    def f(x):
        res = oracle.project(x, w.n_angles, w.n_bins) - small.y
        return 0.5 * float(np.sum(res * res))

    for xk, xk1 in zip(xs[:-1], xs[1:]):
        gk = oracle.backproject(oracle.project(xk, w.n_angles, w.n_bins) - small.y, w.n)
        drop = 2.0 * f(xk) - 2.0 * f(xk1)
        bound = float(np.sum(gk * gk)) / (32.0 * c * c)
        assert drop >= bound - 1e-10 * 2.0 * f(xk), (drop, bound)
        assert bound > 0.0


def test_eta_rule_in_a_batch_equals_solo(small, eta):
    _, e0 = eta
    probs = [small] + [inputs.make_problem(inputs.Workload(f"e{q}", n, na, nb, 6, 0.01, 1.05, 100), 40 + q,
                                           oracle.project)
                       for q, (n, na, nb) in enumerate([(48, 60, 70), (33, 45, 47)])]
    ys = [torch.tensor(p.y, dtype=torch.float32, device=DEV) for p in probs]
    got = scg.scg_solve_batch(ys, [p.work.n for p in probs], "S-CG", [p.eps for p in probs], perturb="eta",
                              eta0=e0)
    for p, yv, g in zip(probs, ys, got):
        solo = scg.scg_solve(yv, p.work.n, "S-CG", p.eps, perturb="eta", eta0=e0)
        assert g.iters == solo.iters and g.status == solo.status
        assert torch.equal(g.x, solo.x)


def test_eta_rule_parameters_validated():
    y = torch.zeros((4, 5), dtype=torch.float32, device=DEV)
    with pytest.raises(scg.ScgError):
        scg.scg_solve(y, 4, "S-CG", 1.0, perturb="eta", eta0=0.0)
