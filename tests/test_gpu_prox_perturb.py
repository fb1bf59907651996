"""The proximal perturbation on the device (SCG_PERTURB_PROX), through the C
ABI: x_{k+1/2} = prox_{lambda TV}(x_k) by prox_iters FGP steps, lambda =
gamma_0 a^l / ||dTV(x_k)|| (footnote to Eq. superiorized; the reading is the
oracle's, pinned in test_oracle_prox_perturb.py).

* Whole solves of every superiorized variant against the oracle's prox rule
  (FP64: same iterations, same l after every step, same lambda, x within
  1e-9; FP32: the same iterations, x within a bound ~3x the measured error).
* Where the rule is not built -- 16-bit storage, the batch -- the library
  refuses it, and it needs at least one FGP step.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_1709_04912_gb300 import inputs, scg

pytestmark = pytest.mark.gpu
DEV = "cuda:0"
S_VARIANTS = ["S-CG", "S-CG-CD", "S-CG-K", "S-PCG", "S-PCG-K"]
KW = dict(perturb="prox", gamma0_rel=0.05, prox_iters=20)
# trace columns: trials, accepted, l after the step, lambda
TRIALS, ACCEPTED, ELL, LAM = 4, 5, 6, 7


def rel(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


@pytest.fixture(scope="module", autouse=True)
def lib():
    assert torch.cuda.is_available()
    return scg.load()


@pytest.fixture(scope="module")
def small():
    return inputs.make_problem(inputs.SMALL_FP64, 0, oracle.project)


def gpu(prob, dtype, variant, **kw):
    y = torch.tensor(prob.y, dtype=dtype, device=DEV)
    return scg.scg_solve(y, prob.work.n, variant, prob.eps, trace=True, **kw)


@pytest.mark.parametrize("variant", S_VARIANTS)
def test_prox_rule_matches_the_oracle_fp64(small, variant):
    xo, ro, to = oracle.solve(small.y, small.work.n, variant=variant, eps=small.eps, **KW)
    r = gpu(small, torch.float64, variant, **KW)
    assert r.status == ro["status"] == "ok" and r.iters == ro["iters"] and r.ell == ro["ell"]
    np.testing.assert_array_equal(r.trace[:, [TRIALS, ACCEPTED, ELL]], to[:, [TRIALS, ACCEPTED, ELL]])
    assert np.all(to[1:, ACCEPTED] == 1) and r.ell >= r.iters - 1
    np.testing.assert_allclose(r.trace[:, LAM], to[:, LAM], rtol=1e-9)
    assert rel(r.x.cpu().numpy(), xo) <= 1e-9


@pytest.mark.parametrize("variant", ["S-CG", "S-PCG"])
def test_prox_rule_fp32(small, variant):
    xo, ro, _ = oracle.solve(small.y, small.work.n, variant=variant, eps=small.eps, **KW)
    r = gpu(small, torch.float32, variant, **KW)
    err = rel(r.x.cpu().numpy(), xo)
    print(f"prox rule {variant} FP32: iters {r.iters}/{ro['iters']} l {r.ell}/{ro['ell']} rel L2 {err:.2e}")
    assert r.status == "ok" and r.iters == ro["iters"] and r.ell == ro["ell"]
    assert err <= 5e-5


def test_prox_rule_refused_where_not_built(small):
    y16 = torch.tensor(small.y, dtype=torch.float16, device=DEV)
    with pytest.raises(scg.ScgError, match=r"-5"):
        scg.scg_solve(y16, small.work.n, "S-CG", small.eps, **KW)
    y = torch.tensor(small.y, dtype=torch.float32, device=DEV)
    with pytest.raises(scg.ScgError, match=r"-5"):
        scg.scg_solve_batch([y, y], [small.work.n] * 2, "S-CG", [small.eps] * 2, **KW)
    with pytest.raises(scg.ScgError):
        scg.scg_solve(y, small.work.n, "S-CG", small.eps, perturb="prox", prox_iters=0)
