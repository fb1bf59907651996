"""The local operators of an angle-sharded solve on the device
(scg_operator_create_angles) and the sharded S-CG driver running on them.

* A block's projection is exactly those rows of the whole scan's projection
  (every ray is computed alike, whatever block it falls in).
* The blocks' backprojection shares add up to the whole A^T r: to rounding of
  the order of the sums in FP64; in FP32 within the operator tolerance, since
  with 64 | N the whole scan takes the mirror-paired gather and an angle
  block the plain one (two roundings of the same weights, each within 3.3e-6
  of the oracle).
* The sharded driver on one rank with the device operators (FP64) reproduces
  scg_solve's S-CG: iterations, decisions, l, x within 1e-9.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_1709_04912_gb300 import inputs, scg
from paper_1709_04912_gb300.sharded import ShardedSCG, angle_blocks, device_operators

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def rel(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


@pytest.mark.parametrize("dtype,tol", [(torch.float32, 1e-5), (torch.float64, 1e-13)])
@pytest.mark.parametrize("n,na,nb,world", [(64, 90, 95, 2), (77, 33, 110, 3), (130, 181, 185, 4)])
def test_angle_block_operators(n, na, nb, world, dtype, tol):
    x = torch.tensor(inputs.ellipse_phantom(n, 8, n) + 0.1 * inputs.normal(n, "i", n * n).reshape(n, n),
                     dtype=dtype, device=DEV)
    r = torch.tensor(inputs.normal(na, "r", na * nb).reshape(na, nb), dtype=dtype, device=DEV)
    full = scg.Operator(n, na, nb, dtype, DEV)
    y_full = full.project(x)
    g_full = full.backproject(r)
    g_sum = torch.zeros_like(g_full)
    for a0, cnt in angle_blocks(na, world):
        op = scg.Operator(n, na, nb, dtype, DEV, angles=(a0, cnt))
        assert torch.equal(op.project(x), y_full[a0:a0 + cnt])
        g_sum += op.backproject(r[a0:a0 + cnt].contiguous())
        op.close()
    torch.cuda.synchronize()
    assert rel(g_sum.cpu().numpy(), g_full.cpu().numpy()) <= tol
    full.close()


def test_sharded_driver_on_device_operators_equals_scg_solve():
    prob = inputs.make_problem(inputs.SMALL_FP64, 0, oracle.project)
    w = prob.work
    y = torch.tensor(prob.y, dtype=torch.float64, device=DEV)
    ref = scg.scg_solve(y, w.n, "S-CG", prob.eps, gamma0_rel=0.05, trace=True)
    ops = device_operators(w.n, w.n_angles, w.n_bins, (0, w.n_angles), torch.float64, DEV)
    solver = ShardedSCG(*ops, allreduce=lambda a: a)
    r = solver.solve(y, torch.zeros((w.n, w.n), dtype=torch.float64, device=DEV), prob.eps, gamma0_rel=0.05)
    assert r.status == ref.status == "ok" and r.iters == ref.iters and r.ell == ref.ell
    np.testing.assert_array_equal(np.array(r.trace)[:, [2, 3, 4]], ref.trace[:, [4, 5, 6]])
    assert rel(r.x.cpu().numpy(), ref.x.cpu().numpy()) <= 1e-9
