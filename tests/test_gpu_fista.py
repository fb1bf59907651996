"""FISTA with the TV prox on the device (SCG_FISTA: Sec. 2, Eqs. FISTA, FISTA-u,
the comparison method of Sec. 4) against the oracle's FISTA, through the C ABI.

* FP64: the same iteration count and status, x within 1e-9, the momentum
  sequence t_k and (t_k - 1)/t_{k+1} and f(x_k) per iteration as the oracle's.
* FP32: the same iteration count, x within ~3x the measured error.
* c^2 = ||A||_2^2 estimated on the device (100 power iterations from the same
  start vector as the oracle's) equals the oracle's estimate.
* lambda = 0 (no prox: accelerated gradient on f), f(x0) <= eps, max_iter.
* scg_solve_batch and the server refuse FISTA.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_1709_04912_gb300 import inputs, scg

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def rel(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


@pytest.fixture(scope="module")
def small():
    p = inputs.make_problem(inputs.SMALL_FP64, 0, oracle.project)
    c = oracle.norm_A(p.work.n, p.work.n_angles, p.work.n_bins, 100)
    return p, c * c


def gpu_fista(p, dtype, lam, c2, prox_iters=10, max_iter=300, eps=None, x0=None):
    y = torch.tensor(p.y, dtype=dtype, device=DEV)
    if x0 is not None:
        x0 = torch.tensor(x0, dtype=dtype, device=DEV)
    return scg.scg_solve(y, p.work.n, "FISTA", p.eps if eps is None else eps, x0=x0, trace=True,
                         lambda_=lam, lipschitz=c2, prox_iters=prox_iters, max_iter=max_iter)


@pytest.mark.parametrize("lam,prox_iters", [(1.0, 10), (5.0, 10), (5.0, 1), (2.0, 25)])
def test_fista_fp64_equals_the_oracle(small, lam, prox_iters):
    p, c2 = small
    xo, ro, to = oracle.fista(p.y, p.work.n, p.eps, lam, c2, prox_iters=prox_iters, max_iter=300)
    r = gpu_fista(p, torch.float64, lam, c2, prox_iters)
    assert r.status == ro["status"] and r.iters == ro["iters"]
    assert rel(r.x.cpu().numpy(), xo) <= 1e-9
    assert r.f_final == pytest.approx(ro["f_final"], rel=1e-9)
    assert r.tv_final == pytest.approx(ro["tv_final"], rel=1e-9)
    np.testing.assert_allclose(r.trace[:, 8:10], to[:, 8:10], rtol=1e-12)   # t_k, beta_k
    assert r.lipschitz_used == c2


@pytest.mark.parametrize("lam", [1.0, 5.0])
def test_fista_fp32(small, lam):
    p, c2 = small
    xo, ro, _ = oracle.fista(p.y, p.work.n, p.eps, lam, c2, prox_iters=10, max_iter=300)
    r = gpu_fista(p, torch.float32, lam, c2)
    err = rel(r.x.cpu().numpy(), xo)
    print(f"FISTA FP32 lambda {lam}: iters {r.iters}/{ro['iters']} rel L2 {err:.2e}")
    assert r.status == ro["status"] == "ok" and r.iters == ro["iters"]
    assert err <= 2e-5
    assert r.f_final <= p.eps


@pytest.mark.parametrize("dtype,tol", [(torch.float64, 1e-9), (torch.float32, 1e-5)])
def test_device_power_iteration_matches_the_oracle(small, dtype, tol):
    p, c2 = small
    scg.release()
    r = scg.scg_solve(torch.tensor(p.y, dtype=dtype, device=DEV), p.work.n, "FISTA", p.eps, lambda_=1.0,
                      prox_iters=10, max_iter=300)
    assert r.lipschitz_used == pytest.approx(c2, rel=tol)
    assert r.status == "ok"


def test_fista_without_prox_and_edge_cases(small):
    p, c2 = small
    xo, ro, _ = oracle.fista(p.y, p.work.n, p.eps, 0.0, c2, prox_iters=10, max_iter=300)
    r = gpu_fista(p, torch.float64, 0.0, c2)
    assert r.iters == ro["iters"] and rel(r.x.cpu().numpy(), xo) <= 1e-9
    r = gpu_fista(p, torch.float64, 1.0, c2, eps=1e30)               # f(x0) <= eps: no iteration
    assert r.iters == 0 and r.status == "ok" and float(r.x.abs().max()) == 0.0
    x0 = 0.5 * p.x_true
    xo, ro, _ = oracle.fista(p.y, p.work.n, p.eps * 1e-3, 2.0, c2, prox_iters=5, max_iter=7, x0=x0)
    r = gpu_fista(p, torch.float64, 2.0, c2, prox_iters=5, max_iter=7, eps=p.eps * 1e-3, x0=x0)
    assert r.status == ro["status"] == "max_iter" and r.iters == 7
    assert rel(r.x.cpu().numpy(), xo) <= 1e-9


def test_batch_and_server_refuse_fista(small):
    p, c2 = small
    y = torch.tensor(p.y, dtype=torch.float32, device=DEV)
    with pytest.raises(scg.ScgError):
        scg.scg_solve_batch([y], [p.work.n], "FISTA", p.eps, lambda_=1.0, lipschitz=c2)
    with pytest.raises(scg.ScgError):
        scg.Server("FISTA", torch.float32, pool_bytes=64 << 20, lambda_=1.0, lipschitz=c2)
