"""Batched solves (scg_solve_batch) against solo solves, through the C ABI.

A batch advances problems of different sizes together, each with its own
state and stop test, so every problem's result must be the one scg_solve
gives for it alone, bit for bit: same output image, iteration count, status,
final f and TV, and perturbation count.  The mixes below put problems that
stop early beside ones that run long (different eps factors), include one
that stops at max_iter, and run two mixes in a row on one workspace so the
second reuses the first's captured loop.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_1709_04912_gb300 import inputs, scg

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def work(n, na, nb, ef, name):
    return inputs.Workload(name, n, na, nb, 6, 0.01, ef, 100)


MIX_A = [work(64, 90, 95, 1.05, "a0"), work(48, 60, 70, 1.3, "a1"), work(77, 33, 110, 1.02, "a2"),
         work(32, 45, 47, 1.5, "a3")]
MIX_B = [work(40, 50, 60, 1.1, "b0"), work(64, 90, 95, 1.05, "b1"), work(70, 40, 100, 1.2, "b2"),
         work(33, 45, 47, 1.05, "b3")]


@pytest.fixture(scope="module", autouse=True)
def lib():
    assert torch.cuda.is_available()
    return scg.load()


def problems(mix, seed):
    return [inputs.make_problem(w, seed + q, oracle.project) for q, w in enumerate(mix)]


def params_for(variant):
    kw = dict(gamma0_rel=0.05, max_iter=60)
    if variant in ("CG", "PCG"):
        kw["perturb"] = "none"
    return kw


def same(a, b):
    assert a.status_code == b.status_code
    assert a.iters == b.iters and a.k_final == b.k_final and a.ell == b.ell
    assert a.f_final == b.f_final and a.tv_final == b.tv_final
    assert torch.equal(a.x, b.x)


@pytest.mark.parametrize("dtype", [torch.float32, torch.float64])
@pytest.mark.parametrize("variant", ["CG", "PCG", "S-CG", "S-CG-CD", "S-CG-K", "S-PCG", "S-PCG-K"])
def test_batch_equals_solo_bitwise(variant, dtype):
    probs = problems(MIX_A, 10)
    ys = [torch.tensor(p.y, dtype=dtype, device=DEV) for p in probs]
    kw = params_for(variant)
    got = scg.scg_solve_batch(ys, [p.work.n for p in probs], variant, [p.eps for p in probs], **kw)
    iters = []
    for p, y, g in zip(probs, ys, got):
        solo = scg.scg_solve(y, p.work.n, variant, p.eps, **kw)
        same(g, solo)
        iters.append(g.iters)
        assert g.device_loop == 1
    # the loop ran as long as its slowest problem
    assert got[0].body_launches >= max(iters)


def test_two_mixes_reuse_one_workspace():
    # the second mix has other geometries but the same rounded sizes: the
    # captured loop is reused and must still give each problem its solo result
    dtype = torch.float32
    w = None
    for mix, seed in ((MIX_A, 20), (MIX_B, 30), (MIX_A, 40)):
        probs = problems(mix, seed)
        ys = [torch.tensor(p.y, dtype=dtype, device=DEV) for p in probs]
        ns = [p.work.n for p in probs]
        nbytes = scg.batch_workspace_bytes([(p.work.n, p.work.n_angles, p.work.n_bins) for p in probs],
                                           "S-CG", dtype)
        if w is None or w.numel() < nbytes:
            w = torch.empty(2 * nbytes, dtype=torch.uint8, device=DEV)
        got = scg.scg_solve_batch(ys, ns, "S-CG", [p.eps for p in probs], work=w, gamma0_rel=0.05)
        for p, y, g in zip(probs, ys, got):
            same(g, scg.scg_solve(y, p.work.n, "S-CG", p.eps, gamma0_rel=0.05))


def test_batch_with_x0_and_max_iter_stop():
    dtype = torch.float64
    probs = problems(MIX_A[:3], 50)
    ys = [torch.tensor(p.y, dtype=dtype, device=DEV) for p in probs]
    ns = [p.work.n for p in probs]
    x0s = [torch.tensor(0.01 * inputs.normal(q, "x0", n * n).reshape(n, n), dtype=dtype, device=DEV)
           for q, n in enumerate(ns)]
    eps = [probs[0].eps, probs[1].eps * 1e-6, probs[2].eps]     # the middle one cannot stop
    got = scg.scg_solve_batch(ys, ns, "S-CG-K", eps, x0s=x0s, gamma0_rel=0.05, max_iter=12)
    assert got[1].status == "max_iter" and got[1].iters == 12
    for q in range(3):
        solo = scg.scg_solve(ys[q], ns[q], "S-CG-K", eps[q], x0=x0s[q], gamma0_rel=0.05, max_iter=12)
        same(got[q], solo)


def test_batch_of_one_and_already_converged():
    dtype = torch.float32
    p = problems(MIX_A[:1], 60)[0]
    y = torch.tensor(p.y, dtype=dtype, device=DEV)
    for eps in (p.eps, 1e30):                    # 1e30: f(x0) <= eps, no iteration
        (g,) = scg.scg_solve_batch([y], [p.work.n], "S-PCG", eps, gamma0_rel=0.05)
        same(g, scg.scg_solve(y, p.work.n, "S-PCG", eps, gamma0_rel=0.05))
    assert g.iters == 0


def test_full_size_batch_of_uneven_problems():
    # four problems of the uneven batch recipe (N up to 768): each within its
    # eps (checked with the oracle's A) and equal to its solo solve
    ws = inputs.batch_workloads(4, 3)
    probs = [inputs.make_problem(w, 70 + q, oracle.project) for q, w in enumerate(ws)]
    ys = [torch.tensor(p.y, dtype=torch.float32, device=DEV) for p in probs]
    ns = [p.work.n for p in probs]
    got = scg.scg_solve_batch(ys, ns, "S-CG", [p.eps for p in probs], gamma0_rel=0.05, max_iter=100)
    for p, y, g in zip(probs, ys, got):
        assert g.status == "ok"
        r = oracle.project(g.x.double().cpu().numpy(), p.work.n_angles, p.work.n_bins) - p.y
        assert 0.5 * float(np.sum(r * r)) <= p.eps * (1 + 1e-4)
        same(g, scg.scg_solve(y, p.work.n, "S-CG", p.eps, gamma0_rel=0.05, max_iter=100))


def rel(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


@pytest.mark.parametrize("variant", ["CG", "PCG", "S-CG", "S-CG-CD", "S-CG-K", "S-PCG", "S-PCG-K"])
def test_batch_members_match_the_oracle(variant):
    # every member of an FP64 batch against the oracle's solve of that problem
    # alone: same status, iteration count, perturbation index l, output within
    # 1e-9 relative L2 (the FP64 single-solve bar)
    probs = problems(MIX_A + MIX_B[:2], 80)
    ys = [torch.tensor(p.y, dtype=torch.float64, device=DEV) for p in probs]
    kw = params_for(variant)
    got = scg.scg_solve_batch(ys, [p.work.n for p in probs], variant, [p.eps for p in probs], **kw)
    for p, g in zip(probs, got):
        xo, ro, to = oracle.solve(p.y, p.work.n, variant=variant, eps=p.eps, **kw)
        assert g.status == ro["status"] and g.iters == ro["iters"] and g.ell == ro["ell"], p.work.name
        assert rel(g.x.cpu().numpy(), xo) <= 1e-9, p.work.name
        assert g.tv_final == pytest.approx(ro["tv_final"], rel=1e-9)
        assert g.f_final == pytest.approx(ro["f_final"], rel=1e-9)
