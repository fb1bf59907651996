"""The continuous-batching server (scg_server_*) against solo solves.

Requests of different sizes, angle counts and eps join while others are
resident on the device, wait for pool memory or a slot when there is none,
and leave when they stop.  Every completion must equal scg_solve of the same
request alone, bit for bit (output image, iterations, status, final f and
TV, perturbation count): the work items keep each request's single-solve
block order, so being in a mix changes no rounding.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_1709_04912_gb300 import inputs, scg

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


@pytest.fixture(scope="module", autouse=True)
def lib():
    assert torch.cuda.is_available()
    return scg.load()


def work(n, na, nb, ef, name):
    return inputs.Workload(name, n, na, nb, 6, 0.01, ef, 100)


STREAM = [work(64, 90, 95, 1.05, "r0"), work(48, 60, 70, 1.3, "r1"), work(77, 33, 110, 1.02, "r2"),
          work(32, 45, 47, 1.5, "r3"), work(96, 30, 136, 1.1, "r4"), work(40, 50, 60, 1.2, "r5"),
          work(64, 120, 91, 1.02, "r6")]


@pytest.fixture(scope="module")
def requests():
    return [inputs.make_problem(w, 100 + q, oracle.project) for q, w in enumerate(STREAM)]


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


def serve(srv, probs, ys, waves, max_steps=2000):
    """Submit the requests in waves (one wave before each of the first
    len(waves) steps) and step until every request has completed."""
    done = {}
    tags = {}
    steps = 0
    while len(done) < len(probs):
        if steps < len(waves):
            for q in waves[steps]:
                tags[srv.submit(ys[q], probs[q].work.n, probs[q].eps)] = q
        for tag, r in srv.step():
            done[tags[tag]] = r
        queued, active = srv.pending()
        steps += 1
        assert steps < max_steps
    return done


@pytest.mark.parametrize("variant", ["CG", "PCG", "S-CG", "S-CG-CD", "S-CG-K", "S-PCG", "S-PCG-K"])
def test_served_results_equal_solo(requests, variant):
    dtype = torch.float32
    ys = [torch.tensor(p.y, dtype=dtype, device=DEV) for p in requests]
    kw = params_for(variant)
    srv = scg.Server(variant, dtype, pool_bytes=256 << 20, max_active=8, **kw)
    # requests arrive in three waves while earlier ones are running
    done = serve(srv, requests, ys, [[0, 1, 2], [], [3, 4], [5], [], [6]])
    srv.close()
    for q, p in enumerate(requests):
        same(done[q], scg.scg_solve(ys[q], p.work.n, variant, p.eps, **kw))


def test_admission_waits_for_pool_memory(requests):
    dtype = torch.float64
    ys = [torch.tensor(p.y, dtype=dtype, device=DEV) for p in requests]
    fp = max(scg.server_footprint(p.work.n, p.work.n_angles, p.work.n_bins, "S-CG", dtype) for p in requests)
    # room for two of the largest resident requests (plus descriptors and lists):
    # well below the seven requests' total, so some must wait for memory
    srv = scg.Server("S-CG", dtype, pool_bytes=2 * fp + (256 << 10), max_active=8, gamma0_rel=0.05)
    for q, p in enumerate(requests):
        srv.submit(ys[q], p.work.n, p.eps, tag=q)
    done = {}
    peak = 0
    for _ in range(2000):
        for tag, r in srv.step():
            done[tag] = r
        queued, active = srv.pending()
        peak = max(peak, active)
        if len(done) == len(requests):
            break
    srv.close()
    assert len(done) == len(requests) and 2 <= peak < len(requests)
    for q, p in enumerate(requests):
        same(done[q], scg.scg_solve(ys[q], p.work.n, "S-CG", p.eps, gamma0_rel=0.05))


@pytest.mark.parametrize("max_active,bodies", [(1, 1), (3, 4)])
def test_slots_and_bodies_per_step(requests, max_active, bodies):
    dtype = torch.float32
    ys = [torch.tensor(p.y, dtype=dtype, device=DEV) for p in requests]
    srv = scg.Server("S-CG-K", dtype, pool_bytes=256 << 20, max_active=max_active, bodies_per_step=bodies,
                     gamma0_rel=0.05, max_iter=40)
    done = serve(srv, requests, ys, [list(range(len(requests)))])
    srv.close()
    for q, p in enumerate(requests):
        same(done[q], scg.scg_solve(ys[q], p.work.n, "S-CG-K", p.eps, gamma0_rel=0.05, max_iter=40))


def test_request_stopping_at_max_iter_and_at_x0(requests):
    dtype = torch.float32
    ys = [torch.tensor(p.y, dtype=dtype, device=DEV) for p in requests[:3]]
    eps = [requests[0].eps * 1e-6, 1e30, requests[2].eps]      # cannot stop / stops at x0 / normal
    srv = scg.Server("S-CG", dtype, pool_bytes=128 << 20, max_active=4, gamma0_rel=0.05, max_iter=10)
    tags = [srv.submit(ys[q], requests[q].work.n, eps[q]) for q in range(3)]
    done = {}
    for _ in range(100):
        for tag, r in srv.step():
            done[tag] = r
        if len(done) == 3:
            break
    srv.close()
    assert done[tags[0]].status == "max_iter" and done[tags[1]].iters == 0
    for q in range(3):
        same(done[tags[q]], scg.scg_solve(ys[q], requests[q].work.n, "S-CG", eps[q], gamma0_rel=0.05, max_iter=10))


def test_serving_workload_sizes_in_binary16():
    # requests drawn from the serving recipe (N up to 1024, 30..180 angles,
    # eps factor 1.02..1.2): each served result equals its solo FP16 solve and
    # meets its eps under the oracle's A
    ws = inputs.serving_workloads(5, 11)
    probs = [inputs.make_problem(w, 300 + q, oracle.project) for q, w in enumerate(ws)]
    ys = [torch.tensor(p.y, dtype=torch.float32).to(torch.float16).to(DEV) for p in probs]
    srv = scg.Server("S-CG", torch.float16, pool_bytes=1 << 30, max_active=8, gamma0_rel=0.05)
    done = serve(srv, probs, ys, [[0, 1], [2], [3, 4]])
    srv.close()
    for q, p in enumerate(probs):
        solo = scg.scg_solve(ys[q], p.work.n, "S-CG", p.eps, gamma0_rel=0.05)
        same(done[q], solo)
        assert done[q].status == "ok"
        yq = ys[q].double().cpu().numpy()
        r = oracle.project(done[q].x.double().cpu().numpy(), p.work.n_angles, p.work.n_bins) - yq
        assert 0.5 * float(np.sum(r * r)) <= p.eps * (1 + 1e-3)


def rel(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


@pytest.mark.parametrize("variant", ["CG", "S-CG", "S-CG-CD", "S-PCG-K"])
def test_served_results_match_the_oracle(requests, variant):
    # an FP64 server: every completion against the oracle's solve of that
    # request alone (status, iterations, l, output within 1e-9 relative L2)
    ys = [torch.tensor(p.y, dtype=torch.float64, device=DEV) for p in requests]
    kw = params_for(variant)
    srv = scg.Server(variant, torch.float64, pool_bytes=256 << 20, max_active=4, **kw)
    done = serve(srv, requests, ys, [[0, 1, 2], [3], [4, 5], [], [6]])
    srv.close()
    for q, p in enumerate(requests):
        xo, ro, _ = oracle.solve(p.y, p.work.n, variant=variant, eps=p.eps, **kw)
        g = done[q]
        assert g.status == ro["status"] and g.iters == ro["iters"] and g.ell == ro["ell"], p.work.name
        assert rel(g.x.cpu().numpy(), xo) <= 1e-9, p.work.name
        assert g.tv_final == pytest.approx(ro["tv_final"], rel=1e-9)
