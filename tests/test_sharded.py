"""The angle-sharded S-CG (paper_1709_04912_gb300/sharded.py) on CPU ranks: two
and three gloo processes (127.0.0.1), each holding one block of the angles and
its rows of the data, with the oracle's operators restricted to that block as
the local A_r and A_r^T.  Every rank must end with the single-process oracle
solve's result: the same iterations, perturbation decisions and l, and the
same x up to the rounding of summing backprojection shares in another order
(FP64, 1e-9), after exactly 3 (bodies + 1) all-reduces: the set-up and every
body exchange f (a scalar) and two images (g and h).  No GPU.
"""
import os
import socket
import sys

import numpy as np
import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

from paper_1709_04912_gb300.sharded import ShardedSCG, angle_blocks, torch_allreduce  # noqa: E402

WORK = dict(name="sh40", n=40, n_angles=45, n_bins=59, n_ellipses=6, noise_frac=0.01, eps_factor=1.05)


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def problem():
    import oracle
    from paper_1709_04912_gb300 import inputs
    return inputs.make_problem(inputs.Workload(**WORK), 4, oracle.project)


def local_ops(block, n, na, nb):
    import oracle
    a0, cnt = block

    def project_local(x):
        return oracle.project(x, na, nb)[a0:a0 + cnt]

    def backproject_local(r):
        full = np.zeros((na, nb))
        full[a0:a0 + cnt] = r
        return oracle.backproject(full, n)

    def tv_grad(x):
        t, g = oracle.tv_grad(x)
        return g, t

    return project_local, backproject_local, oracle.tv, tv_grad


def rank_main(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", init_method="env://", rank=rank, world_size=world)
    prob = problem()
    w = prob.work
    block = angle_blocks(w.n_angles, world)[rank]
    ops = local_ops(block, w.n, w.n_angles, w.n_bins)
    solver = ShardedSCG(*ops, allreduce=torch_allreduce)
    y_loc = prob.y[block[0]:block[0] + block[1]]
    r = solver.solve(y_loc, np.zeros((w.n, w.n)), prob.eps, gamma0_rel=0.05)
    q.put((rank, r.x, r.iters, r.status, r.ell, np.array(r.trace), r.exchanges, r.f_final, r.tv_final))
    dist.barrier()
    dist.destroy_process_group()


def test_angle_blocks_partition():
    for na in (1, 7, 90, 720):
        for world in (1, 2, 3, 8):
            bl = angle_blocks(na, world)
            assert len(bl) == world and bl[0][0] == 0
            assert sum(c for _, c in bl) == na
            assert all(bl[i][0] + bl[i][1] == bl[i + 1][0] for i in range(world - 1))
            assert max(c for _, c in bl) - min(c for _, c in bl) <= 1


def test_one_rank_equals_the_oracle():
    import oracle
    prob = problem()
    w = prob.work
    solver = ShardedSCG(*local_ops((0, w.n_angles), w.n, w.n_angles, w.n_bins), allreduce=lambda a: a)
    r = solver.solve(prob.y, np.zeros((w.n, w.n)), prob.eps, gamma0_rel=0.05)
    xo, ro, to = oracle.solve(prob.y, w.n, variant="S-CG", eps=prob.eps, gamma0_rel=0.05)
    assert r.status == ro["status"] == "ok" and r.iters == ro["iters"] and r.ell == ro["ell"]
    np.testing.assert_array_equal(np.array(r.trace)[:, [2, 3, 4]], to[:, [4, 5, 6]])
    assert np.linalg.norm(r.x - xo) / np.linalg.norm(xo) <= 1e-12


@pytest.mark.parametrize("world", [2, 3])
def test_gloo_ranks_equal_the_single_process_oracle(world):
    import oracle
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = free_port()
    procs = [ctx.Process(target=rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    got = sorted((q.get(timeout=300) for _ in procs), key=lambda t: t[0])
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    prob = problem()
    xo, ro, to = oracle.solve(prob.y, prob.work.n, variant="S-CG", eps=prob.eps, gamma0_rel=0.05)
    for rank, x, iters, status, ell, tr, exchanges, f, tv in got:
        assert status == ro["status"] == "ok" and iters == ro["iters"] and ell == ro["ell"]
        np.testing.assert_array_equal(tr[:, [2, 3, 4]], to[:, [4, 5, 6]])
        assert np.linalg.norm(x - xo) / np.linalg.norm(xo) <= 1e-9
        assert f == pytest.approx(ro["f_final"], rel=1e-9) and tv == pytest.approx(ro["tv_final"], rel=1e-9)
        # set-up: f + g0, h0 (3); each body: f + g', h' (3)
        assert exchanges == 3 * (iters + 1)
    # the ranks agree with each other bit for bit (replicated image-space work)
    for _, x, *_ in got[1:]:
        np.testing.assert_array_equal(x, got[0][1])
