"""A device-side wait that runs out is reported, not faulted.

The gather waits on an mbarrier for its TMA copies, with a time limit.  The
host-side test hook scg_test_stall_copies makes every copy 16 bytes shorter
than the barriers expect: every copy still completes, but each wait runs out.  The solve (and the batch) must then return SCG_ERR_CUDA, the
device loop must stop at its next test instead of running to max_iter, and the
context must stay usable: the next solve, with the hook cleared, gives the
same result as before, bit for bit.
"""
import time

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


# 64 x 64 takes the gather's mirror-paired path (slots of an angle and its
# mirror, eight a chunk): 90 angles give each gather block two chunks of bands,
# 360 angles six, so after the first wait runs out one more chunk is in flight
# (waited for, with its limit) and the rest are never issued; 77 x 77 takes the
# plain path (32 angles a chunk: one chunk per block at 90 angles)
WORKLOADS = {"a90": inputs.SMALL_FP64, "a360": inputs.Workload("ellipse64_a360_b95", 64, 360, 95, 6, 0.01, 1.05, 100),
             "n77": inputs.Workload("ellipse77_a90_b110", 77, 90, 110, 6, 0.01, 1.05, 100)}


def make(name):
    prob = inputs.make_problem(WORKLOADS[name], 0, oracle.project)
    return prob, torch.tensor(prob.y, dtype=torch.float32, device=DEV)


@pytest.fixture
def problem():
    return make("a90")


@pytest.mark.parametrize("dtype,name", [(torch.float32, "a90"), (torch.float16, "a90"), (torch.float32, "a360"),
                                        (torch.float32, "n77")])
def test_solve_reports_a_wait_that_ran_out(dtype, name):
    prob, y = make(name)
    y = y.to(dtype)
    n = prob.work.n
    good = scg.scg_solve(y, n, "S-CG", prob.eps, gamma0_rel=0.05)
    assert good.status_code >= 0
    scg.set_copy_stall(True)
    try:
        t0 = time.time()
        with pytest.raises(scg.ScgError, match=r"failed: -2"):
            scg.scg_solve(y, n, "S-CG", prob.eps, gamma0_rel=0.05)
        # the init's gathers time out once per chunk (about 0.13 s each); the
        # loop stops at its first test rather than running max_iter bodies
        assert time.time() - t0 < 30.0
    finally:
        scg.set_copy_stall(False)
    torch.cuda.synchronize()                      # the context still answers
    again = scg.scg_solve(y, n, "S-CG", prob.eps, gamma0_rel=0.05)
    assert again.status_code == good.status_code and again.iters == good.iters and torch.equal(again.x, good.x)


def test_batch_reports_a_wait_that_ran_out(problem):
    prob, y = problem
    n = prob.work.n
    y2 = y.clone()
    eps = [prob.eps, 1.5 * prob.eps]
    good = scg.scg_solve_batch([y, y2], [n, n], "S-CG", eps, gamma0_rel=0.05)
    scg.set_copy_stall(True)
    try:
        with pytest.raises(scg.ScgError, match=r"failed: -2"):
            scg.scg_solve_batch([y, y2], [n, n], "S-CG", eps, gamma0_rel=0.05)
    finally:
        scg.set_copy_stall(False)
    again = scg.scg_solve_batch([y, y2], [n, n], "S-CG", eps, gamma0_rel=0.05)
    for a, b in zip(good, again):
        assert a.status_code == b.status_code and a.iters == b.iters and torch.equal(a.x, b.x)
