"""The prepared operator pair (scg_operator_*): same values as the one-shot
entry points, repeated applications, and capture in a CUDA graph."""
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


@pytest.mark.parametrize("dtype", [torch.float32, torch.float64, torch.float16, torch.bfloat16])
@pytest.mark.parametrize("n,na,nb", [(64, 90, 95), (77, 33, 110), (130, 181, 185)])
def test_operator_equals_one_shot_entry_points(n, na, nb, dtype):
    op = scg.Operator(n, na, nb, dtype)
    for seed in range(2):                       # repeated applications on one workspace
        x = torch.tensor(inputs.normal(seed, "x", n * n).reshape(n, n), dtype=torch.float32).to(dtype).to(DEV)
        r = torch.tensor(inputs.normal(seed, "r", na * nb).reshape(na, nb), dtype=torch.float32).to(dtype).to(DEV)
        assert torch.equal(op.project(x), scg.scg_project(x, na, nb))
        assert torch.equal(op.backproject(r), scg.scg_backproject(r, n))
    op.close()


def test_operator_in_a_cuda_graph():
    n, na, nb = 96, 120, 137
    op = scg.Operator(n, na, nb, torch.float32)
    x = torch.tensor(inputs.ellipse_phantom(n, 6, 1), dtype=torch.float32, device=DEV)
    y = torch.empty((na, nb), dtype=torch.float32, device=DEV)
    z = torch.empty((n, n), dtype=torch.float32, device=DEV)
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):                  # warm up off the default stream before capture
        op.project(x, y)
        op.backproject(y, z)
    torch.cuda.current_stream().wait_stream(s)
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        op.project(x, y)
        op.backproject(y, z)                    # A^T A x
    x.copy_(torch.tensor(inputs.ellipse_phantom(n, 6, 2), dtype=torch.float32, device=DEV))
    graph.replay()
    torch.cuda.synchronize()
    ref = oracle.backproject(oracle.project(x.double().cpu().numpy(), na, nb), n)
    got = z.double().cpu().numpy()
    assert np.linalg.norm(got - ref) <= 1e-5 * np.linalg.norm(ref)
    op.close()


def test_release_then_solve_again_gives_the_same_result():
    prob = inputs.make_problem(inputs.SMALL_FP64, 0, oracle.project)
    y = torch.tensor(prob.y, dtype=torch.float32, device=DEV)
    a = scg.scg_solve(y, prob.work.n, "S-CG", prob.eps, gamma0_rel=0.05)
    scg.release()
    b = scg.scg_solve(y, prob.work.n, "S-CG", prob.eps, gamma0_rel=0.05)
    assert a.iters == b.iters and torch.equal(a.x, b.x)


def test_projector_output_does_not_depend_on_the_tuned_shape():
    # a solve tunes the projector shape of this geometry bucket; a prepared
    # operator then uses the tuned shape while scg_project keeps the default
    # one: every ray is computed identically, so the sinograms are equal
    prob = inputs.make_problem(inputs.SMALL_FP64, 3, oracle.project)
    n, na, nb = prob.work.n, prob.work.n_angles, prob.work.n_bins
    y = torch.tensor(prob.y, dtype=torch.float32, device=DEV)
    scg.scg_solve(y, n, "S-CG", prob.eps, gamma0_rel=0.05, max_iter=2)
    op = scg.Operator(n, na, nb, torch.float32)
    x = torch.tensor(inputs.normal(5, "x", n * n).reshape(n, n), dtype=torch.float32, device=DEV)
    assert torch.equal(op.project(x), scg.scg_project(x, na, nb))
    op.close()


def test_operator_kernel_times_are_recorded():
    # scg_operator_kernel_ms: the projector's and the gather's own device time
    # from events the library records around the kernel alone, once timing is
    # on; untimed applications and calls captured into a graph record none
    n, na, nb = 128, 90, 183
    op = scg.Operator(n, na, nb, torch.float32, DEV)
    x = torch.rand((n, n), device=DEV)
    y = op.project(x)
    op.backproject(y)
    assert op.kernel_ms() == (None, None)
    op.set_timing(True)
    y = op.project(x)
    tp, tb = op.kernel_ms()
    assert tp is not None and tp > 0.0 and tb is None
    op.backproject(y)
    tp2, tb2 = op.kernel_ms()
    assert tp2 == tp and tb2 is not None and tb2 > 0.0
    op.set_timing(False)
    op.project(x)
    assert op.kernel_ms() == (tp, tb2)          # the last timed calls' values
    op.close()
