"""GPU <-> oracle parity of the operators, through the C ABI.

A (ray-driven projector), A^T (pixel-driven backprojector), TV, its
subgradient and the preconditioner's row filter, on seeded inputs.  Small
cases (several tiles plus ragged tails, axis-aligned and diagonal angles, odd
and even sizes) are compared element by element; the full-size workloads are
compared on sampled rays/pixels that the oracle evaluates one by one.  The
gather's mirror-paired path (64 | N) has its own cases: single and unpaired
angles, odd counts, narrow and wide detectors, 16-bit storage, and a
weight-by-weight comparison with the projector.

Tolerances: relative L2 <= 1e-5 for FP32 (FP32 geometry and accumulation over
at most ~2N weights per ray; the measured error is ~1e-7), <= 1e-12 for FP64.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_1709_04912_gb300 import inputs, scg

pytestmark = pytest.mark.gpu

DEV = "cuda:0"
TOL = {torch.float32: 1e-5, torch.float64: 1e-12}

CASES = [
    (64, 90, 95),       # the FP64 workload's shape
    (77, 33, 110),      # ragged tiles (N % 32, N % 8 != 0), bins % 128 != 0
    (130, 181, 185),    # several tiles and ray blocks, odd angle count
    (33, 4, 47),        # angles 0, 45, 90, 135 degrees only
    (40, 1, 57),        # a single angle (theta = 0: every ray on pixel edges)
    (2, 3, 3),          # smallest image
    (16, 7, 1),         # a single detector bin
]


def rel(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def image(n, seed):
    x = inputs.ellipse_phantom(n, 8, seed)
    return x + 0.1 * inputs.normal(seed, "img", n * n).reshape(n, n)


@pytest.fixture(scope="module", autouse=True)
def lib():
    assert torch.cuda.is_available()
    return scg.load()


@pytest.mark.parametrize("dtype", [torch.float32, torch.float64])
@pytest.mark.parametrize("n,na,nb", CASES)
def test_project_matches_oracle(n, na, nb, dtype):
    x = image(n, n + na)
    ref = oracle.project(x, na, nb)
    got = scg.scg_project(torch.tensor(x, dtype=dtype, device=DEV), na, nb).cpu().numpy()
    assert rel(got, ref) <= TOL[dtype]


@pytest.mark.parametrize("dtype", [torch.float32, torch.float64])
@pytest.mark.parametrize("n,na,nb", CASES)
def test_backproject_matches_oracle(n, na, nb, dtype):
    r = inputs.normal(7 * n + na, "sino", na * nb).reshape(na, nb)
    ref = oracle.backproject(r, n)
    got = scg.scg_backproject(torch.tensor(r, dtype=dtype, device=DEV), n).cpu().numpy()
    assert rel(got, ref) <= TOL[dtype]


@pytest.mark.parametrize("n,na,nb", [(256, 360, 363), (300, 257, 190)])
def test_project_random_sign_image(n, na, nb):
    # zero-mean input: every ray sum cancels, exposing geometric rounding
    # (including rays that miss part of the image: 190 bins < sqrt(2) * 300)
    x = inputs.normal(n, "zm", n * n).reshape(n, n)
    ref = oracle.project(x, na, nb)
    got = scg.scg_project(torch.tensor(x, dtype=torch.float32, device=DEV), na, nb).cpu().numpy()
    assert rel(got, ref) <= 1e-5


@pytest.mark.parametrize("n,na,nb", [(64, 90, 95), (130, 181, 185)])
def test_pair_is_adjoint_in_fp32(n, na, nb):
    x = torch.tensor(image(n, 3), dtype=torch.float32, device=DEV)
    r = torch.tensor(inputs.normal(9, "r", na * nb).reshape(na, nb), dtype=torch.float32, device=DEV)
    ax = scg.scg_project(x, na, nb).double()
    atr = scg.scg_backproject(r, n).double()
    lhs = float((ax * r.double()).sum())
    rhs = float((x.double() * atr).sum())
    # <Ax, r> cancels heavily for random r; the FP32 bound scales with the norms
    assert abs(lhs - rhs) <= 1e-6 * float(ax.norm()) * float(r.double().norm())


def test_pair_is_matched_weight_by_weight():
    # dense A from unit images and dense A^T from unit sinograms, both in FP32:
    # the backprojector gathers the projector's weights (same chord lengths,
    # evaluated by different FP32 expressions), so A^T is A's transpose to
    # rounding, with no weight missing on either side
    n, na, nb = 8, 12, 12
    A = np.zeros((na * nb, n * n))
    for q in range(n * n):
        e = torch.zeros(n * n, dtype=torch.float32, device=DEV)
        e[q] = 1
        A[:, q] = scg.scg_project(e.view(n, n), na, nb).cpu().numpy().ravel()
    AT = np.zeros((n * n, na * nb))
    for q in range(na * nb):
        e = torch.zeros(na * nb, dtype=torch.float32, device=DEV)
        e[q] = 1
        AT[:, q] = scg.scg_backproject(e.view(na, nb), n).cpu().numpy().ravel()
    scale = np.max(np.abs(A))
    assert np.max(np.abs(A - AT.T)) <= 1e-5 * scale
    # a weight present on one side only is a rounding-level sliver of a chord
    one_sided = (A != 0) != (AT.T != 0)
    assert np.all(np.abs(A - AT.T)[one_sided] <= 1e-5 * scale)


@pytest.mark.parametrize("dtype", [torch.float32, torch.float64])
@pytest.mark.parametrize("n", [2, 7, 64, 77, 130])
def test_tv_and_subgradient_match_oracle(n, dtype):
    x = image(n, n)
    tv_ref, g_ref = oracle.tv_grad(x)
    xt = torch.tensor(x, dtype=dtype, device=DEV)
    grad, tv = scg.scg_tv_grad(xt)
    tv_only = float(scg.scg_tv(xt))
    tol = 1e-6 if dtype == torch.float32 else 1e-12
    assert abs(float(tv) - tv_ref) <= tol * max(tv_ref, 1e-12)
    assert tv_only == float(tv)
    assert rel(grad.cpu().numpy(), g_ref) <= (1e-5 if dtype == torch.float32 else 1e-12)


def test_tv_of_constant_is_zero_on_device():
    grad, tv = scg.scg_tv_grad(torch.full((50, 50), 2.5, device=DEV))
    assert float(tv) == 0.0 and float(grad.abs().max()) == 0.0


@pytest.mark.parametrize("dtype", [torch.float32, torch.float64])
@pytest.mark.parametrize("na,nb,mu,gain", [(5, 95, 0.0, 1.0), (3, 130, 0.02, 2.0), (2, 725, 0.0, 1.0),
                                           (1, 1, 0.0, 1.0), (4, 2, 0.1, 0.5), (7, 1449, 0.0, 1.0),
                                           (3, 4096, 0.0, 1.0)])
def test_filter_matches_oracle(na, nb, mu, gain, dtype):
    # the FFT of two rows at a time: odd row counts leave a block with one row;
    # P from 2 (one bin) to 8192
    r = inputs.normal(nb, "f", na * nb).reshape(na, nb)
    ref = oracle.filter_rows(r, mu, gain)
    got = scg.scg_filter(torch.tensor(r, dtype=dtype, device=DEV), mu, gain).cpu().numpy()
    assert rel(got, ref) <= (1e-5 if dtype == torch.float32 else 1e-11)


def test_filter_at_the_fp32_length_limit():
    # n_bins = 8192: P = 16384, the largest padded row pair the FP32 kernel
    # holds in shared memory (128 KiB); checked on rows the naive DFT of the
    # oracle evaluates in seconds
    na, nb = 2, 8192
    r = inputs.normal(9, "f", na * nb).reshape(na, nb)
    got = scg.scg_filter(torch.tensor(r, dtype=torch.float32, device=DEV)).cpu().numpy()
    assert rel(got, oracle.filter_rows(r)) <= 1e-5


# Geometries of the gather's mirror-paired path (64 | N, FP32 arithmetic): one
# angle (slot 0 alone), two (0 and the self-mirrored pi/2: no pair), an odd count
# (pairs and angle 0), the batch's and server's sizes, a detector narrower than
# the image (rays and bands beyond it), and a band reaching past both ends.
MIRROR_CASES = [
    (64, 1, 91),
    (64, 2, 91),
    (64, 7, 91),
    (128, 33, 182),
    (192, 120, 272),
    (64, 90, 20),
    (256, 61, 400),
]


@pytest.mark.parametrize("n,na,nb", MIRROR_CASES)
def test_mirror_gather_matches_oracle(n, na, nb):
    r = inputs.normal(5 * n + na, "msino", na * nb).reshape(na, nb)
    ref = oracle.backproject(r, n)
    got = scg.scg_backproject(torch.tensor(r, dtype=torch.float32, device=DEV), n).cpu().numpy()
    assert rel(got, ref) <= 1e-5
    # and the pixels of each half: the mirror images of the left half's pixels
    # are gathered from the other rows of each angle pair
    assert rel(got[:, n // 2:], ref[:, n // 2:]) <= 1e-5
    assert rel(got[:, :n // 2], ref[:, :n // 2]) <= 1e-5


@pytest.mark.parametrize("dtype,tol", [(torch.float16, 2e-3), (torch.bfloat16, 1.5e-2)])
@pytest.mark.parametrize("n,na,nb", [(64, 7, 91), (128, 33, 182)])
def test_mirror_gather_reduced_storage(n, na, nb, dtype, tol):
    # 16-bit storage: the sinogram rounded to the format, the gather in FP32
    r = inputs.normal(3 * n + na, "msino16", na * nb).reshape(na, nb)
    rq = torch.tensor(r, dtype=torch.float32).to(dtype)
    ref = oracle.backproject(rq.double().numpy(), n)
    got = scg.scg_backproject(rq.to(DEV), n).double().cpu().numpy()
    assert rel(got, ref) <= tol


def test_mirror_gather_is_matched_weight_by_weight():
    # the mirror-paired gather (n = 64) against the projector, weight by
    # weight: dense A from unit images, dense A^T from unit sinograms, with
    # angle pairs (1, 5), (2, 4) and the unpaired angles 0 and 3
    n, na, nb = 64, 6, 91
    A = np.zeros((na * nb, n * n))
    for q in range(n * n):
        e = torch.zeros(n * n, dtype=torch.float32, device=DEV)
        e[q] = 1
        A[:, q] = scg.scg_project(e.view(n, n), na, nb).cpu().numpy().ravel()
    AT = np.zeros((n * n, na * nb))
    for q in range(na * nb):
        e = torch.zeros(na * nb, dtype=torch.float32, device=DEV)
        e[q] = 1
        AT[:, q] = scg.scg_backproject(e.view(na, nb), n).cpu().numpy().ravel()
    scale = np.max(np.abs(A))
    assert np.max(np.abs(A - AT.T)) <= 1e-5 * scale
    one_sided = (A != 0) != (AT.T != 0)
    assert np.all(np.abs(A - AT.T)[one_sided] <= 1e-5 * scale)
    # no ray the projector sees is missing from the gather (a slot's band lost)
    assert np.all(np.abs(AT).sum(axis=0)[np.abs(A).sum(axis=1) > 0] > 0)


@pytest.mark.parametrize("dtype", [torch.float32, torch.float64])
@pytest.mark.parametrize("n,na,nb", CASES)
def test_fbp_matches_oracle(n, na, nb, dtype):
    x = image(n, 3 * n + na)
    y = oracle.project(x, na, nb) + 0.05 * inputs.normal(n, "fbp", na * nb).reshape(na, nb)
    ref = oracle.fbp(y, n)
    got = scg.scg_fbp(torch.tensor(y, dtype=dtype, device=DEV), n).cpu().numpy()
    assert rel(got, ref) <= (1e-5 if dtype == torch.float32 else 1e-11)


@pytest.mark.parametrize("dtype,tol", [(torch.float16, 2e-3), (torch.bfloat16, 1.5e-2)])
def test_fbp_reduced_storage(dtype, tol):
    n, na, nb = 130, 181, 185
    x = image(n, 11)
    y = oracle.project(x, na, nb)
    yq = torch.tensor(y, dtype=torch.float32).to(dtype)
    ref = oracle.fbp(yq.double().numpy(), n)
    got = scg.scg_fbp(yq.to(DEV), n).double().cpu().numpy()
    err = rel(got, ref)
    print(f"FBP {dtype}: rel L2 {err:.2e}")
    assert err <= tol


def test_fbp_of_full_size_phantom_on_sampled_pixels():
    # 512^2 / 720 x 725: FBP of the phantom's exact projections, sampled pixels
    # of A^T(filtered rows) against the oracle's filter and A^T one by one
    work = inputs.SINGLE_512
    n, na, nb = work.n, work.n_angles, work.n_bins
    x = inputs.ellipse_phantom(n, work.n_ellipses, 0)
    y = oracle.project(x, na, nb)
    got = scg.scg_fbp(torch.tensor(y, dtype=torch.float32, device=DEV), n).cpu().numpy()
    q = oracle.filter_rows(y, 1e-300, 1.0 / (2 * na))    # mu -> 0 (exact 0 selects the default)
    rng = np.random.default_rng(7)
    i = rng.integers(0, n, 200)
    j = rng.integers(0, n, 200)
    assert rel(got[i, j], oracle.backproject_pixels(q, n, i, j)) <= 1e-5
    # and it is an image of the phantom: the field of view within 10 % in L2 (the oracle: 6.3 %)
    fov = (np.arange(n)[:, None] - (n - 1) / 2) ** 2 + (np.arange(n)[None, :] - (n - 1) / 2) ** 2 <= (0.45 * n) ** 2
    assert rel(got[fov], x[fov]) <= 0.10


@pytest.mark.parametrize("work", [inputs.SINGLE_512, inputs.MIXED_1024], ids=lambda w: w.name)
def test_full_size_operators_on_sampled_outputs(work):
    n, na, nb = work.n, work.n_angles, work.n_bins
    x = inputs.normal(n, "zm", n * n).reshape(n, n)     # zero mean: cancelling ray sums
    y = scg.scg_project(torch.tensor(x, dtype=torch.float32, device=DEV), na, nb).cpu().numpy()
    rng = np.random.default_rng(1)
    a = rng.integers(0, na, 300)
    b = rng.integers(0, nb, 300)
    a[:4] = [0, na // 2, na // 4, na - 1]          # axis-aligned and diagonal angles
    ref = oracle.project_rays(x, na, nb, a, b)
    assert rel(y[a, b], ref) <= 1e-5
    r = inputs.normal(2, "r", na * nb).reshape(na, nb)
    g = scg.scg_backproject(torch.tensor(r, dtype=torch.float32, device=DEV), n).cpu().numpy()
    i = rng.integers(0, n, 200)
    j = rng.integers(0, n, 200)
    i[:2] = [0, n - 1]
    j[:2] = [0, n - 1]
    refp = oracle.backproject_pixels(r, n, i, j)
    assert rel(g[i, j], refp) <= 1e-5


def test_largest_image_side_on_sampled_outputs():
    # N = 8192 (the largest side the boundary accepts) with a few angles and a
    # detector wide enough for every ray: sampled rays and pixels against the
    # oracle evaluated one by one (the index arithmetic's extreme range)
    n, na, nb = 8192, 6, 11587
    x = torch.randn((n, n), dtype=torch.float32, device=DEV, generator=torch.Generator(DEV).manual_seed(3))
    y = scg.scg_project(x, na, nb).cpu().numpy()
    xh = x.double().cpu().numpy()
    rng = np.random.default_rng(4)
    a = rng.integers(0, na, 16)              # each sampled ray costs the oracle N^2 weights
    b = rng.integers(0, nb, 16)
    a[:3] = [0, na // 2, na // 3]
    b[:3] = [nb // 2, 0, nb - 1]
    assert rel(y[a, b], oracle.project_rays(xh, na, nb, a, b)) <= 1e-5
    r = torch.randn((na, nb), dtype=torch.float32, device=DEV, generator=torch.Generator(DEV).manual_seed(5))
    g = scg.scg_backproject(r, n).cpu().numpy()
    i = rng.integers(0, n, 40)
    j = rng.integers(0, n, 40)
    i[:2] = [0, n - 1]
    j[:2] = [n - 1, 0]
    assert rel(g[i, j], oracle.backproject_pixels(r.double().cpu().numpy(), n, i, j)) <= 1e-5
