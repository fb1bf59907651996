"""Pins of the oracle's system matrix A and its transpose (CPU only).

A is the paper's L x J matrix of discretised line integrals (Sec. 1, Eq. LS1)
for the parallel-beam scan of Sec. 4; here its entries are exact ray-pixel
chord lengths.  Each test pins the oracle to a fact outside itself: a second
derivation of the chord, hand-worked single-pixel profiles, the chord of the
whole image square, the line integral of a disk, the unit area of a pixel and
the adjoint identity.
"""
import math

import numpy as np
import pytest

import oracle


def dense_matrix(n, na, nb, clip=False):
    J = n * n
    A = np.zeros((na * nb, J))
    for q in range(J):
        e = np.zeros(J)
        e[q] = 1.0
        A[:, q] = oracle.project_dense(e.reshape(n, n), na, nb, clip=clip).ravel()
    return A


@pytest.mark.parametrize("n,na,nb", [(4, 8, 6), (5, 12, 7), (6, 9, 9), (7, 16, 11)])
def test_two_weight_derivations_agree(n, na, nb):
    # slab clipping and the closed-form trapezoid are independent derivations
    A_clip = dense_matrix(n, na, nb, clip=True)
    A_trap = dense_matrix(n, na, nb, clip=False)
    assert np.max(np.abs(A_clip - A_trap)) < 1e-13


@pytest.mark.parametrize("n,na,nb", [(6, 8, 9), (7, 12, 10), (8, 20, 12), (9, 7, 13)])
def test_footprint_loops_equal_dense_definition(n, na, nb):
    rng = np.random.default_rng(n * 100 + na)
    x = rng.standard_normal((n, n))
    r = rng.standard_normal((na, nb))
    np.testing.assert_allclose(oracle.project(x, na, nb), oracle.project_dense(x, na, nb),
                               rtol=0, atol=1e-12)
    np.testing.assert_allclose(oracle.backproject(r, n), oracle.backproject_dense(r, n),
                               rtol=0, atol=1e-12)


def test_single_pixel_axis_profiles_hand_worked():
    # N = 4: pixel (i=2, j=1) has centre (xc, yc) = (-0.5, 0.5).
    e = np.zeros((4, 4))
    e[2, 1] = 1.0
    # odd bin count: bin centres are integers, so at theta = 0 the rays
    # s = -1 and s = 0 run along the pixel's two vertical edges -> 1/2 each
    y = oracle.project(e, 4, 5)          # angles 0, pi/4, pi/2, 3pi/4
    np.testing.assert_allclose(y[0], [0, 0.5, 0.5, 0, 0], atol=1e-15)
    # at theta = pi/2 the ray coordinate is yc = 0.5: rays s = 0 and s = 1 share it
    np.testing.assert_allclose(y[2], [0, 0, 0.5, 0.5, 0], atol=1e-15)
    # even bin count: bin centres are half-integers, one ray through the centre
    y = oracle.project(e, 4, 4)
    np.testing.assert_allclose(y[0], [0, 1, 0, 0], atol=1e-15)
    np.testing.assert_allclose(y[2], [0, 0, 1, 0], atol=1e-15)


def test_diagonal_profile_is_triangle():
    # theta = pi/4: peak sqrt(2) at d = 0, half-width sqrt(2)/2, linear between
    c, s = oracle.angle(1, 4)
    assert oracle.weight_trap(0.0, c, s) == pytest.approx(math.sqrt(2), abs=1e-12)
    assert oracle.weight_trap(math.sqrt(2) / 4, c, s) == pytest.approx(math.sqrt(2) / 2, abs=1e-12)
    assert oracle.weight_trap(math.sqrt(2) / 2 + 1e-9, c, s) == 0.0
    # and the same value from clipping a centred pixel
    assert oracle.weight_clip(0.0, 0.0, c, s, 0.0) == pytest.approx(math.sqrt(2), abs=1e-12)


@pytest.mark.parametrize("theta_deg", [7.0, 30.0, 45.0, 63.0, 89.0, 101.0])
def test_generic_angle_trapezoid(theta_deg):
    th = math.radians(theta_deg)
    c, s = math.cos(th), math.sin(th)
    m, n = max(abs(c), abs(s)), min(abs(c), abs(s))
    # plateau height 1/m, zero beyond (m+n)/2, halfway down at the ramp centre
    assert oracle.weight_trap(0.0, c, s) == pytest.approx(1 / m, rel=1e-14)
    assert oracle.weight_trap((m - n) / 2 + n / 2, c, s) == pytest.approx(0.5 / m, rel=1e-12)
    assert oracle.weight_trap((m + n) / 2, c, s) == 0.0


def square_chord(d, c, s, side):
    """Chord of the line at signed distance d through a centred square of side
    ``side``: flat top side/m, linear ramps of width side*n, shared half on an
    edge when the line is axis-aligned."""
    m, n = max(abs(c), abs(s)), min(abs(c), abs(s))
    ad = abs(d)
    if n == 0.0:
        if ad < side / 2:
            return side / m
        return side / (2 * m) if ad == side / 2 else 0.0
    if ad <= side * (m - n) / 2:
        return side / m
    if ad < side * (m + n) / 2:
        return (side * (m + n) / 2 - ad) / (m * n)
    return 0.0


@pytest.mark.parametrize("n,na,nb", [(8, 16, 13), (9, 12, 14), (16, 36, 24)])
def test_ones_image_gives_chord_of_image_square(n, na, nb):
    # chords are additive over the pixels a ray crosses
    y = oracle.project(np.ones((n, n)), na, nb)
    for a in range(na):
        c, s = oracle.angle(a, na)
        for b in range(nb):
            sb = b - (nb - 1) / 2
            assert y[a, b] == pytest.approx(square_chord(sb, c, s, n), abs=1e-11)


def test_disk_line_integrals():
    n, na, nb, R = 64, 30, 91, 20.0
    idx = np.arange(n) - (n - 1) / 2
    yy, xx = np.meshgrid(idx, idx, indexing="ij")
    disk = (xx ** 2 + yy ** 2 <= R * R).astype(float)
    y = oracle.project(disk, na, nb)
    s = np.arange(nb) - (nb - 1) / 2
    inside = np.abs(s) < R - 1
    exact = 2 * np.sqrt(np.maximum(R * R - s ** 2, 0))
    err = np.abs(y[:, inside] - exact[inside])
    # pixelisation of a centre-sampled disk moves each chord end by < 1 pixel
    assert err.max() < 2.0
    assert err.mean() / exact[inside].mean() < 2.0 / R


@pytest.mark.parametrize("a,na", [(1, 7), (3, 10), (5, 12), (0, 4), (2, 4), (13, 40)])
def test_weight_integrates_to_pixel_area(a, na):
    c, s = oracle.angle(a, na)
    h = 1e-4
    d = np.arange(-1.0, 1.0 + h / 2, h)
    vals = np.array([oracle.weight_trap(v, c, s) for v in d])
    assert np.sum(vals) * h == pytest.approx(1.0, abs=2e-4)


@pytest.mark.parametrize("n,na,nb", [(16, 20, 23), (32, 45, 46), (33, 60, 47)])
def test_adjoint_identity(n, na, nb):
    rng = np.random.default_rng(n + na)
    x = rng.standard_normal((n, n))
    r = rng.standard_normal((na, nb))
    lhs = np.sum(oracle.project(x, na, nb) * r)
    rhs = np.sum(x * oracle.backproject(r, n))
    assert abs(lhs - rhs) <= 1e-12 * (abs(lhs) + np.linalg.norm(x) * np.linalg.norm(r))


def test_sampled_rays_and_pixels_match_full_operators():
    n, na, nb = 24, 30, 35
    rng = np.random.default_rng(5)
    x = rng.standard_normal((n, n))
    r = rng.standard_normal((na, nb))
    y = oracle.project(x, na, nb)
    g = oracle.backproject(r, n)
    a = rng.integers(0, na, 50)
    b = rng.integers(0, nb, 50)
    np.testing.assert_allclose(oracle.project_rays(x, na, nb, a, b), y[a, b], atol=1e-12)
    i = rng.integers(0, n, 50)
    j = rng.integers(0, n, 50)
    np.testing.assert_allclose(oracle.backproject_pixels(r, n, i, j), g[i, j], atol=1e-12)
