"""Pins of the oracle's filtered backprojection (Sec. 4's FBP reference image;
the Hamming-windowed ramp factors of Sec. 3 with mu = 0, in cycles per bin).

* The filtering step against numpy's FFT: rows zero-padded to P, multiplied by
  the ramp |nu| = |w|/(2 pi), the Hamming window and the angle step
  pi/n_angles, transformed back, cropped; then the oracle's A^T (pinned by the
  adjoint and chord tests).
* Reconstruction of a uniform disk from its exact projections: the interior
  is 1 and the outside 0, up to the discretisation (centre-sampled disk edge,
  windowed ramp, the DC term a sampled ramp drops).
* Linearity: FBP of s y is s FBP(y).
"""
import numpy as np
import pytest

import oracle


def fft_route(y, n):
    na, nb = y.shape
    P = 1
    while P < 2 * nb:
        P *= 2
    k = np.arange(P)
    w = np.where(k <= P // 2, 2 * np.pi * k / P, 2 * np.pi * (k - P) / P)
    nu = np.abs(w) / (2 * np.pi)                      # cycles per bin width
    c = nu * (0.54 + 0.46 * np.cos(w)) * np.pi / na    # ramp, Hamming window, d theta
    pad = np.zeros((na, P))
    pad[:, :nb] = y
    q = np.real(np.fft.ifft(np.fft.fft(pad, axis=1) * c, axis=1))[:, :nb]
    return oracle.backproject(q, n)


@pytest.mark.parametrize("n,na,nb", [(16, 20, 23), (33, 45, 47), (40, 1, 57)])
def test_fbp_filter_matches_numpy_fft(n, na, nb):
    rng = np.random.default_rng(n + na)
    y = rng.standard_normal((na, nb))
    ref = fft_route(y, n)
    got = oracle.fbp(y, n)
    assert np.linalg.norm(got - ref) / np.linalg.norm(ref) <= 1e-12


@pytest.mark.parametrize("radius", [10.0, 20.0])
def test_fbp_reconstructs_a_uniform_disk(radius):
    n, na, nb = 64, 180, 95
    idx = np.arange(n) - 0.5 * (n - 1)
    yy, xx = np.meshgrid(idx, idx, indexing="ij")
    r2 = xx ** 2 + yy ** 2
    disk = (r2 <= radius * radius).astype(float)
    x = oracle.fbp(oracle.project(disk, na, nb), n)
    inner = r2 <= (radius - 4) ** 2
    outer = (r2 >= (radius + 4) ** 2) & (r2 <= 30 ** 2)
    assert abs(x[inner].mean() - 1.0) <= 0.02
    assert np.max(np.abs(x[inner] - 1.0)) <= 0.08
    assert abs(x[outer].mean()) <= 0.02


def test_fbp_is_linear():
    rng = np.random.default_rng(5)
    y = rng.standard_normal((30, 29))
    np.testing.assert_allclose(oracle.fbp(2.5 * y, 20), 2.5 * oracle.fbp(y, 20), rtol=1e-13, atol=1e-13)
