"""Pins of the oracle's TV, TV subgradient and preconditioning filter (CPU only).

TV is the paper's secondary criterion (Sec. 1, Sec. 3); the paper gives no
formula, so the isotropic forward-difference TV over the (N-1)^2 interior
terms is this project's reading.  The filter is Sec. 3's
c(w) = (|w| + mu)(0.54 + 0.46 cos w) applied to each projection row.
"""
import math

import numpy as np
import pytest

import oracle


def test_tv_of_constant_is_zero():
    assert oracle.tv(np.full((9, 9), 3.25)) == 0.0
    t, g = oracle.tv_grad(np.full((9, 9), -1.0))
    assert t == 0.0 and np.all(g == 0.0)


@pytest.mark.parametrize("alpha,beta,n", [(0.3, -1.1, 7), (2.0, 0.0, 10), (-0.5, 0.25, 16)])
def test_tv_of_linear_ramp_closed_form(alpha, beta, n):
    i, j = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    x = alpha * i + beta * j
    assert oracle.tv(x) == pytest.approx((n - 1) ** 2 * math.hypot(alpha, beta), rel=1e-13)


def test_tv_hand_worked_2x2():
    # one interior term: du = x[1,0]-x[0,0] = 2, dv = x[0,1]-x[0,0] = 1
    x = np.array([[0.0, 1.0], [2.0, 3.0]])
    t, g = oracle.tv_grad(x)
    r5 = math.sqrt(5.0)
    assert t == pytest.approx(r5, rel=1e-15)
    np.testing.assert_allclose(g, [[-3 / r5, 1 / r5], [2 / r5, 0.0]], rtol=1e-15)


def test_tv_subgradient_matches_central_differences():
    rng = np.random.default_rng(3)
    n = 8
    x = rng.standard_normal((n, n))          # no zero-norm terms almost surely
    t, g = oracle.tv_grad(x)
    h = 1e-6
    fd = np.zeros_like(x)
    for i in range(n):
        for j in range(n):
            xp = x.copy(); xp[i, j] += h
            xm = x.copy(); xm[i, j] -= h
            fd[i, j] = (oracle.tv(xp) - oracle.tv(xm)) / (2 * h)
    np.testing.assert_allclose(g, fd, rtol=1e-5, atol=1e-6)


def test_tv_subgradient_is_nonascending_direction():
    rng = np.random.default_rng(4)
    x = rng.standard_normal((12, 12))
    t, g = oracle.tv_grad(x)
    v = -g / np.linalg.norm(g)
    assert oracle.tv(x + 1e-4 * v) < t


def test_filter_factor_special_values():
    mu = 0.01
    assert oracle.filter_factor(0.0, mu) == pytest.approx(mu, rel=1e-15)
    assert oracle.filter_factor(math.pi, mu) == pytest.approx((math.pi + mu) * 0.08, rel=1e-14)
    assert oracle.filter_factor(-1.0, mu) == oracle.filter_factor(1.0, mu)


@pytest.mark.parametrize("nb,expect", [(5, 16), (8, 16), (95, 256), (725, 2048), (1449, 4096)])
def test_filter_length(nb, expect):
    assert oracle.filter_length(nb) == expect


@pytest.mark.parametrize("na,nb,mu,gain", [(3, 7, 0.0, 1.0), (5, 20, 0.05, 1.0), (4, 33, 0.0, 2.5)])
def test_filter_matches_fft_route(na, nb, mu, gain):
    rng = np.random.default_rng(nb)
    r = rng.standard_normal((na, nb))
    P = oracle.filter_length(nb)
    mu_eff = mu if mu > 0 else 2 * math.pi / P
    w = 2 * math.pi * np.fft.fftfreq(P)
    c = gain * (np.abs(w) + mu_eff) * (0.54 + 0.46 * np.cos(w))
    pad = np.zeros((na, P))
    pad[:, :nb] = r
    ref = np.real(np.fft.ifft(c * np.fft.fft(pad, axis=1), axis=1))[:, :nb]
    np.testing.assert_allclose(oracle.filter_rows(r, mu, gain), ref, rtol=0, atol=1e-12)
