"""Pins of the oracle's per-angle weighted data term (F = 1/2 sum_a w_a ||A_a x - g_a||^2 + lambda
Phi), against facts that do not go through the weighted functions themselves: unit weights give
the unweighted kernel, a zero weight removes its angle, K_w(0) has a closed form, the Toeplitz
convolution with K_w is the brute-force A^T W A, and the Toeplitz objective equals the
brute-force weighted objective."""
import math

import numpy as np
import pytest

import oracle as orc


@pytest.fixture(scope="module")
def geo():
    N, nd, na = 8, 8, 5
    rng = np.random.default_rng(5)
    theta = np.sort(rng.uniform(0.0, math.pi, na))
    w = rng.uniform(0.1, 1.0, na)
    return N, nd, theta, w


def test_unit_weights_give_the_unweighted_kernel(geo):
    N, nd, theta, _ = geo
    K1 = orc.kernel_weighted(N, theta, nd, np.ones(theta.size))
    K = orc.kernel(N, theta, nd)
    assert np.max(np.abs(K1 - K)) <= 1e-12 * np.max(np.abs(K))


def test_zero_weight_removes_its_angle(geo):
    N, nd, theta, w = geo
    w0 = w.copy()
    w0[2] = 0.0
    keep = np.array([a for a in range(theta.size) if a != 2])
    Ka = orc.kernel_weighted(N, theta, nd, w0)
    Kb = orc.kernel_weighted(N, theta[keep], nd, w[keep])
    assert np.max(np.abs(Ka - Kb)) <= 1e-12 * np.max(np.abs(Kb))


def test_kernel_at_zero_offset(geo):
    # D(0) = nd - 1 for every angle (the |k| <= nd/2 - 1 sum of ones), so K_w(0) = (nd - 1)/nd sum w
    N, nd, theta, w = geo
    K = orc.kernel_weighted(N, theta, nd, w)
    assert abs(K[N - 1, N - 1] - (nd - 1) / nd * np.sum(w)) <= 1e-12 * np.sum(w)


def test_toeplitz_with_weighted_kernel_is_brute_force_normal_operator(geo):
    N, nd, theta, w = geo
    rng = np.random.default_rng(6)
    x = rng.standard_normal((N, N))
    z = orc.toeplitz(x, orc.kernel_weighted(N, theta, nd, w))
    ref = orc.adjoint(w[:, None] * orc.forward(x, theta, nd), N, theta)
    assert np.linalg.norm(z - ref) <= 1e-10 * np.linalg.norm(ref)


def test_weighted_objective_matches_brute_force(geo):
    N, nd, theta, w = geo
    rng = np.random.default_rng(7)
    S = 2
    x = rng.uniform(0.0, 1.0, (S, N, N))
    g = rng.standard_normal((S, theta.size, nd))
    pr = orc.Prior()
    K = orc.kernel_weighted(N, theta, nd, w)
    atg = orc.adjoint_weighted(g, N, theta, w)
    F = orc.objective(x, atg, orc.gtg_weighted(g, w), K, pr)
    Fd = orc.objective_direct_weighted(x, g, theta, pr, w)
    assert abs(F - Fd) <= 1e-10 * abs(Fd)
    # and its gradient is K_w * x - R* W g + lambda grad Phi: a finite difference along a direction
    v = rng.standard_normal(x.shape)
    h = 1e-6
    fd = (orc.objective_direct_weighted(x + h * v, g, theta, pr, w)
          - orc.objective_direct_weighted(x - h * v, g, theta, pr, w)) / (2 * h)
    G = orc.gradient(x, atg, K, pr)
    assert abs(float(np.sum(G * v)) - fd) <= 1e-6 * abs(fd)
