"""The single-voxel oracle functions the full-size GPU parity tests sample (normal_point,
adjoint_point, forward_point, prior_point, and the FBP start at a pixel) equal the corresponding entries of the
whole-array oracle functions, at corners, edges and interior voxels."""
import math

import numpy as np

import synth

PRIOR = dict(p=1.2, q=2.0, c=0.01, sigma=0.1, lam=1.7)
PIXELS = [(0, 0), (0, 11), (11, 0), (11, 11), (5, 6), (3, 9)]


def test_normal_point_equals_the_direct_product(orc):
    N = 12
    th = synth.angles(9)
    K = orc.kernel(N, th, N)
    x = np.random.default_rng(21).standard_normal((N, N))
    full = orc.normal_direct(x, K)
    for r, c in PIXELS:
        assert abs(orc.normal_point(x, K, r, c) - full[r, c]) <= 1e-12 * np.abs(full).max()


def test_adjoint_point_equals_the_adjoint(orc):
    N = 12
    th = synth.angles(9)
    g = np.random.default_rng(22).standard_normal((th.size, N))
    full = orc.adjoint(g, N, th)
    for r, c in PIXELS:
        assert abs(orc.adjoint_point(g, N, th, r, c) - full[r, c]) <= 1e-12 * np.abs(full).max()


def test_prior_point_equals_the_prior_gradient(orc):
    pr = orc.Prior(**PRIOR)
    x = np.random.default_rng(23).normal(0, 0.05, (3, 12, 12))
    g, _ = orc.prior(x, pr)
    for z in (0, 1, 2):
        for r, c in PIXELS:
            assert abs(orc.prior_point(x, pr, z, r, c) - g[z, r, c]) <= 1e-12 * np.abs(g).max()
    # one slice: the in-plane neighbours only
    g1, _ = orc.prior(x[1], pr)
    for r, c in PIXELS:
        assert abs(orc.prior_point(x[1], pr, 0, r, c) - g1[r, c]) <= 1e-12 * np.abs(g1).max()


def test_fbp_at_a_pixel_equals_the_fbp_image(orc):
    N = 16
    th = synth.angles(20)
    g = np.random.default_rng(24).standard_normal((th.size, N))
    full = orc.fbp(g, N, th, math.pi)
    filtered = orc.ramp_filter(g)
    for r, c in [(0, 0), (15, 15), (7, 8), (2, 13)]:
        v = (math.pi / th.size) * orc.adjoint_point(filtered, N, th, r, c)
        assert abs(v - full[r, c]) <= 1e-12 * np.abs(full).max()


def test_forward_point_equals_the_forward_projection(orc):
    N = 12
    th = synth.angles(9, 2 * math.pi / 3)
    x = np.random.default_rng(25).standard_normal((N, N))
    full = orc.forward(x, th, N)
    for a, m in [(0, 0), (8, 11), (4, 6), (2, 0), (6, 9)]:
        assert abs(orc.forward_point(x, th[a], N, m) - full[a, m]) <= 1e-12 * np.abs(full).max()
