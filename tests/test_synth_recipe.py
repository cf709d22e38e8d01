"""The seeded input generator follows the recipe stated for the workloads: random ellipses and
ellipsoids inside the inscribed disc, exact line integrals at the bin centres, Gaussian noise of
1 % of the maximum (volumes) or Poisson transmission noise (single slices), uniform angles."""
import numpy as np

import synth


def test_angles_are_uniform_over_the_span():
    th = synth.angles(128, 2 * np.pi / 3)
    assert th[0] == 0.0 and th[-1] < 2 * np.pi / 3
    assert np.allclose(np.diff(th), (2 * np.pi / 3) / 128, rtol=0, atol=1e-15)


def test_ellipses_stay_in_the_recipe_ranges():
    N = 512
    R = N / 2
    e = synth.random_ellipses(np.random.default_rng(3), 2000, N)
    r0 = np.hypot(e.x0, e.y0)
    assert r0.max() <= 0.55 * R
    assert np.all(r0 + np.maximum(e.a, e.b) <= 0.95 * R + 1e-9)  # inside the inscribed disc
    assert e.a.max() <= 0.35 * R and e.b.max() <= 0.35 * R and min(e.a.min(), e.b.min()) > 0
    assert 0.0 <= e.phi.min() and e.phi.max() < np.pi
    assert 0.0 <= e.rho.min() and e.rho.max() < 1.0


def test_ellipsoids_extent_along_the_slice_axis():
    S = 64
    v = synth.random_ellipsoids(np.random.default_rng(4), 500, 256, S)
    assert v.cz.min() >= 0.1 * S and v.cz.max() <= 0.5 * S
    assert v.z0.min() >= 0.0 and v.z0.max() < S
    # a cross-section outside an ellipsoid drops it; at its centre it is the full ellipse
    one = synth.Ellipsoids(synth.Ellipses(*[a[:1] for a in (v.plane.x0, v.plane.y0, v.plane.a, v.plane.b,
                                                               v.plane.phi, v.plane.rho)]), v.z0[:1], v.cz[:1])
    assert synth.ellipsoid_slice(one, float(v.z0[0] + 1.01 * v.cz[0])).x0.size == 0
    mid = synth.ellipsoid_slice(one, float(v.z0[0]))
    assert mid.a[0] == v.plane.a[0] and mid.b[0] == v.plane.b[0]


def test_volume_noise_is_one_percent_of_the_maximum():
    S, N, na, seed = 4, 128, 60, 11
    p = synth.volume(S=S, N=N, n_angles=na, n_ellipsoids=6, seed=seed)
    # the same phantom without noise: the generator's own exact line integrals
    e = synth.random_ellipsoids(np.random.default_rng(seed), 6, N, S)
    g = np.stack([synth.ellipse_projections(synth.ellipsoid_slice(e, z + 0.5), p.theta, N) for z in range(S)])
    noise = p.sino.astype(np.float64) - g
    assert abs(noise.std() / (0.01 * g.max()) - 1.0) < 0.05
    assert abs(noise.mean()) < 0.05 * 0.01 * g.max()


def test_poisson_noise_vanishes_with_many_photons():
    g = synth.ellipse_projections(synth.random_ellipses(np.random.default_rng(5), 5, 128), synth.angles(30), 128)
    y = synth.poisson_noise(np.random.default_rng(6), g, 1e14)
    assert np.max(np.abs(y - g)) < 1e-4 * g.max()
