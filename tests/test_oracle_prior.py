"""Pins for the oracle's qGGMRF prior (Sec. 2, Eq. 5; 26-neighbour coupling of Sec. 2.4).

Closed forms of the potential, finite differences of Phi, invariances and
single-voxel volumes whose Phi and gradient can be written down by hand.
"""
import itertools
import math

import numpy as np

PRIOR = dict(p=1.2, q=2.0, c=0.01, sigma=0.1, lam=1.0)


def P(orc, **kw):
    d = dict(PRIOR)
    d.update(kw)
    return orc.Prior(**d)


def test_weights(orc):
    ws = {o: orc.neighbour_weight(*o) for o in itertools.product((-1, 0, 1), repeat=3) if o != (0, 0, 0)}
    assert len(ws) == 26
    assert abs(sum(ws.values()) - 1.0) < 1e-14
    face, edge, corner = ws[(0, 0, 1)], ws[(0, 1, 1)], ws[(1, 1, 1)]
    assert abs(face / edge - math.sqrt(2)) < 1e-14 and abs(face / corner - math.sqrt(3)) < 1e-14
    assert abs(face - 1.0 / (6 + 12 / math.sqrt(2) + 8 / math.sqrt(3))) < 1e-15


def test_potential_closed_forms(orc):
    pr = P(orc)
    # |D| = c sigma: u = 1, rho = c^q / 2
    assert abs(orc.rho(pr.c * pr.sigma, pr) - pr.c ** pr.q / 2) < 1e-15
    assert orc.rho(0.0, pr) == 0.0 and orc.drho(0.0, pr) == 0.0
    # p = q: Gaussian MRF rho = (D/sigma)^2 / 2, rho' = D / sigma^2
    g = P(orc, p=2.0)
    for d in (-0.3, 0.05, 1.7):
        assert abs(orc.rho(d, g) - 0.5 * (d / g.sigma) ** 2) < 1e-12
        assert abs(orc.drho(d, g) - d / g.sigma ** 2) < 1e-10
    # large |D|: rho ~ c^(q-p) |D/sigma|^p (edge-preserving tail)
    d = 1e6 * pr.c * pr.sigma
    assert abs(orc.rho(d, pr) / (pr.c ** (pr.q - pr.p) * (d / pr.sigma) ** pr.p) - 1) < 1e-3


def test_drho_is_derivative_of_rho(orc):
    pr = P(orc)
    for d in (-0.5, -0.02, -1e-3, 2e-4, 0.003, 0.1, 2.0):
        h = 1e-6 * max(abs(d), 1e-3)
        fd = (orc.rho(d + h, pr) - orc.rho(d - h, pr)) / (2 * h)
        assert abs(orc.drho(d, pr) - fd) <= 1e-6 * max(abs(fd), 1e-8)
    assert orc.drho(-0.3, pr) == -orc.drho(0.3, pr)


def test_max_curvature_bound(orc):
    pr = P(orc)
    d = np.concatenate([np.geomspace(1e-9, 10, 4000)])
    h = 1e-7
    curv = [(orc.drho(v + h, pr) - orc.drho(v - h, pr)) / (2 * h) for v in d[d > 1e-6]]
    assert max(curv) <= orc.max_rho2(pr) * (1 + 1e-6)
    assert max(curv) > 0.95 * orc.max_rho2(pr)


def test_gradient_matches_finite_differences(orc):
    rng = np.random.default_rng(11)
    pr = P(orc)
    x = rng.normal(0, 0.05, (3, 5, 6))
    g, _ = orc.prior(x, pr)
    h = 1e-7
    for idx in [(0, 0, 0), (1, 2, 3), (2, 4, 5), (1, 0, 2), (2, 3, 0)]:
        xp = x.copy()
        xp[idx] += h
        xm = x.copy()
        xm[idx] -= h
        fd = (orc.prior(xp, pr)[1] - orc.prior(xm, pr)[1]) / (2 * h)
        assert abs(g[idx] - fd) <= 1e-6 * max(abs(fd), 1e-6)


def test_single_voxel_volume(orc):
    pr = P(orc, lam=1.7)
    v = 0.37
    x = np.zeros((3, 3, 3))
    x[1, 1, 1] = v
    g, phi = orc.prior(x, pr)
    # all 26 neighbours present, weights sum to 1
    assert abs(phi - pr.lam * orc.rho(v, pr)) < 1e-12
    assert abs(g[1, 1, 1] - pr.lam * orc.drho(v, pr)) < 1e-12
    assert abs(g[0, 0, 0] + pr.lam * orc.neighbour_weight(1, 1, 1) * orc.drho(v, pr)) < 1e-12
    # a single slice keeps its 8 in-plane neighbours with the same weights
    s = np.zeros((3, 3))
    s[1, 1] = v
    g2, phi2 = orc.prior(s, pr)
    w8 = sum(orc.neighbour_weight(0, dy, dx) for dy in (-1, 0, 1) for dx in (-1, 0, 1) if (dy, dx) != (0, 0))
    assert abs(phi2 - pr.lam * w8 * orc.rho(v, pr)) < 1e-12
    assert abs(g2[1, 1] - pr.lam * w8 * orc.drho(v, pr)) < 1e-12


def test_invariances(orc):
    rng = np.random.default_rng(12)
    pr = P(orc)
    x = rng.normal(0, 0.1, (4, 7, 7))
    g, phi = orc.prior(x, pr)
    assert abs(g.sum()) < 1e-9 * np.abs(g).sum()  # translation invariance
    g2, phi2 = orc.prior(x + 3.0, pr)
    assert np.allclose(g, g2, atol=1e-9) and abs(phi - phi2) < 1e-9 * phi
    gq = P(orc, p=2.0)
    assert abs(orc.prior(2.5 * x, gq)[1] - 2.5 ** 2 * orc.prior(x, gq)[1]) < 1e-9 * orc.prior(x, gq)[1]
    # mirror symmetry of the neighbourhood
    gm, phim = orc.prior(x[::-1, ::-1, ::-1].copy(), pr)
    assert np.allclose(gm, g[::-1, ::-1, ::-1], atol=1e-12) and abs(phim - phi) < 1e-10 * phi


def test_potential_with_q_below_two(orc):
    # q != 2 (the general qGGMRF): the closed forms and derivatives hold for any 1 <= p <= q
    for p, q in ((1.1, 1.8), (1.0, 1.5), (1.5, 1.9)):
        pr = P(orc, p=p, q=q)
        cs = pr.c * pr.sigma
        assert abs(orc.rho(cs, pr) - pr.c ** q / 2) < 1e-15  # u = 1 at |D| = c sigma
        for d in (-0.4, -3e-3, 5e-4, 0.02, 1.3):
            h = 1e-6 * abs(d)
            fd = (orc.rho(d + h, pr) - orc.rho(d - h, pr)) / (2 * h)
            assert abs(orc.drho(d, pr) - fd) <= 1e-6 * abs(fd)
            assert orc.drho(-d, pr) == -orc.drho(d, pr)
        # far tail: rho ~ c^(q-p) |D/sigma|^p
        d = 1e8 * cs
        assert abs(orc.rho(d, pr) / (pr.c ** (q - p) * (d / pr.sigma) ** p) - 1) < 1e-3
    # p = q < 2: the generalised Gaussian |D/sigma|^q / 2
    g = P(orc, p=1.6, q=1.6)
    for d in (-0.3, 0.05, 1.7):
        assert abs(orc.rho(d, g) - 0.5 * abs(d / g.sigma) ** 1.6) < 1e-12


def test_gradient_with_q_below_two_matches_finite_differences(orc):
    rng = np.random.default_rng(13)
    pr = P(orc, p=1.1, q=1.8)
    x = rng.normal(0, 0.05, (3, 5, 6))
    g, _ = orc.prior(x, pr)
    h = 1e-7
    for idx in [(0, 0, 0), (1, 2, 3), (2, 4, 5), (1, 0, 2)]:
        xp = x.copy()
        xp[idx] += h
        xm = x.copy()
        xm[idx] -= h
        fd = (orc.prior(xp, pr)[1] - orc.prior(xm, pr)[1]) / (2 * h)
        assert abs(g[idx] - fd) <= 1e-6 * max(abs(fd), 1e-6)
