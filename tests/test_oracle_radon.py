"""Pins for the oracle's Radon operators (Sec. 2, Eqs. 1-4) and Toeplitz identity (Sec. 2.1, Eqs. 7-9).

Every check here compares the oracle with something it does not compute itself:
an explicit non-uniform DFT written out in numpy, the exact line integrals of a
Gaussian blob and of ellipses, the adjoint identity, closed forms for K, or the
dense matrix of A^T A.
"""
import numpy as np
import pytest

import synth


def nudft_forward(x, theta, nd):
    """Eq. 3 written out: type-2 non-uniform DFT onto the polar samples, then 1D inverse DFT per angle."""
    N = x.shape[0]
    cc = np.arange(N) - N // 2
    X, Y = np.meshgrid(cc, cc)  # X: column coordinate, Y: row coordinate
    k = np.arange(-(nd // 2 - 1), nd // 2)
    s = np.arange(nd) - nd / 2
    out = np.zeros((theta.size, nd))
    for a, th in enumerate(theta):
        proj = X * np.cos(th) + Y * np.sin(th)
        F = np.array([np.sum(x * np.exp(-2j * np.pi * kk * proj / nd)) for kk in k])
        out[a] = (np.exp(2j * np.pi * np.outer(s, k) / nd) @ F).real / nd
    return out


def test_dirichlet_matches_its_series(orc):
    rng = np.random.default_rng(1)
    for nd in (8, 16, 64):
        k = np.arange(-(nd // 2 - 1), nd // 2)
        for t in np.concatenate([rng.uniform(-3 * nd, 3 * nd, 20), [0.0, nd, -2.0 * nd, 1e-9]]):
            ref = np.sum(np.cos(2 * np.pi * k * t / nd))
            assert abs(orc.dirichlet(t, nd) - ref) < 1e-10 * nd


def test_forward_is_eq3_nudft(orc):
    rng = np.random.default_rng(2)
    N, nd = 10, 12
    th = rng.uniform(0, np.pi, 7)
    x = rng.standard_normal((N, N))
    ref = nudft_forward(x, th, nd)
    got = orc.forward(x, th, nd)
    assert np.max(np.abs(got - ref)) < 1e-11 * np.max(np.abs(ref))


def test_forward_exact_on_gaussian_blob(orc):
    # a blob of width 2.5 px is band-limited to ~1e-13 at the pixel Nyquist frequency,
    # so the discrete projections must equal its exact line integrals
    N, nd = 48, 64
    th = synth.angles(13)
    x = synth.gaussian_blob(N, 2.3, -1.7, 2.5)
    got = orc.forward(x, th, nd)
    ref = synth.gaussian_blob_projections(th, nd, 2.3, -1.7, 2.5)
    assert np.linalg.norm(got - ref) / np.linalg.norm(ref) < 1e-12
    # the mirrored blob (x and y swapped) is far away: geometry and angle sense are pinned
    bad = synth.gaussian_blob_projections(th, nd, -1.7, 2.3, 2.5)
    assert np.linalg.norm(got - bad) / np.linalg.norm(ref) > 0.5


def test_forward_approximates_ellipse_line_integrals(orc):
    errs = []
    for N in (32, 64, 128):
        rng = np.random.default_rng(5)
        e = synth.random_ellipses(rng, 6, N)
        th = synth.angles(24)
        g = orc.forward(synth.rasterize(e, N, 8), th, N)
        ref = synth.ellipse_projections(e, th, N)
        errs.append(np.linalg.norm(g - ref) / np.linalg.norm(ref))
    assert errs[-1] < 0.02
    assert errs[0] > errs[1] > errs[2]


def test_adjoint_identity(orc):
    rng = np.random.default_rng(3)
    N, nd = 16, 20
    th = rng.uniform(0, np.pi, 9)
    x = rng.standard_normal((N, N))
    y = rng.standard_normal((9, nd))
    lhs = np.sum(orc.forward(x, th, nd) * y)
    rhs = np.sum(x * orc.adjoint(y, N, th))
    assert abs(lhs - rhs) <= 1e-12 * max(abs(lhs), 1.0)


def test_mass_is_conserved_per_angle(orc):
    rng = np.random.default_rng(4)
    N, nd = 16, 24
    th = rng.uniform(0, np.pi, 5)
    x = rng.uniform(0, 1, (N, N))
    g = orc.forward(x, th, nd)
    assert np.allclose(g.sum(axis=1), x.sum(), rtol=1e-12)


def test_kernel_closed_forms(orc):
    N, nd, na = 12, 16, 11
    th = synth.angles(na)
    K = orc.kernel(N, th, nd)
    assert abs(K[N - 1, N - 1] - na * (nd - 1) / nd) < 1e-12
    assert np.allclose(K, K[::-1, ::-1], atol=1e-12)  # K(-d) = K(d)
    assert np.allclose(K, K[::-1, :], atol=1e-12)  # uniform [0, pi) angles: K(dx, -dy) = K(dx, dy)
    # limited angle set breaks the mirror symmetry but keeps the point symmetry
    K2 = orc.kernel(N, synth.angles(na, 2 * np.pi / 3), nd)
    assert np.allclose(K2, K2[::-1, ::-1], atol=1e-12)
    assert not np.allclose(K2, K2[::-1, :], atol=1e-3)


def test_toeplitz_equals_normal_operator(orc):
    rng = np.random.default_rng(6)
    N, nd = 14, 16
    th = rng.uniform(0, np.pi, 9)
    x = rng.standard_normal((N, N))
    K = orc.kernel(N, th, nd)
    ata = orc.adjoint(orc.forward(x, th, nd), N, th)
    direct = orc.normal_direct(x, K)
    fft_min = orc.toeplitz(x, K)  # padded to 2N-1, as printed in Eq. 9
    fft_2n = orc.toeplitz(x, K, orc.circulant_spectrum(K, 2 * N))
    scale = np.linalg.norm(ata)
    assert np.linalg.norm(direct - ata) < 1e-12 * scale
    assert np.linalg.norm(fft_min - ata) < 1e-12 * scale
    assert np.linalg.norm(fft_2n - ata) < 1e-12 * scale


def test_normal_operator_matches_dense_nudft_matrix(orc):
    # A^T A from the explicit non-uniform DFT matrix (independent of the Dirichlet closed form)
    rng = np.random.default_rng(7)
    N, nd = 6, 8
    th = rng.uniform(0, np.pi, 5)
    A = np.stack([nudft_forward(e.reshape(N, N), th, nd).ravel() for e in np.eye(N * N)], axis=1)
    x = rng.standard_normal((N, N))
    K = orc.kernel(N, th, nd)
    assert np.allclose(orc.toeplitz(x, K).ravel(), A.T @ (A @ x.ravel()), atol=1e-11)


def test_spectrum_real_and_operator_psd(orc):
    rng = np.random.default_rng(8)
    N, nd = 16, 16
    th = synth.angles(12, 2 * np.pi / 3)
    K = orc.kernel(N, th, nd)
    C = orc.circulant_spectrum(K, 2 * N)
    assert np.max(np.abs(C.imag)) < 1e-12 * np.max(np.abs(C.real))
    for _ in range(5):
        x = rng.standard_normal((N, N))
        assert np.sum(x * orc.toeplitz(x, K)) >= -1e-10


@pytest.mark.parametrize("nd", [16, 32])
def test_nyquist_drop_makes_operator_real(orc, nd):
    # keeping the Nyquist bin would give a complex projection for a real image; the
    # Dirichlet form (Nyquist dropped) agrees with the real part of the series without it
    t = np.linspace(-nd, nd, 101)
    k = np.arange(-(nd // 2 - 1), nd // 2)
    series = np.exp(2j * np.pi * np.outer(t, k) / nd).sum(axis=1)
    assert np.max(np.abs(series.imag)) < 1e-9
    assert np.allclose([orc.dirichlet(v, nd) for v in t], series.real, atol=1e-9)
