"""Seeded synthetic inputs shared by the oracle tests, the GPU tests and the benchmark.

This module only makes data: random ellipse / ellipsoid phantoms, their exact
parallel-beam line integrals (the textbook ellipse projection, Kak & Slaney ch. 3),
detector noise and angle sets.  It holds none of the reconstruction method's
arithmetic and imports neither the oracle nor the CUDA package.

Geometry matches the rest of the code: pixel (row r, col c) of an N x N slice sits at
(x, y) = (c - N/2, r - N/2); detector bin m of n_d sits at s = m - n_d/2; angle theta
projects onto s = x cos(theta) + y sin(theta).

The paper's TomoBank nano-CT projections are not available here; these phantoms
stand in for them with the shapes of the paper's workloads (Sec. 3).
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np


@dataclass
class Ellipses:
    """n ellipses: centre (x0, y0), semi-axes (a, b), rotation phi, density rho."""

    x0: np.ndarray
    y0: np.ndarray
    a: np.ndarray
    b: np.ndarray
    phi: np.ndarray
    rho: np.ndarray


@dataclass
class Ellipsoids:
    """n ellipsoids rotated about the slice axis only: in-plane ellipse + z centre and semi-axis."""

    plane: Ellipses
    z0: np.ndarray
    cz: np.ndarray


def angles(n: int, span: float = np.pi) -> np.ndarray:
    """n equally spaced projection angles a * span / n, a = 0..n-1 (FP64)."""
    return np.arange(n, dtype=np.float64) * (span / n)


def random_ellipses(rng: np.random.Generator, n: int, N: int) -> Ellipses:
    """Centres uniform in the disc of radius 0.55 N/2, semi-axes U[0.05, 0.35] N/2,
    rotation U[0, pi), density U[0, 1]; each shape shrunk to stay inside 0.95 N/2."""
    R = N / 2.0
    rad = 0.55 * R * np.sqrt(rng.uniform(0, 1, n))
    ang = rng.uniform(0, 2 * np.pi, n)
    x0, y0 = rad * np.cos(ang), rad * np.sin(ang)
    a = rng.uniform(0.05, 0.35, n) * R
    b = rng.uniform(0.05, 0.35, n) * R
    phi = rng.uniform(0, np.pi, n)
    rho = rng.uniform(0, 1, n)
    limit = 0.95 * R
    reach = rad + np.maximum(a, b)
    s = np.minimum(1.0, (limit - rad) / np.maximum(reach - rad, 1e-12))
    return Ellipses(x0, y0, a * s, b * s, phi, rho)


def random_ellipsoids(rng: np.random.Generator, n: int, N: int, S: int) -> Ellipsoids:
    """In-plane parameters as ``random_ellipses``; z semi-axis U[0.1, 0.5] S, z centre U[0, S)."""
    plane = random_ellipses(rng, n, N)
    cz = rng.uniform(0.1, 0.5, n) * S
    z0 = rng.uniform(0, S, n)
    return Ellipsoids(plane, z0, cz)


def ellipsoid_slice(e: Ellipsoids, z: float) -> Ellipses:
    """Cross-section at height z: each ellipse scaled by sqrt(1 - ((z - z0)/cz)^2), absent outside."""
    t = (z - e.z0) / e.cz
    f = np.sqrt(np.clip(1.0 - t * t, 0.0, None))
    p = e.plane
    keep = f > 0
    return Ellipses(p.x0[keep], p.y0[keep], p.a[keep] * f[keep], p.b[keep] * f[keep], p.phi[keep], p.rho[keep])


def rasterize(e: Ellipses, N: int, supersample: int = 4) -> np.ndarray:
    """Pixel-area average of the summed ellipse densities (supersample^2 points per pixel)."""
    k = supersample
    off = (np.arange(k) + 0.5) / k - 0.5
    img = np.zeros((N, N))
    cc = np.arange(N) - N // 2
    for i in range(e.x0.size):
        cph, sph = np.cos(e.phi[i]), np.sin(e.phi[i])
        acc = np.zeros((N, N))
        for oy in off:
            for ox in off:
                X = cc[None, :] + ox - e.x0[i]
                Y = cc[:, None] + oy - e.y0[i]
                u = X * cph + Y * sph
                v = -X * sph + Y * cph
                acc += (u / e.a[i]) ** 2 + (v / e.b[i]) ** 2 <= 1.0
        img += e.rho[i] * acc / (k * k)
    return img


def ellipse_projections(e: Ellipses, theta: np.ndarray, nd: int) -> np.ndarray:
    """Exact line integrals at the bin centres: p(s, th) = 2 rho a b sqrt(al^2 - s'^2) / al^2,
    al^2 = a^2 cos^2(th - phi) + b^2 sin^2(th - phi), s' = s - x0 cos th - y0 sin th."""
    s = np.arange(nd) - nd / 2.0
    g = np.zeros((theta.size, nd))
    for i in range(e.x0.size):
        d = theta - e.phi[i]
        al2 = (e.a[i] * np.cos(d)) ** 2 + (e.b[i] * np.sin(d)) ** 2
        sp = s[None, :] - (e.x0[i] * np.cos(theta) + e.y0[i] * np.sin(theta))[:, None]
        inside = al2[:, None] - sp * sp
        g += np.where(inside > 0, 2.0 * e.rho[i] * e.a[i] * e.b[i] * np.sqrt(np.clip(inside, 0, None)) / al2[:, None], 0.0)
    return g


def gaussian_blob(N: int, x0: float, y0: float, width: float) -> np.ndarray:
    """exp(-|x - x0|^2 / (2 width^2)) sampled at the pixel centres."""
    cc = np.arange(N) - N // 2
    return np.exp(-(((cc[None, :] - x0) ** 2) + ((cc[:, None] - y0) ** 2)) / (2.0 * width * width))


def gaussian_blob_projections(theta: np.ndarray, nd: int, x0: float, y0: float, width: float) -> np.ndarray:
    """Exact line integrals of the blob: sqrt(2 pi) width exp(-(s - t0)^2 / (2 width^2))."""
    s = np.arange(nd) - nd / 2.0
    t0 = x0 * np.cos(theta) + y0 * np.sin(theta)
    return np.sqrt(2 * np.pi) * width * np.exp(-((s[None, :] - t0[:, None]) ** 2) / (2 * width * width))


def poisson_noise(rng: np.random.Generator, g: np.ndarray, photons: float) -> np.ndarray:
    """Transmission counts y ~ Poisson(I0 exp(-kappa g)), kappa = 3 / max g; returns -ln(max(y,1)/I0)/kappa."""
    kappa = 3.0 / max(float(g.max()), 1e-12)
    y = rng.poisson(photons * np.exp(-kappa * g))
    return -np.log(np.maximum(y, 1) / photons) / kappa


def gaussian_noise(rng: np.random.Generator, g: np.ndarray, rel: float) -> np.ndarray:
    """g + N(0, (rel * max g)^2)."""
    return g + rng.normal(0.0, rel * float(g.max()), g.shape)


@dataclass
class Problem:
    """One synthetic reconstruction problem: sinogram (S, n_angles, nd) FP32, angles FP64."""

    N: int
    nd: int
    theta: np.ndarray
    span: float
    sino: np.ndarray
    truth: np.ndarray | None


def single_slice(N: int = 128, n_angles: int = 90, n_ellipses: int = 10, photons: float = 1e4,
                 seed: int = 1001, with_truth: bool = True) -> Problem:
    """One slice of random ellipses, uniform angles in [0, pi), Poisson noise (the
    128 x 128, 90-angle plain single-slice workload at the defaults)."""
    rng = np.random.default_rng(seed)
    e = random_ellipses(rng, n_ellipses, N)
    th = angles(n_angles)
    g = ellipse_projections(e, th, N)
    g = poisson_noise(np.random.default_rng(seed + 500), g, photons)
    truth = rasterize(e, N) if with_truth else None
    return Problem(N, N, th, np.pi, g.astype(np.float32)[None], truth if truth is None else truth[None])


def volume(S: int = 64, N: int = 1024, n_angles: int = 256, n_ellipsoids: int = 20, span: float = np.pi,
           rel_noise: float = 0.01, seed: int = 1002, with_truth: bool = False) -> Problem:
    """S slices of a random-ellipsoid volume with Gaussian noise of rel_noise * max
    (64 x 1024^2, 256 angles at the defaults)."""
    rng = np.random.default_rng(seed)
    e = random_ellipsoids(rng, n_ellipsoids, N, S)
    th = angles(n_angles, span)
    g = np.zeros((S, n_angles, N), dtype=np.float64)
    truth = np.zeros((S, N, N)) if with_truth else None
    for z in range(S):
        es = ellipsoid_slice(e, z + 0.5)
        g[z] = ellipse_projections(es, th, N)
        if with_truth:
            truth[z] = rasterize(es, N, 2)
    nrng = np.random.default_rng(seed + 500)
    g = g + nrng.normal(0.0, rel_noise * float(g.max()), g.shape)
    return Problem(N, N, th, span, g.astype(np.float32), truth)


def random_image(rng: np.random.Generator, shape, scale: float = 1.0) -> np.ndarray:
    """Uniform [0, scale) test image (FP32) for operator parity checks."""
    return (rng.uniform(0.0, scale, shape)).astype(np.float32)
