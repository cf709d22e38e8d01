"""FP64 CPU oracle for the Toeplitz-accelerated MBIR gradient path.

TEST INFRASTRUCTURE ONLY.  Only the test suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  It shares no code with the
CUDA path (it never imports ``paper_2603_28756_gb300``) and nothing in the product
path may call it.

What each function computes, with the passage of the paper it follows:

* ``forward`` / ``adjoint``: the Radon transform through the central-slice
  construction R = F^-1 NUFFT2 and its adjoint (Sec. 2, Eqs. 3-4), evaluated by the
  brute-force Dirichlet sum in ``radon.c``.
* ``kernel``: the point-spread kernel K = NUFFT1(ones) of Sec. 2.1 by direct sums.
* ``normal_direct``: A^T A x = K (*) x (Eq. 8) by the O(N^4) convolution sum.
* ``toeplitz``: the same product by zero-padded FFT convolution (Eq. 9), padded to
  the paper's minimal 2N-1 (the CUDA path pads to 2N).
* ``prior``: the qGGMRF prior (Sec. 2, Eq. 5), see ``prior.c``.
* ``objective`` / ``gradient``: Eq. 5 (direct) and Eqs. 10-11 (Toeplitz form) with
  the sign of the prior term in Eq. 6 read as "+": the gradient of Eq. 5.
* ``lipschitz``: the step constant L of Eq. 6 (not given in the paper; read as
  1.01 x the largest eigenvalue of A^T A from 100 power steps started at the
  all-ones image, plus lambda * 2 * max rho'' for the prior, max rho'' = 2/sigma^2
  when q = 2).
* ``nesterov``: the fast gradient method with restart of Sec. 2 (accelerated
  Nesterov steps with momentum t_{k+1} = (1 + sqrt(1 + 4 t_k^2))/2, restarted when
  <grad F(y_k), x_{k+1} - x_k> > 0).  ``gradient_descent`` is the plain Eq. 6 step.
* ``ramp_filter`` / ``fbp``: Eqs. 12-14, f0 = dtheta * A^T (h (*) g).
* ``lanczos_up`` / ``downsample_sino``: Eqs. 16-17 and the projection subsampling
  of Sec. 2.3.
* ``cnn_forward`` / ``cnn_backward``: the learned warm-start refiner (not in the paper;
  four 3x3 convolutions 1 -> 32 -> 32 -> 32 -> 1 with ReLU), see ``cnn.c``.

Parity unpinned: none of these; the pins live in ``tests/test_oracle_*.py``.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liboracle.so")
_SOURCES = ["radon.c", "prior.c", "interp.c", "cnn.c"]
_lib = None


def build(force: bool = False) -> str:
    """Compile the C part of the oracle with gcc (FP64, OpenMP) into oracle/_build."""
    srcs = [os.path.join(_HERE, s) for s in _SOURCES if os.path.exists(os.path.join(_HERE, s))]
    if not force and os.path.exists(_SO):
        so_t = os.path.getmtime(_SO)
        if all(os.path.getmtime(s) <= so_t for s in srcs):
            return _SO
    os.makedirs(_BUILD, exist_ok=True)
    tmp = _SO + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-fPIC", "-shared", "-fopenmp", "-std=c11", "-o", tmp] + srcs + ["-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _SO)
    return _SO


def lib():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        dp = ctypes.POINTER(ctypes.c_double)
        i = ctypes.c_int
        d = ctypes.c_double
        L = _lib
        L.orc_dirichlet.restype = d
        L.orc_dirichlet.argtypes = [d, i]
        L.orc_forward.argtypes = [dp, i, dp, i, i, dp]
        L.orc_adjoint.argtypes = [dp, i, dp, i, i, dp]
        L.orc_kernel.argtypes = [i, dp, i, i, dp]
        L.orc_normal_direct.argtypes = [dp, i, dp, dp]
        L.orc_normal_point.restype = d
        L.orc_normal_point.argtypes = [dp, i, dp, i, i]
        L.orc_adjoint_point.restype = d
        L.orc_adjoint_point.argtypes = [dp, i, dp, i, i, i, i]
        L.orc_forward_point.restype = d
        L.orc_forward_point.argtypes = [dp, i, d, i, i]
        L.orc_rho.restype = d
        L.orc_rho.argtypes = [d, d, d, d, d]
        L.orc_drho.restype = d
        L.orc_drho.argtypes = [d, d, d, d, d]
        L.orc_neighbour_weight.restype = d
        L.orc_neighbour_weight.argtypes = [i, i, i]
        L.orc_prior.argtypes = [dp, i, i, d, d, d, d, d, dp, dp]
        L.orc_ramp_filter.argtypes = [dp, i, i, dp]
        L.orc_lanczos.restype = d
        L.orc_lanczos.argtypes = [d, i]
        L.orc_lanczos_up.argtypes = [dp, i, i, dp, dp]
        L.orc_downsample_sino.argtypes = [dp, i, i, i, i, dp]
        L.orc_cnn_param_count.restype = i
        L.orc_cnn_param_count.argtypes = []
        L.orc_cnn_forward.argtypes = [dp, i, i, i, dp, dp]
        L.orc_cnn_backward.argtypes = [dp, i, i, i, dp, dp, dp, dp]
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def set_threads(n: int) -> None:
    """Number of OpenMP threads the C part uses (0 keeps the runtime default)."""
    if n > 0:
        os.environ["OMP_NUM_THREADS"] = str(n)


@dataclass(frozen=True)
class Prior:
    """qGGMRF parameters: exponents p <= q, threshold c, scale sigma, weight lambda."""

    p: float = 1.2
    q: float = 2.0
    c: float = 0.01
    sigma: float = 0.1
    lam: float = 1.0


# ----------------------------------------------------------------------------- Radon


def dirichlet(t: float, nd: int) -> float:
    return lib().orc_dirichlet(float(t), int(nd))


def forward(x, theta, nd: int) -> np.ndarray:
    """A x for one slice (N, N) or a stack (S, N, N); returns (n_angles, nd) or (S, n_angles, nd)."""
    x = _f64(x)
    th = _f64(theta)
    if x.ndim == 3:
        return np.stack([forward(s, th, nd) for s in x])
    N = x.shape[0]
    g = np.zeros((th.size, nd))
    lib().orc_forward(_p(x), N, _p(th), th.size, nd, _p(g))
    return g


def adjoint(g, N: int, theta) -> np.ndarray:
    """A^T g for one sinogram (n_angles, nd) or a stack (S, n_angles, nd)."""
    g = _f64(g)
    th = _f64(theta)
    if g.ndim == 3:
        return np.stack([adjoint(s, N, th) for s in g])
    x = np.zeros((N, N))
    lib().orc_adjoint(_p(g), N, _p(th), th.size, g.shape[1], _p(x))
    return x


def kernel(N: int, theta, nd: int) -> np.ndarray:
    """K(dx, dy) on [-(N-1), N-1]^2, indexed K[dy + N-1, dx + N-1]."""
    th = _f64(theta)
    K = np.zeros((2 * N - 1, 2 * N - 1))
    lib().orc_kernel(N, _p(th), th.size, nd, _p(K))
    return K


def kernel_weighted(N: int, theta, nd: int, w) -> np.ndarray:
    """K_w = sum_a w_a K_a: the kernel of R* W R for per-angle data-term weights w_a, written as the
    weighted sum of the kernels of each angle alone (each K_a the Dirichlet sum of Sec. 2.1)."""
    th = _f64(theta)
    w = _f64(w)
    K = np.zeros((2 * N - 1, 2 * N - 1))
    for a in range(th.size):
        if w[a] != 0.0:
            K += w[a] * kernel(N, th[a:a + 1], nd)
    return K


def adjoint_weighted(g, N: int, theta, w) -> np.ndarray:
    """R* W g: every projection g_a scaled by its weight w_a, then the adjoint."""
    g = _f64(g)
    return adjoint(g * _f64(w).reshape((1,) * (g.ndim - 2) + (-1, 1)), N, theta)


def gtg_weighted(g, w) -> float:
    """g . W g = sum_a w_a ||g_a||^2 (the objective takes its half)."""
    g = _f64(g)
    return float(np.sum(_f64(w).reshape((1,) * (g.ndim - 2) + (-1, 1)) * g * g))


def objective_direct_weighted(x, g, theta, pr: Prior, w) -> float:
    """1/2 sum_a w_a ||A_a x - g_a||^2 + lambda Phi(x), A by brute force."""
    x = _f64(x)
    g = _f64(g)
    r = forward(x, theta, g.shape[-1]) - g
    return 0.5 * float(np.sum(_f64(w).reshape((1,) * (g.ndim - 2) + (-1, 1)) * r * r)) + prior(x, pr)[1]


def normal_direct(x, K) -> np.ndarray:
    """sum_i K(x_j - x_i) x_i by the direct sum, for a slice or a stack."""
    x = _f64(x)
    K = _f64(K)
    if x.ndim == 3:
        return np.stack([normal_direct(s, K) for s in x])
    N = x.shape[0]
    z = np.zeros_like(x)
    lib().orc_normal_direct(_p(x), N, _p(K), _p(z))
    return z


def normal_point(x, K, r: int, c: int) -> float:
    """(K (*) x)[r, c] of one slice by the direct sum."""
    x = _f64(x)
    K = _f64(K)
    return lib().orc_normal_point(_p(x), x.shape[0], _p(K), r, c)


def adjoint_point(g, N: int, theta, r: int, c: int) -> float:
    """(A^T g)[r, c] of one sinogram by the direct sum."""
    g = _f64(g)
    th = _f64(theta)
    return lib().orc_adjoint_point(_p(g), N, _p(th), th.size, g.shape[1], r, c)


def forward_point(x, theta_a: float, nd: int, m: int) -> float:
    """(A x)(a, m) of one slice at one angle and bin by the direct sum (Eq. 3 in closed form)."""
    x = _f64(x)
    return lib().orc_forward_point(_p(x), x.shape[0], float(theta_a), nd, m)


def prior_point(x, pr: Prior, z: int, r: int, c: int) -> float:
    """lambda * dPhi/dx at voxel (z, r, c) of a volume, from its 3x3x3 neighbourhood only."""
    x = _f64(x)
    v = x.reshape((1,) + x.shape) if x.ndim == 2 else x
    S, N = v.shape[0], v.shape[1]
    g = 0.0
    for dz in (-1, 0, 1):
        for dy in (-1, 0, 1):
            for dx in (-1, 0, 1):
                if (dz, dy, dx) == (0, 0, 0):
                    continue
                z2, r2, c2 = z + dz, r + dy, c + dx
                if 0 <= z2 < S and 0 <= r2 < N and 0 <= c2 < N:
                    g += neighbour_weight(dz, dy, dx) * drho(v[z, r, c] - v[z2, r2, c2], pr)
    return pr.lam * g


def circulant_spectrum(K, M: int | None = None) -> np.ndarray:
    """FFT of K embedded circulantly in an M x M grid (Eq. 9); M defaults to 2N-1."""
    K = _f64(K)
    N = (K.shape[0] + 1) // 2
    M = 2 * N - 1 if M is None else M
    assert M >= 2 * N - 1
    C = np.zeros((M, M))
    d = np.arange(-(N - 1), N)
    C[np.ix_(d % M, d % M)] = K
    return np.fft.fft2(C)


def toeplitz(x, K, Chat=None) -> np.ndarray:
    """Res_{NxN} F^-1 (F K . F Pad x), Eq. 9, for a slice or a stack."""
    x = _f64(x)
    if Chat is None:
        Chat = circulant_spectrum(K)
    M = Chat.shape[0]
    N = x.shape[-1]
    pad = np.zeros(x.shape[:-2] + (M, M))
    pad[..., :N, :N] = x
    z = np.fft.ifft2(Chat * np.fft.fft2(pad))
    return z.real[..., :N, :N].copy()


# ----------------------------------------------------------------------------- prior


def neighbour_weight(dz: int, dy: int, dx: int) -> float:
    return lib().orc_neighbour_weight(dz, dy, dx)


def rho(d: float, pr: Prior) -> float:
    return lib().orc_rho(float(d), pr.p, pr.q, pr.c, pr.sigma)


def drho(d: float, pr: Prior) -> float:
    return lib().orc_drho(float(d), pr.p, pr.q, pr.c, pr.sigma)


def prior(x, pr: Prior):
    """(lambda * grad Phi(x), lambda * Phi(x)) for a slice (N, N) or a volume (S, N, N)."""
    x = _f64(x)
    shape = x.shape
    v = x.reshape((1,) + shape) if x.ndim == 2 else x
    S, N = v.shape[0], v.shape[1]
    grad = np.zeros_like(v)
    phi = np.zeros(1)
    lib().orc_prior(_p(v), S, N, pr.p, pr.q, pr.c, pr.sigma, pr.lam, _p(grad), _p(phi))
    return grad.reshape(shape), float(phi[0])


# ----------------------------------------------------------------------------- objective


def objective_direct(x, g, theta, pr: Prior) -> float:
    """Eq. 5: 1/2 ||A x - g||^2 + lambda Phi(x), A by brute force."""
    x = _f64(x)
    g = _f64(g)
    r = forward(x, theta, g.shape[-1]) - g
    return 0.5 * float(np.sum(r * r)) + prior(x, pr)[1]


def objective(x, atg, gtg: float, K, pr: Prior, Chat=None) -> float:
    """Eq. 10 plus the prior: 1/2 x.(K*x) - x.A^T g + 1/2 g.g + lambda Phi(x)."""
    x = _f64(x)
    z = toeplitz(x, K, Chat)
    return 0.5 * float(np.sum(x * z)) - float(np.sum(x * atg)) + 0.5 * gtg + prior(x, pr)[1]


def gradient(x, atg, K, pr: Prior, Chat=None) -> np.ndarray:
    """Eq. 11 plus the prior: K*x - A^T g + lambda grad Phi(x)."""
    x = _f64(x)
    return toeplitz(x, K, Chat) - atg + prior(x, pr)[0]


def max_rho2(pr: Prior) -> float:
    """Largest rho'' of the potential; closed form 2/sigma^2 for q = 2 (attained at 0)."""
    if pr.q != 2.0:
        raise ValueError("closed-form curvature bound needs q = 2")
    return 2.0 / (pr.sigma * pr.sigma)


def power_lambda_max(K, N: int, steps: int = 100, Chat=None) -> float:
    """Largest eigenvalue of A^T A by power iteration from the all-ones image."""
    if Chat is None:
        Chat = circulant_spectrum(K)
    v = np.ones((N, N))
    v /= np.linalg.norm(v)
    lam = 0.0
    for _ in range(steps):
        w = toeplitz(v, K, Chat)
        lam = float(np.sum(v * w))
        v = w / np.linalg.norm(w)
    return lam


def lipschitz(K, N: int, pr: Prior, steps: int = 100, Chat=None) -> float:
    """L = 1.01 lambda_max(A^T A) + lambda * 2 * max rho'' (neighbour weights sum to 1)."""
    return 1.01 * power_lambda_max(K, N, steps, Chat) + pr.lam * 2.0 * max_rho2(pr)


# ----------------------------------------------------------------------------- optimisers


def nesterov(x0, atg, gtg: float, K, pr: Prior, L: float, iters: int, Chat=None, log=None, restart="gradient",
             nonneg=False):
    """Fast gradient method with adaptive restart (Sec. 2, which cites the restarted scheme
    without stating the test).

    t_0 = 1, x_{-1} = x_0.  Each step:
      t' = (1 + sqrt(1 + 4 t^2)) / 2,  beta = (t - 1) / t'
      y = x + beta (x - x_prev)
      G = K*y - A^T g + lambda grad Phi(y)
      x_new = y - G / L
      restart (t' = 1) when
        "gradient": <G, x_new - x> > 0
        "function": F(y_k) > F(y_{k-1})
        "none":     never
    ``log`` (a list) receives (F(y_k), <G,x_new-x>, restarted) per step.  With ``nonneg`` every
    x_new is projected onto x >= 0 (max(., 0)) before the restart test: the projected fast
    gradient method on Eq. 5 restricted to non-negative images, a variant the paper does not use.
    """
    if restart not in ("gradient", "function", "none"):
        raise ValueError(restart)
    if Chat is None:
        Chat = circulant_spectrum(K)
    x = _f64(x0).copy()
    x_prev = x.copy()
    t = 1.0
    F_prev = None
    for _ in range(iters):
        t_next = 0.5 * (1.0 + math.sqrt(1.0 + 4.0 * t * t))
        beta = (t - 1.0) / t_next
        y = x + beta * (x - x_prev)
        z = toeplitz(y, K, Chat)
        gp, phi = prior(y, pr)
        G = z - atg + gp
        x_new = y - G / L
        if nonneg:
            x_new = np.maximum(x_new, 0.0)
        dot = float(np.sum(G * (x_new - x)))
        F = 0.5 * float(np.sum(y * z)) - float(np.sum(y * atg)) + 0.5 * gtg + phi
        if restart == "gradient":
            restarted = dot > 0.0
        elif restart == "function":
            restarted = F_prev is not None and F > F_prev
        else:
            restarted = False
        if restarted:
            t_next = 1.0
        if log is not None:
            log.append((F, dot, restarted))
        F_prev = F
        x_prev, x, t = x, x_new, t_next
    return x


def gradient_descent(x0, atg, K, pr: Prior, L: float, iters: int, Chat=None):
    """Plain Eq. 6 (with the '+' sign on the prior gradient): x <- x - grad F(x) / L."""
    if Chat is None:
        Chat = circulant_spectrum(K)
    x = _f64(x0).copy()
    for _ in range(iters):
        x = x - gradient(x, atg, K, pr, Chat) / L
    return x


# ----------------------------------------------------------------------------- warm start / levels


def ramp_filter(g) -> np.ndarray:
    """Eq. 12 with the unit-pitch Ram-Lak kernel, per projection row (linear convolution)."""
    g = _f64(g)
    if g.ndim == 3:
        return np.stack([ramp_filter(s) for s in g])
    out = np.zeros_like(g)
    lib().orc_ramp_filter(_p(g), g.shape[0], g.shape[1], _p(out))
    return out


def fbp(g, N: int, theta, angular_range: float) -> np.ndarray:
    """Eq. 14 with the quadrature weight: f0 = (angular_range / n_angles) A^T (h (*) g)."""
    th = _f64(theta)
    return (angular_range / th.size) * adjoint(ramp_filter(g), N, th)


def lanczos(x: float, a: int = 3) -> float:
    return lib().orc_lanczos(float(x), int(a))


def lanczos_up(x) -> np.ndarray:
    """x2 separable Lanczos-3 upsampling (Eqs. 16-17) of a slice or a stack."""
    x = _f64(x)
    shape = x.shape
    v = x.reshape((1,) + shape) if x.ndim == 2 else x
    S, Nc = v.shape[0], v.shape[1]
    out = np.zeros((S, 2 * Nc, 2 * Nc))
    tmp = np.zeros((S, Nc, 2 * Nc))
    lib().orc_lanczos_up(_p(v), S, Nc, _p(out), _p(tmp))
    return out[0] if x.ndim == 2 else out


def downsample_sino(g, factor: int) -> np.ndarray:
    """Every factor-th detector bin about the centre bin, divided by factor (Sec. 2.3)."""
    g = _f64(g)
    shape = g.shape
    v = g.reshape((1,) + shape) if g.ndim == 2 else g
    S, na, nd = v.shape
    out = np.zeros((S, na, nd // factor))
    lib().orc_downsample_sino(_p(v), S, na, nd, factor, _p(out))
    return out[0] if g.ndim == 2 else out


# ----------------------------------------------------------------------------- learned warm start


def cnn_param_count() -> int:
    return lib().orc_cnn_param_count()


def cnn_forward(x, params) -> np.ndarray:
    """net(x) for a batch (B, H, W) or one image (H, W)."""
    x = _f64(x)
    v = x.reshape((1,) + x.shape) if x.ndim == 2 else x
    p = _f64(params)
    assert p.size == cnn_param_count()
    out = np.zeros_like(v)
    lib().orc_cnn_forward(_p(v), v.shape[0], v.shape[1], v.shape[2], _p(p), _p(out))
    return out.reshape(x.shape)


def cnn_backward(x, params, gout):
    """(d/dparams, d/dx) of sum(gout * net(x))."""
    x = _f64(x)
    v = x.reshape((1,) + x.shape) if x.ndim == 2 else x
    p = _f64(params)
    g = _f64(gout).reshape(v.shape)
    gp = np.zeros_like(p)
    gx = np.zeros_like(v)
    lib().orc_cnn_backward(_p(v), v.shape[0], v.shape[1], v.shape[2], _p(p), _p(g), _p(gp), _p(gx))
    return gp, gx.reshape(x.shape)


def cnn_layer_slices():
    """(weight slice, bias slice, cin, cout) of each layer in the flat parameter vector."""
    out, off = [], 0
    for cin, cout in ((1, 32), (32, 32), (32, 32), (32, 1)):
        nw = cout * cin * 9
        out.append((slice(off, off + nw), slice(off + nw, off + nw + cout), cin, cout))
        off += nw + cout
    return out
