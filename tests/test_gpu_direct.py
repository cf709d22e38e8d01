"""The direct operators of Sec. 2 (Eqs. 3-4) through the C ABI: R by the type-2 NUFFT, R* by the
type-1 NUFFT, and the gradient R*(R x - g) + lambda grad Phi(x) computed without the Toeplitz
structure, against the FP64 oracle (brute-force Dirichlet sums) and against the Toeplitz
gradient of Sec. 2.1, which Sec. 3.1 compares it with (relative L2, FP32 arithmetic: 1e-5).
"""
import math

import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2603_28756_gb300 as tm  # noqa: E402

PRIOR = dict(p=1.2, q=2.0, c=0.01, sigma=0.1, lam=1.0)


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / np.linalg.norm(b))


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32).ravel()).cuda()


def host(t, shape):
    torch.cuda.synchronize()
    return t.double().cpu().numpy().reshape(shape)


@pytest.fixture(scope="module", params=[(64, 3, 37, math.pi), (128, 2, 45, 2 * math.pi / 3)],
                ids=["N64", "N128limited"])
def case(request, orc):
    N, S, na, span = request.param
    p = synth.volume(S=S, N=N, n_angles=na, n_ellipsoids=6, span=span, seed=15)
    ctx = tm.Context([tm.Group(N=N, angles=list(p.theta), n_slices=S, span=span)])
    rng = np.random.default_rng(16)
    x = synth.random_image(rng, (S, N, N), 0.5).astype(np.float64)
    return dict(N=N, S=S, na=na, p=p, ctx=ctx, g=p.sino.astype(np.float64), x=x)


def test_forward_matches_oracle(case, orc):
    S, N, na = case["S"], case["N"], case["na"]
    Rx = host(case["ctx"].forward(dev(case["x"])), (S, na, N))
    assert rel(Rx, orc.forward(case["x"], case["p"].theta, N)) < 1e-5


def test_adjoint_matches_oracle(case, orc):
    S, N = case["S"], case["N"]
    Rg = host(case["ctx"].adjoint(dev(case["g"])), (S, N, N))
    assert rel(Rg, orc.adjoint(case["g"], N, case["p"].theta)) < 1e-5


def test_forward_and_adjoint_are_adjoint(case):
    # <R x, g> = <x, R* g> for the two GPU operators (FP64 inner products of FP32 results)
    S, N, na = case["S"], case["N"], case["na"]
    Rx = host(case["ctx"].forward(dev(case["x"])), (S, na, N))
    Rg = host(case["ctx"].adjoint(dev(case["g"])), (S, N, N))
    a, b = float(np.sum(Rx * case["g"])), float(np.sum(case["x"] * Rg))
    assert abs(a - b) <= 1e-5 * abs(b)


def test_direct_gradient_matches_oracle_and_toeplitz(case, orc):
    S, N, p = case["S"], case["N"], case["p"]
    pr = orc.Prior(**PRIOR)
    ctx, x = case["ctx"], case["x"]
    G, F = ctx.gradient_direct(dev(x), dev(case["g"]), tm.Params(**PRIOR), want_objective=True)
    G = host(G, x.shape)
    K = orc.kernel(N, p.theta, N)
    atg = orc.adjoint(case["g"], N, p.theta)
    assert rel(G, orc.gradient(x, atg, K, pr)) < 1e-5
    Fo = orc.objective(x, atg, float(np.sum(case["g"] ** 2)), K, pr)
    assert abs(F - Fo) <= 1e-5 * abs(Fo)
    # the Toeplitz gradient of the same point (Sec. 3.1 compares the two)
    d_atg = ctx.build_operator(dev(case["g"]))
    Gt = host(ctx.gradient(dev(x), d_atg, tm.Params(**PRIOR)), x.shape)
    assert rel(G, Gt) < 1e-5


def test_n2048_limited_angle_direct_gradient(orc):
    """Two slices of 2048^2 with 128 angles over [0, 2 pi/3): R x at sampled (angle, bin) pairs
    and the direct gradient at sampled voxels against the oracle's sums, and the whole direct
    gradient against the Toeplitz gradient."""
    S, N, na, span = 2, 2048, 128, 2 * math.pi / 3
    p = synth.volume(S=S, N=N, n_angles=na, n_ellipsoids=6, span=span, seed=1003)
    ctx = tm.Context([tm.Group(N=N, angles=list(p.theta), n_slices=S, span=span)])
    rng = np.random.default_rng(17)
    x = synth.random_image(rng, (S, N, N), 0.5)
    d_x, d_g = dev(x), dev(p.sino)
    Rx = host(ctx.forward(d_x), (S, na, N))
    rmax = np.abs(Rx).max()
    for z, a, m in [(0, 0, 0), (1, na - 1, N - 1), (0, 37, N // 2), (1, 90, 301), (0, 64, 1700)]:
        assert abs(Rx[z, a, m] - orc.forward_point(x[z].astype(np.float64), p.theta[a], N, m)) <= 1e-5 * rmax
    pr = orc.Prior(**PRIOR)
    G = host(ctx.gradient_direct(d_x, d_g, tm.Params(**PRIOR)), (S, N, N))
    d_atg = ctx.build_operator(d_g)
    Gt = host(ctx.gradient(d_x, d_atg, tm.Params(**PRIOR)), (S, N, N))
    assert rel(G, Gt) < 1e-5
    K = orc.kernel(N, p.theta, N)
    g = p.sino.astype(np.float64)
    gscale = np.sqrt(np.mean(G ** 2))
    x64 = x.astype(np.float64)
    for z, r, c in [(0, 0, 0), (1, N - 1, N - 1), (0, N // 2, N // 2), (1, 700, 1500), (0, 1999, 3)]:
        ref = (orc.normal_point(x64[z], K, r, c) - orc.adjoint_point(g[z], N, p.theta, r, c)
               + orc.prior_point(x64, pr, z, r, c))
        assert abs(G[z, r, c] - ref) <= 1e-5 * gscale
