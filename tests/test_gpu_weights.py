"""The per-angle weighted data term through the C ABI (tmbir_set_angle_weights): the weighted
kernel K_w, R* W g, lambda_max, the gradient, the iterations and the direct gradient against the
FP64 oracle's weighted functions (whose pins are in test_oracle_weights.py)."""
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


@pytest.fixture(scope="module", params=[(64, 3, 37, math.pi), (128, 2, 45, 2 * math.pi / 3)], ids=["N64", "N128limited"])
def wp(request, orc):
    N, S, na, span = request.param
    p = synth.volume(S=S, N=N, n_angles=na, n_ellipsoids=6, span=span, seed=31)
    rng = np.random.default_rng(32)
    w = rng.uniform(0.2, 1.0, na)
    w[3] = 0.0  # a view left out entirely
    ctx = tm.Context([tm.Group(N=N, angles=list(p.theta), n_slices=S, span=span)])
    ctx.set_angle_weights(0, list(w))
    d_sino = dev(p.sino)
    d_atg = ctx.build_operator(d_sino)
    g = p.sino.astype(np.float64)
    K = orc.kernel_weighted(N, p.theta, N, w)
    atg = orc.adjoint_weighted(g, N, p.theta, w)
    x = synth.random_image(rng, (S, N, N), 0.5).astype(np.float64)
    return dict(N=N, S=S, p=p, w=w, ctx=ctx, d_sino=d_sino, d_atg=d_atg, g=g, K=K, atg=atg, x=x)


def test_weighted_kernel_and_adjoint(wp):
    K = host(wp["ctx"].kernel(0), wp["K"].shape)
    assert np.max(np.abs(K - wp["K"])) <= 1e-10 * np.max(np.abs(wp["K"]))
    assert rel(host(wp["d_atg"], wp["atg"].shape), wp["atg"]) < 1e-6


def test_weighted_lambda_max_gradient_and_objective(wp, orc):
    lam = wp["ctx"].lambda_max()[0]
    ref = orc.power_lambda_max(wp["K"], wp["N"])
    assert abs(lam - ref) <= 1e-5 * ref
    pr = orc.Prior(**PRIOR)
    G = host(wp["ctx"].gradient(dev(wp["x"]), wp["d_atg"], tm.Params(**PRIOR)), wp["x"].shape)
    assert rel(G, orc.gradient(wp["x"], wp["atg"], wp["K"], pr)) < 1e-5
    F = wp["ctx"].objective(dev(wp["x"]), wp["d_atg"], tm.Params(**PRIOR))
    Fo = orc.objective_direct_weighted(wp["x"], wp["g"], wp["p"].theta, pr, wp["w"])
    assert abs(F - Fo) <= 1e-5 * abs(Fo)


def test_weighted_iterations_follow_oracle(wp, orc):
    pr = orc.Prior(**PRIOR)
    iters = 30
    x = torch.zeros(wp["x"].size, dtype=torch.float32, device="cuda")
    st = wp["ctx"].reconstruct(x, wp["d_atg"], tm.Params(**PRIOR, max_iter=iters))
    L = orc.lipschitz(wp["K"], wp["N"], pr)
    assert st.iterations == iters and abs(st.L - L) <= 1e-5 * L
    ref = orc.nesterov(np.zeros(wp["x"].shape), wp["atg"], orc.gtg_weighted(wp["g"], wp["w"]), wp["K"], pr, L, iters)
    assert rel(host(x, wp["x"].shape), ref) < 1e-4


def test_weighted_direct_gradient(wp, orc):
    pr = orc.Prior(**PRIOR)
    G, F = wp["ctx"].gradient_direct(dev(wp["x"]), wp["d_sino"], tm.Params(**PRIOR), want_objective=True)
    G = host(G, wp["x"].shape)
    assert rel(G, orc.gradient(wp["x"], wp["atg"], wp["K"], pr)) < 1e-5
    Fo = orc.objective_direct_weighted(wp["x"], wp["g"], wp["p"].theta, pr, wp["w"])
    assert abs(F - Fo) <= 1e-5 * abs(Fo)


def test_weights_reset_and_errors(wp):
    ctx = wp["ctx"]
    with pytest.raises(tm.TmbirError) as e:
        ctx.set_angle_weights(0, [2.0] * len(wp["w"]))
    assert e.value.code == -1
    with pytest.raises(tm.TmbirError) as e:
        ctx.set_angle_weights(1, list(wp["w"]))
    assert e.value.code == -1
    # back to unit weights: the unweighted operator of a fresh context
    ctx.set_angle_weights(0, None)
    a1 = ctx.build_operator(wp["d_sino"])
    plain = tm.Context([tm.Group(N=wp["N"], angles=list(wp["p"].theta), n_slices=wp["S"], span=wp["p"].span)])
    a0 = plain.build_operator(wp["d_sino"])
    torch.cuda.synchronize()
    assert torch.equal(a1, a0) and torch.equal(ctx.kernel(0), plain.kernel(0))
    ctx.set_angle_weights(0, list(wp["w"]))
    ctx.build_operator(wp["d_sino"], wp["d_atg"])


def test_weighted_kernel_by_direct_sums_at_2560(orc):
    """At N = 2560 the kernel is summed directly (no NUFFT): sampled offsets against the oracle."""
    N, na = 2560, 6
    theta = np.linspace(0.0, math.pi, na, endpoint=False) + 0.1
    w = np.array([1.0, 0.5, 0.0, 0.25, 0.75, 0.9])
    ctx = tm.Context([tm.Group(N=N, angles=list(theta), n_slices=1)])
    ctx.set_angle_weights(0, list(w))
    ctx.build_operator(torch.zeros(na * N, dtype=torch.float32, device="cuda"))
    K = host(ctx.kernel(0), (2 * N - 1, 2 * N - 1))
    ref = orc.kernel_weighted(N, theta, N, w)
    scale = np.max(np.abs(ref))
    for dy, dx in [(0, 0), (1, 0), (0, 7), (-300, 41), (1000, -2000), (N - 1, -(N - 1)), (17, 2559)]:
        assert abs(K[dy + N - 1, dx + N - 1] - ref[dy + N - 1, dx + N - 1]) <= 1e-10 * scale, (dy, dx)
