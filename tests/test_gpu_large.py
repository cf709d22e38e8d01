"""Parity at large sizes.

* The workload bench.py times: 64 slices of 1024^2, 256 angles over [0, pi), 20 ellipsoids.
* The finest level of the hierarchical geometry: 2048^2 slices seen under 128 angles over
  [0, 2 pi/3) (missing wedge), two slices compared in full and the full 512-slice volume on
  sampled outputs.

The oracle evaluates sampled outputs one by one (R*g, K (*) x, the prior gradient and the FBP
start at a pixel); the kernel K and, at 2048^2 with two slices, whole results are compared in
full.  Tolerances as in test_gpu_parity.py.
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


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32).ravel()).cuda()


def host(t, shape):
    torch.cuda.synchronize()
    return t.double().cpu().numpy().reshape(shape)


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / np.linalg.norm(b))


def samples(rng, S, N, n):
    """n voxels: the corners and edges of the volume and random interior ones."""
    pts = [(0, 0, 0), (S - 1, N - 1, N - 1), (0, N - 1, 0), (S - 1, 0, N - 1), (S // 2, N // 2, N // 2)]
    while len(pts) < n:
        pts.append((int(rng.integers(S)), int(rng.integers(N)), int(rng.integers(N))))
    return pts


@pytest.fixture(scope="module")
def bench_case(orc):
    S, N, na = 64, 1024, 256
    p = synth.volume(S=S, N=N, n_angles=na, n_ellipsoids=20, seed=1002)
    ctx = tm.Context([tm.Group(N=N, angles=list(p.theta), n_slices=S)])
    sino = dev(p.sino)
    atg = ctx.build_operator(sino)
    K = orc.kernel(N, p.theta, N)
    return dict(S=S, N=N, p=p, ctx=ctx, sino=sino, atg=atg, K=K)


def test_bench_workload_setup(bench_case, orc):
    c = bench_case
    S, N, p = c["S"], c["N"], c["p"]
    K = host(c["ctx"].kernel(0), c["K"].shape)
    assert np.max(np.abs(K - c["K"])) <= 1e-10 * np.max(np.abs(c["K"]))
    atg = host(c["atg"], (S, N, N))
    fbp = host(c["ctx"].fbp(c["sino"]), (S, N, N))
    g = p.sino.astype(np.float64)
    scale = np.max(np.abs(atg))
    rng = np.random.default_rng(7)
    filtered = {}
    for z, r, col in samples(rng, S, N, 24):
        ref = orc.adjoint_point(g[z], N, p.theta, r, col)
        assert abs(atg[z, r, col] - ref) <= 1e-6 * scale
        if z not in filtered:
            filtered[z] = orc.ramp_filter(g[z])
        fref = (math.pi / len(p.theta)) * orc.adjoint_point(filtered[z], N, p.theta, r, col)
        assert abs(fbp[z, r, col] - fref) <= 1e-4 * np.max(np.abs(fbp))


def test_bench_workload_gradient_and_step(bench_case, orc):
    # gradient and one step for a seeded image and a seeded stand-in for R*g (any image is a
    # valid input of the operator), compared at sampled voxels
    c = bench_case
    S, N = c["S"], c["N"]
    pr = orc.Prior(**PRIOR)
    rng = np.random.default_rng(8)
    x = synth.random_image(rng, (S, N, N), 0.5).astype(np.float64)
    b = synth.random_image(rng, (S, N, N), 4.0e4).astype(np.float64)
    d_b = dev(b)
    G = host(c["ctx"].gradient(dev(x), d_b, tm.Params(**PRIOR)), (S, N, N))
    z = host(c["ctx"].normal_apply(dev(x)), (S, N, N))
    zscale = np.sqrt(np.mean(z ** 2))
    gscale = np.sqrt(np.mean(G ** 2))
    # one fast-gradient step from x (beta = 0) with an explicit step constant
    L = 3.0e5
    xs = dev(x)
    c["ctx"].reconstruct(xs, d_b, tm.Params(**PRIOR, L=L, max_iter=1))
    x1 = host(xs, (S, N, N))
    for zz, r, col in samples(rng, S, N, 24):
        zr = orc.normal_point(x[zz], c["K"], r, col)
        assert abs(z[zz, r, col] - zr) <= 1e-5 * zscale
        gr = zr - b[zz, r, col] + orc.prior_point(x, pr, zz, r, col)
        assert abs(G[zz, r, col] - gr) <= 1e-5 * gscale
        assert abs(x1[zz, r, col] - (x[zz, r, col] - gr / L)) <= 1e-5 * gscale / L + 1e-7


def test_bench_workload_bf16_spectra(bench_case):
    """BF16 storage of the padded spectra at the bench size (eight-warp pass 3a, BF16 gathers):
    one step's K (*) y within 3e-3 relative L2 of the FP32 path's over the whole volume (BF16
    changes only the stored spectra, so the two steps differ by (K (*) y)_bf16 - (K (*) y)_fp32
    over L)."""
    c = bench_case
    S, N = c["S"], c["N"]
    x = synth.random_image(np.random.default_rng(9), (S, N, N), 0.5)
    L = 3.0e5
    steps = []
    for bf16 in (False, True):
        xs = dev(x)
        c["ctx"].reconstruct(xs, c["atg"], tm.Params(**PRIOR, L=L, max_iter=1, bf16=bf16))
        steps.append(host(xs, (S, N, N)))
    z = host(c["ctx"].normal_apply(dev(x)), (S, N, N))
    assert np.linalg.norm(L * (steps[1] - steps[0])) <= 3e-3 * np.linalg.norm(z)


@pytest.fixture(scope="module")
def n2048(orc):
    """Two slices at the finest level of the hierarchical geometry: 2048^2, 128 angles over
    [0, 2 pi/3) (missing wedge); the oracle's kernel K and its spectrum on the 4096^2 grid."""
    S, N, na, span = 2, 2048, 128, 2 * math.pi / 3
    p = synth.volume(S=S, N=N, n_angles=na, n_ellipsoids=6, span=span, seed=1003, with_truth=True)
    ctx = tm.Context([tm.Group(N=N, angles=list(p.theta), n_slices=S, span=span)])
    d_atg = ctx.build_operator(dev(p.sino))
    Kref = orc.kernel(N, p.theta, N)
    return dict(S=S, N=N, na=na, span=span, p=p, ctx=ctx, d_atg=d_atg, K=Kref,
                Chat=orc.circulant_spectrum(Kref, 2 * N))


def test_n2048_limited_angle(orc, n2048):
    # two slices at the finest level of the hierarchical geometry, compared in full
    S, N, p, ctx, d_atg, Kref = (n2048[k] for k in ("S", "N", "p", "ctx", "d_atg", "K"))
    K = host(ctx.kernel(0), Kref.shape)
    assert np.max(np.abs(K - Kref)) <= 1e-10 * np.max(np.abs(Kref))
    atg = host(d_atg, (S, N, N))
    g = p.sino.astype(np.float64)
    rng = np.random.default_rng(9)
    for z, r, col in samples(rng, S, N, 12):
        assert abs(atg[z, r, col] - orc.adjoint_point(g[z], N, p.theta, r, col)) <= 1e-6 * np.max(np.abs(atg))
    pr = orc.Prior(**PRIOR)
    x = synth.random_image(rng, (S, N, N), 0.5).astype(np.float64)
    b = synth.random_image(rng, (S, N, N), 4.0e4).astype(np.float64)  # seeded stand-in for R*g
    d_b = dev(b)
    Chat = n2048["Chat"]
    assert rel(host(ctx.normal_apply(dev(x)), x.shape), orc.toeplitz(x, Kref, Chat)) < 1e-5
    assert rel(host(ctx.gradient(dev(x), d_b, tm.Params(**PRIOR)), x.shape), orc.gradient(x, b, Kref, pr, Chat)) < 1e-5
    # three fast-gradient iterations from zero with an explicit step constant
    L = 1.0e5
    xs = torch.zeros(x.size, dtype=torch.float32, device="cuda")
    ctx.reconstruct(xs, d_b, tm.Params(**PRIOR, L=L, max_iter=3))
    ref = orc.nesterov(np.zeros(x.shape), b, 0.0, Kref, pr, L, 3, Chat=Chat)
    assert rel(host(xs, x.shape), ref) < 1e-4


N2048_BF16_ITERS, N2048_TOTAL_ITERS = 4, 12


def test_n2048_bf16_refinement_follows_oracle(orc, n2048):
    """BF16 spectra for the first iterations, then FP32 refinement iterations (a resumed run,
    which continues the momentum state exactly), at 2 x 2048^2 with the limited-angle geometry:
    the final iterate within 1e-3 relative L2 of the FP64 oracle's after the same count.  R*g is
    the oracle's R*R applied to the phantom (the R*g of noiseless data); the step constant is
    the oracle's bound max |C^| (the circulant spectrum bounds the Toeplitz operator's norm) plus
    the prior's curvature bound."""
    S, N, p, ctx, K, Chat = (n2048[k] for k in ("S", "N", "p", "ctx", "K", "Chat"))
    pr = orc.Prior(**PRIOR)
    b = orc.toeplitz(p.truth, K, Chat)
    L = float(np.max(np.abs(Chat))) + pr.lam * 2.0 * orc.max_rho2(pr)
    ref = orc.nesterov(np.zeros((S, N, N)), b, 0.0, K, pr, L, N2048_TOTAL_ITERS, Chat=Chat)
    d_b = dev(b)
    x = torch.zeros(S * N * N, dtype=torch.float32, device="cuda")
    ctx.reconstruct(x, d_b, tm.Params(**PRIOR, L=L, max_iter=N2048_BF16_ITERS, bf16=True))
    st = ctx.reconstruct(x, d_b, tm.Params(**PRIOR, L=L, max_iter=N2048_TOTAL_ITERS - N2048_BF16_ITERS, resume=True))
    assert st.iterations == N2048_TOTAL_ITERS and st.status == 0
    assert rel(host(x, (S, N, N)), ref) < 1e-3


def seeded_slices(seed, S, N, scale):
    """Slice z of a seeded uniform volume, generated slice by slice (the full volume is only
    ever held on the device)."""
    return lambda z: np.random.default_rng(seed * 100003 + z).uniform(0.0, scale, (N, N)).astype(np.float32)


def test_hierarchical_finest_level_full_size(orc):
    # 512 slices of 2048^2, 128 angles over [0, 2 pi/3): R*g, K (*) x, the gradient and one
    # fast-gradient step at sampled voxels
    S, N, na, span = 512, 2048, 128, 2 * math.pi / 3
    p = synth.volume(S=S, N=N, n_angles=na, n_ellipsoids=20, span=span, seed=1003)
    ctx = tm.Context([tm.Group(N=N, angles=list(p.theta), n_slices=S, span=span)])
    d_atg = ctx.build_operator(dev(p.sino))
    g = p.sino
    rng = np.random.default_rng(11)
    pts = samples(rng, S, N, 10)
    amax = float(torch.max(torch.abs(d_atg)).item())
    atg = d_atg.view(S, N, N)
    for z, r, c in pts:
        ref = orc.adjoint_point(g[z].astype(np.float64), N, p.theta, r, c)
        assert abs(float(atg[z, r, c].item()) - ref) <= 1e-6 * amax
    del atg
    gen_x, gen_b = seeded_slices(21, S, N, 0.5), seeded_slices(22, S, N, 4.0e4)
    x = torch.empty(S * N * N, dtype=torch.float32, device="cuda")
    b = torch.empty_like(x)
    for z in range(S):
        x[z * N * N:(z + 1) * N * N] = torch.from_numpy(gen_x(z).ravel()).cuda()
        b[z * N * N:(z + 1) * N * N] = torch.from_numpy(gen_b(z).ravel()).cuda()
    zk = ctx.normal_apply(x).view(S, N, N)
    G = ctx.gradient(x, b, tm.Params(**PRIOR)).view(S, N, N)
    L = 1.0e5
    x1 = x.clone()
    ctx.reconstruct(x1, b, tm.Params(**PRIOR, L=L, max_iter=1))
    x1 = x1.view(S, N, N)
    torch.cuda.synchronize()
    zscale = float(torch.sqrt(torch.mean(zk.double() ** 2)).item())
    gscale = float(torch.sqrt(torch.mean(G.double() ** 2)).item())
    Kref = orc.kernel(N, p.theta, N)
    pr = orc.Prior(**PRIOR)
    for zz, r, c in pts:
        # the slice and its neighbours, regenerated on the host
        lo, hi = max(zz - 1, 0), min(zz + 2, S)
        xs = np.stack([gen_x(k) for k in range(lo, hi)]).astype(np.float64)
        zr = orc.normal_point(xs[zz - lo], Kref, r, c)
        assert abs(float(zk[zz, r, c].item()) - zr) <= 1e-5 * zscale
        gr = zr - float(gen_b(zz)[r, c]) + orc.prior_point(xs, pr, zz - lo, r, c)
        assert abs(float(G[zz, r, c].item()) - gr) <= 1e-5 * gscale
        assert abs(float(x1[zz, r, c].item()) - (xs[zz - lo, r, c] - gr / L)) <= 1e-5 * gscale / L + 1e-7


@pytest.mark.parametrize("N,na", [(1536, 96), (2560, 64)])
def test_mixed_radix_sides(orc, N, na):
    # image sides whose 2N transforms take radix 3 (1536 = 2^9 * 3) or radix 5 (2560 = 2^9 * 5):
    # K in full, R*g and the FBP start at sampled pixels, then whole-slice products, the
    # gradient and three fast-gradient iterations against the oracle
    S, span = 2, math.pi
    p = synth.volume(S=S, N=N, n_angles=na, n_ellipsoids=6, seed=1004)
    ctx = tm.Context([tm.Group(N=N, angles=list(p.theta), n_slices=S)])
    d_sino = dev(p.sino)
    d_atg, d_x0 = ctx.build_operator_fbp(d_sino)
    Kref = orc.kernel(N, p.theta, N)
    K = host(ctx.kernel(0), Kref.shape)
    assert np.max(np.abs(K - Kref)) <= 1e-10 * np.max(np.abs(Kref))
    atg = host(d_atg, (S, N, N))
    x0 = host(d_x0, (S, N, N))
    g = p.sino.astype(np.float64)
    rng = np.random.default_rng(13)
    pts = samples(rng, S, N, 8)
    for z, r, col in pts:
        assert abs(atg[z, r, col] - orc.adjoint_point(g[z], N, p.theta, r, col)) <= 1e-6 * np.max(np.abs(atg))
    h = orc.ramp_filter(g)
    for z, r, col in pts:
        ref = (span / na) * orc.adjoint_point(h[z], N, p.theta, r, col)
        assert abs(x0[z, r, col] - ref) <= 2e-4 * np.max(np.abs(x0))
    pr = orc.Prior(**PRIOR)
    x = synth.random_image(rng, (S, N, N), 0.5).astype(np.float64)
    b = synth.random_image(rng, (S, N, N), 4.0e4).astype(np.float64)  # seeded stand-in for R*g
    d_b = dev(b)
    Chat = orc.circulant_spectrum(Kref)
    assert rel(host(ctx.normal_apply(dev(x)), x.shape), orc.toeplitz(x, Kref, Chat)) < 1e-5
    assert rel(host(ctx.gradient(dev(x), d_b, tm.Params(**PRIOR)), x.shape), orc.gradient(x, b, Kref, pr, Chat)) < 1e-5
    L = 1.0e5
    xs = torch.zeros(x.size, dtype=torch.float32, device="cuda")
    ctx.reconstruct(xs, d_b, tm.Params(**PRIOR, L=L, max_iter=3))
    ref = orc.nesterov(np.zeros(x.shape), b, 0.0, Kref, pr, L, 3, Chat=Chat)
    assert rel(host(xs, x.shape), ref) < 1e-4
