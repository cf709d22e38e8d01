"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Tolerances: the FP32 operator and gradient within 1e-5 relative L2 of the oracle; the FP64
setup (kernel K, R*g) within 1e-10 / 1e-6 (the latter is the FP32 storage of R*g); the FP32
FBP start within 1e-4 (FP32 arithmetic end to end).
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


class Problem:
    def __init__(self, orc, N, S, na, span=math.pi, seed=5):
        self.N, self.S, self.na = N, S, na
        p = synth.volume(S=S, N=N, n_angles=na, n_ellipsoids=6, span=span, seed=seed)
        self.theta, self.span = p.theta, span
        self.sino = p.sino  # FP32 (S, na, N)
        self.g = self.sino.astype(np.float64)
        self.ctx = tm.Context([tm.Group(N=N, angles=list(self.theta), n_slices=S, span=span)])
        self.d_sino = dev(self.sino)
        self.d_atg = self.ctx.build_operator(self.d_sino)
        self.K = orc.kernel(N, self.theta, N)
        self.atg = orc.adjoint(self.g, N, self.theta)
        rng = np.random.default_rng(seed + 1)
        self.x = synth.random_image(rng, (S, N, N), 0.5).astype(np.float64)
        self.xp = synth.random_image(rng, (S, N, N), 0.5).astype(np.float64)


@pytest.fixture(scope="module", params=[(64, 3, 37, math.pi), (128, 2, 45, 2 * math.pi / 3)], ids=["N64", "N128limited"])
def prob(request, orc):
    N, S, na, span = request.param
    return Problem(orc, N, S, na, span)


def test_kernel_matches_dirichlet_sum(prob):
    K = host(prob.ctx.kernel(0), prob.K.shape)
    assert np.max(np.abs(K - prob.K)) <= 1e-10 * np.max(np.abs(prob.K))


def test_atg_matches_adjoint(prob):
    got = host(prob.d_atg, prob.atg.shape)
    assert rel(got, prob.atg) < 1e-6


def test_lambda_max_matches_power_iteration(prob, orc):
    lam = prob.ctx.lambda_max()[0]
    ref = orc.power_lambda_max(prob.K, prob.N)
    assert abs(lam - ref) <= 1e-5 * ref


def test_normal_apply(prob, orc):
    z = host(prob.ctx.normal_apply(dev(prob.x)), prob.x.shape)
    ref = orc.toeplitz(prob.x, prob.K)
    assert rel(z, ref) < 1e-5


def test_gradient(prob, orc):
    pr = orc.Prior(**PRIOR)
    G = host(prob.ctx.gradient(dev(prob.x), prob.d_atg, tm.Params(**PRIOR)), prob.x.shape)
    ref = orc.gradient(prob.x, prob.atg, prob.K, pr)
    assert rel(G, ref) < 1e-5


def test_general_q_gradient_and_iterations_follow_oracle(prob, orc):
    # the stencil's general-exponent variant (q != 2: |d/sigma|^(q-2) by a fourth special-function
    # operation per pair), at an exponent pair the oracle's potential is pinned at
    prm = dict(PRIOR, p=1.1, q=1.8)
    pr = orc.Prior(**prm)
    L = 4.0 * orc.power_lambda_max(prob.K, prob.N)  # rho'' is unbounded at 0 for q < 2: a given L
    G = host(prob.ctx.gradient(dev(prob.x), prob.d_atg, tm.Params(**prm, L=L)), prob.x.shape)
    assert rel(G, orc.gradient(prob.x, prob.atg, prob.K, pr)) < 1e-5
    iters = 10
    x = dev(prob.x)
    prob.ctx.reconstruct(x, prob.d_atg, tm.Params(**prm, L=L, max_iter=iters))
    ref = orc.nesterov(prob.x.astype(np.float32).astype(np.float64), prob.atg, float(np.sum(prob.g ** 2)), prob.K,
                       pr, L, iters)
    assert rel(host(x, prob.x.shape), ref) < 1e-4


def test_fused_step_and_partials(prob, orc):
    pr = orc.Prior(**PRIOR)
    beta, L = 0.37, 55.0
    out, parts = prob.ctx.step(dev(prob.x), dev(prob.xp), beta, prob.d_atg, tm.Params(**PRIOR), L)
    xn = host(out, prob.x.shape)
    x32, xp32 = prob.x.astype(np.float32).astype(np.float64), prob.xp.astype(np.float32).astype(np.float64)
    y = x32 + beta * (x32 - xp32)
    z = orc.toeplitz(y, prob.K)
    gp, phi = orc.prior(y, pr)
    G = z - prob.atg + gp
    ref = y - G / L
    assert rel(xn, ref) < 1e-5
    want = [np.sum(y * z), np.sum(y * prob.atg), phi / pr.lam, np.sum(G * (ref - x32)), np.sum(G * G)]
    for k, (a, b) in enumerate(zip(parts, want)):
        assert abs(a - b) <= 1e-5 * max(abs(b), 1e-3 * abs(want[0])), (k, a, b)


def test_objective(prob, orc):
    pr = orc.Prior(**PRIOR)
    F = prob.ctx.objective(dev(prob.x), prob.d_atg, tm.Params(**PRIOR))
    ref = orc.objective(prob.x, prob.atg, float(np.sum(prob.g ** 2)), prob.K, pr)
    assert abs(F - ref) <= 1e-5 * abs(ref)


def test_fbp(prob, orc):
    f0 = host(prob.ctx.fbp(prob.d_sino), prob.atg.shape)
    ref = orc.fbp(prob.g, prob.N, prob.theta, prob.span)
    assert rel(f0, ref) < 1e-4


def test_reconstruct_follows_oracle_trajectory(prob, orc):
    pr = orc.Prior(**PRIOR)
    iters = 30
    x = torch.zeros(prob.x.size, dtype=torch.float32, device="cuda")
    st = prob.ctx.reconstruct(x, prob.d_atg, tm.Params(**PRIOR, max_iter=iters))
    assert st.iterations == iters and st.status == 0
    log = prob.ctx.get_log()
    L = orc.lipschitz(prob.K, prob.N, pr)
    assert abs(st.L - L) <= 1e-5 * L
    olog = []
    ref = orc.nesterov(np.zeros(prob.x.shape), prob.atg, float(np.sum(prob.g ** 2)), prob.K, pr, L, iters, log=olog)
    got = host(x, prob.x.shape)
    assert rel(got, ref) < 1e-4
    # F(y_k) is assembled from terms as large as F(0) = 1/2 g.g, accumulated from FP32
    # products: compare on that scale
    F0 = 0.5 * float(np.sum(prob.g ** 2))
    assert abs(log[0][0] - F0) <= 1e-7 * F0
    for (F, dot, rs, gg), (Fo, doto, rso) in zip(log, olog):
        assert abs(F - Fo) <= 1e-7 * F0
        if abs(doto) > 1e-4 * abs(gg) / L:
            assert bool(rs) == rso


def test_single_slice_plain_method_follows_oracle(orc):
    """The plain single-slice form: one 128^2 slice, 90 angles over [0, pi), Poisson noise at 1e4
    photons per ray, FBP start, 50 iterations; a single slice keeps its 8 in-plane neighbours of
    the 26-neighbourhood.  Final iterate within 1e-3 of the FP64 oracle's."""
    N, iters = 128, 50
    p = synth.single_slice(N=N, n_angles=90, n_ellipses=10, seed=1001, with_truth=False)
    ctx = tm.Context([tm.Group(N=N, angles=list(p.theta), n_slices=1)])
    sino = dev(p.sino)
    atg = ctx.build_operator(sino)
    x = ctx.fbp(sino)
    st = ctx.reconstruct(x, atg, tm.Params(**PRIOR, max_iter=iters))
    assert st.iterations == iters and st.status == 0
    pr = orc.Prior(**PRIOR)
    g = p.sino.astype(np.float64)[0]
    K = orc.kernel(N, p.theta, N)
    L = orc.lipschitz(K, N, pr)
    ref = orc.nesterov(orc.fbp(g, N, p.theta, math.pi), orc.adjoint(g, N, p.theta), float(np.sum(g * g)), K, pr, L,
                       iters)
    assert rel(host(x, (N, N)), ref) < 1e-3


def test_batched_normal_operator_equals_slices_alone(prob):
    """The data term is slice-separable (Sec. 2): R*R applied to a batch equals R*R applied to
    each slice in a context of its own."""
    z = host(prob.ctx.normal_apply(dev(prob.x)), prob.x.shape)
    ctx1 = tm.Context([tm.Group(N=prob.N, angles=list(prob.theta), n_slices=1, span=prob.span)])
    ctx1.build_operator(dev(prob.sino[:1]))
    for s in range(prob.S):
        z1 = host(ctx1.normal_apply(dev(prob.x[s])), (prob.N, prob.N))
        assert rel(z1, z[s]) < 1e-6


def test_nonneg_projection_follows_oracle(prob, orc):
    # the projected variant: every iterate max(y - G/L, 0); 30 iterations from a start with
    # negative entries follow the oracle's projected method and stay non-negative
    pr = orc.Prior(**PRIOR)
    iters = 30
    x0 = prob.x - 0.25
    L = orc.lipschitz(prob.K, prob.N, pr)
    x = dev(x0)
    st = prob.ctx.reconstruct(x, prob.d_atg, tm.Params(**PRIOR, L=L, max_iter=iters, nonneg=True))
    assert st.iterations == iters and st.status == 0
    got = host(x, prob.x.shape)
    ref = orc.nesterov(x0.astype(np.float32).astype(np.float64), prob.atg, float(np.sum(prob.g ** 2)), prob.K, pr, L,
                       iters, nonneg=True)
    assert got.min() >= 0.0 and np.mean(ref == 0.0) > 0.01
    assert rel(got, ref) < 1e-4


def test_graph_replay_is_bitwise_eager(prob):
    prm = dict(PRIOR, max_iter=7)
    a = torch.zeros(prob.x.size, dtype=torch.float32, device="cuda")
    b = torch.zeros_like(a)
    prob.ctx.reconstruct(a, prob.d_atg, tm.Params(**prm, use_graph=True))
    prob.ctx.reconstruct(b, prob.d_atg, tm.Params(**prm, use_graph=False))
    torch.cuda.synchronize()
    assert torch.equal(a, b)
    # a second replay of the cached graph gives the same result again
    c = torch.zeros_like(a)
    prob.ctx.reconstruct(c, prob.d_atg, tm.Params(**prm, use_graph=True))
    torch.cuda.synchronize()
    assert torch.equal(a, c)


RESTART = {"gradient": 0, "none": 1, "function": 2}


@pytest.mark.parametrize("mode", ["function", "none"])
def test_restart_modes_follow_oracle(prob, orc, mode):
    pr = orc.Prior(**PRIOR)
    iters = 30
    x = torch.zeros(prob.x.size, dtype=torch.float32, device="cuda")
    st = prob.ctx.reconstruct(x, prob.d_atg, tm.Params(**PRIOR, max_iter=iters, restart=RESTART[mode]))
    assert st.iterations == iters and st.status == 0
    log = prob.ctx.get_log()
    L = orc.lipschitz(prob.K, prob.N, pr)
    olog = []
    ref = orc.nesterov(np.zeros(prob.x.shape), prob.atg, float(np.sum(prob.g ** 2)), prob.K, pr, L, iters, log=olog,
                       restart=mode)
    assert rel(host(x, prob.x.shape), ref) < 1e-4
    F0 = 0.5 * float(np.sum(prob.g ** 2))
    for k, ((F, dot, rs, gg), (Fo, doto, rso)) in enumerate(zip(log, olog)):
        assert abs(F - Fo) <= 1e-7 * F0
        if mode == "none":
            assert not rs
        elif k > 0 and abs(Fo - olog[k - 1][0]) > 1e-6 * F0:
            assert bool(rs) == rso


def test_device_loop_stops_at_gap(prob):
    # F_ref from a longer run; the device-driven graph loop and the eager launches must stop
    # at the same iteration with bitwise equal iterates, and no kernel runs after the stop
    x = torch.zeros(prob.x.size, dtype=torch.float32, device="cuda")
    F_ref = prob.ctx.reconstruct(x, prob.d_atg, tm.Params(**PRIOR, max_iter=200)).objective
    prm = dict(PRIOR, max_iter=200, gap_tol=1e-2, F_ref=F_ref)
    a = torch.zeros_like(x)
    b = torch.zeros_like(x)
    n0 = prob.ctx.launch_count()
    sa = prob.ctx.reconstruct(a, prob.d_atg, tm.Params(**prm, use_graph=True))
    n1 = prob.ctx.launch_count()
    sb = prob.ctx.reconstruct(b, prob.d_atg, tm.Params(**prm, use_graph=False))
    torch.cuda.synchronize()
    assert 1 < sa.iterations == sb.iterations < 200
    assert torch.equal(a, b)
    # state init + 5 kernels per iteration (passes 1, 2, 3a, 3b, finalize) + final gather and
    # rotation reset
    assert n1 - n0 == 5 * sa.iterations + 3
    log = prob.ctx.get_log()
    F0 = 0.5 * float(np.sum(prob.g ** 2))
    gaps = [(F - F_ref) / (F0 - F_ref) for F, _, _, _ in log]
    assert len(gaps) == sb.iterations and gaps[-1] <= 1e-2 < gaps[-2]
    # a replay of the cached graph with another stop rule reuses it
    a.zero_()
    n2 = prob.ctx.launch_count()
    sc = prob.ctx.reconstruct(a, prob.d_atg, tm.Params(**dict(prm, gap_tol=0.0, max_iter=5), use_graph=True))
    assert sc.iterations == 5 and prob.ctx.launch_count() - n2 == 5 * 5 + 3


def test_bf16_spectra_follow_oracle(prob, orc):
    # BF16 storage of the padded spectrum (8-bit mantissa, relative rounding 2^-9 per entry,
    # two roundings per iteration): one gradient within 3e-3 relative L2 of the FP64 oracle
    pr = orc.Prior(**PRIOR)
    x = dev(prob.x)
    st = prob.ctx.reconstruct(x, prob.d_atg, tm.Params(**PRIOR, max_iter=1, bf16=True))
    G = (prob.x - host(x, prob.x.shape)) * st.L
    assert rel(G, orc.gradient(prob.x, prob.atg, prob.K, pr)) < 3e-3
    # over 30 iterations the rounding noise of every gradient accumulates in the iterate
    iters = 30
    x = torch.zeros(prob.x.size, dtype=torch.float32, device="cuda")
    st = prob.ctx.reconstruct(x, prob.d_atg, tm.Params(**PRIOR, max_iter=iters, bf16=True))
    assert st.iterations == iters and st.status == 0
    L = orc.lipschitz(prob.K, prob.N, pr)
    olog = []
    ref = orc.nesterov(np.zeros(prob.x.shape), prob.atg, float(np.sum(prob.g ** 2)), prob.K, pr, L, iters, log=olog)
    assert rel(host(x, prob.x.shape), ref) < 2e-2
    # F(y_k) = 1/2 y.z - y.R*g + 1/2 g.g is assembled from terms of the size of F(0) = 1/2 g.g
    # that cancel as the iterates converge: bound the BF16 error on that scale (measured about
    # 1.5e-4 F(0))
    F0 = 0.5 * float(np.sum(prob.g ** 2))
    for (F, _, _, _), (Fo, _, _) in zip(prob.ctx.get_log(), olog):
        assert abs(F - Fo) <= 1e-3 * F0


def test_bf16_refinement_matches_fp32(prob):
    # BF16 iterations until the gap reaches 1e-1, FP32 after: the run reaches the 1e-3 gap of
    # the FP32 run; graph and eager launches give bitwise equal iterates
    x = torch.zeros(prob.x.size, dtype=torch.float32, device="cuda")
    F_ref = prob.ctx.reconstruct(x, prob.d_atg, tm.Params(**PRIOR, max_iter=300)).objective
    stop = dict(PRIOR, max_iter=300, gap_tol=1e-3, F_ref=F_ref)
    a = torch.zeros_like(x)
    b = torch.zeros_like(x)
    c = torch.zeros_like(x)
    s32 = prob.ctx.reconstruct(c, prob.d_atg, tm.Params(**stop))
    sa = prob.ctx.reconstruct(a, prob.d_atg, tm.Params(**stop, bf16=True, refine_gap=1e-1, use_graph=True))
    sb = prob.ctx.reconstruct(b, prob.d_atg, tm.Params(**stop, bf16=True, refine_gap=1e-1, use_graph=False))
    torch.cuda.synchronize()
    assert sa.iterations == sb.iterations and torch.equal(a, b)
    assert sa.gap <= 1e-3 and sa.iterations < 300
    assert sa.iterations <= s32.iterations + 5
    assert rel(host(a, prob.x.shape), host(c, prob.x.shape).astype(np.float64)) < 1e-2


REFINE_ITERS = 150


def test_bf16_refinement_follows_oracle(prob, orc):
    """The chosen precision form: BF16 spectra until the relative gap reaches 1e-1, then FP32
    refinement iterations (the device-side switch of refine_gap, inside the graph loop) to a
    fixed count.  The final iterate is within 1e-3 relative L2 of the FP64 oracle's after the
    same count.  F_ref (which places the switch) and the step constant L are the oracle's."""
    pr = orc.Prior(**PRIOR)
    gtg = float(np.sum(prob.g ** 2))
    Chat = orc.circulant_spectrum(prob.K)
    L = orc.lipschitz(prob.K, prob.N, pr, Chat=Chat)
    x0 = np.zeros(prob.x.shape)
    F_ref = orc.objective(orc.nesterov(x0, prob.atg, gtg, prob.K, pr, L, 400, Chat=Chat), prob.atg, gtg, prob.K, pr,
                          Chat)
    ref = orc.nesterov(x0, prob.atg, gtg, prob.K, pr, L, REFINE_ITERS, Chat=Chat)
    x = torch.zeros(prob.x.size, dtype=torch.float32, device="cuda")
    st = prob.ctx.reconstruct(x, prob.d_atg, tm.Params(**PRIOR, L=L, max_iter=REFINE_ITERS, F_ref=F_ref, bf16=True,
                                                       refine_gap=1e-1))
    assert st.iterations == REFINE_ITERS and st.status == 0
    assert rel(host(x, prob.x.shape), ref) < 1e-3


@pytest.mark.parametrize("use_graph", [True, False])
def test_checkpoint_resume_is_bitwise(prob, use_graph):
    # 30 iterations in one run == 18 iterations, export, unrelated work, import, 12 more
    prm = dict(PRIOR, use_graph=use_graph)
    a = torch.zeros(prob.x.size, dtype=torch.float32, device="cuda")
    sa = prob.ctx.reconstruct(a, prob.d_atg, tm.Params(**prm, max_iter=30))
    b = torch.zeros_like(a)
    prob.ctx.reconstruct(b, prob.d_atg, tm.Params(**prm, max_iter=18))
    ck = prob.ctx.state_export()
    other = dev(prob.x)
    prob.ctx.reconstruct(other, prob.d_atg, tm.Params(**prm, max_iter=5))
    prob.ctx.state_import(ck)
    sb = prob.ctx.reconstruct(b, prob.d_atg, tm.Params(**prm, max_iter=12, resume=True))
    torch.cuda.synchronize()
    assert sb.iterations == 30 and sb.restarts == sa.restarts
    assert torch.equal(a, b)
    assert sb.objective == sa.objective


def test_autotune_keeps_results(prob, orc):
    # the tuner only changes how pass 3 splits the slices over blocks: the iterates still
    # follow the oracle, graph == eager, and d_x is left alone
    x0 = dev(prob.x)
    keep = x0.clone()
    zc = prob.ctx.autotune(x0, prob.d_atg, tm.Params(**PRIOR))
    torch.cuda.synchronize()
    assert torch.equal(x0, keep)
    assert len(zc) == 1 and 1 <= zc[0] <= prob.S
    pr = orc.Prior(**PRIOR)
    a = torch.zeros(prob.x.size, dtype=torch.float32, device="cuda")
    b = torch.zeros_like(a)
    prob.ctx.reconstruct(a, prob.d_atg, tm.Params(**PRIOR, max_iter=20, use_graph=True))
    prob.ctx.reconstruct(b, prob.d_atg, tm.Params(**PRIOR, max_iter=20, use_graph=False))
    torch.cuda.synchronize()
    assert torch.equal(a, b)
    L = orc.lipschitz(prob.K, prob.N, pr)
    ref = orc.nesterov(np.zeros(prob.x.shape), prob.atg, float(np.sum(prob.g ** 2)), prob.K, pr, L, 20)
    assert rel(host(a, prob.x.shape), ref) < 1e-4


def test_uneven_groups_equal_separate_contexts(orc):
    specs = [(64, 2, 30), (128, 1, 50), (64, 1, 20)]
    groups, sinos, thetas, ctxs = [], [], [], []
    for k, (N, S, na) in enumerate(specs):
        p = synth.volume(S=S, N=N, n_angles=na, n_ellipsoids=4, seed=40 + k)
        groups.append(tm.Group(N=N, angles=list(p.theta), n_slices=S))
        sinos.append(p.sino.ravel())
        thetas.append(p.theta)
        ctxs.append(tm.Context([groups[-1]]))
    big = tm.Context(groups)
    d_sino = dev(np.concatenate(sinos))
    atg = big.build_operator(d_sino)
    rng = np.random.default_rng(3)
    xs = [synth.random_image(rng, (S, N, N)).ravel() for N, S, _ in specs]
    d_x = dev(np.concatenate(xs))
    G = big.gradient(d_x, atg, tm.Params(**PRIOR))
    torch.cuda.synchronize()
    off = 0
    for k, (N, S, na) in enumerate(specs):
        d_sk, d_xk = dev(sinos[k]), dev(xs[k])
        a1 = ctxs[k].build_operator(d_sk)
        G1 = ctxs[k].gradient(d_xk, a1, tm.Params(**PRIOR))
        torch.cuda.synchronize()
        n = S * N * N
        atg_ref = orc.adjoint(sinos[k].reshape(S, na, N).astype(np.float64), N, thetas[k])
        e_big = rel(host(atg[off:off + n], (S, N, N)), atg_ref)
        e_sep = rel(host(a1, (S, N, N)), atg_ref)
        assert e_big < 1e-6 and e_sep < 1e-6, (k, "R*g vs oracle", e_big, e_sep)
        ref = orc.gradient(xs[k].reshape(S, N, N), atg_ref, orc.kernel(N, thetas[k], N), orc.Prior(**PRIOR))
        e_big = rel(host(G[off:off + n], (S, N, N)), ref)
        e_sep = rel(host(G1, (S, N, N)), ref)
        assert e_big < 1e-5 and e_sep < 1e-5, (k, "gradient vs oracle", e_big, e_sep)
        # and the batched run is bit-identical to the separate one
        assert torch.equal(big.kernel(k), ctxs[k].kernel(0)), (k, "kernel")
        assert big.lambda_max()[k] == ctxs[k].lambda_max()[0], (k, "lambda_max")
        assert torch.equal(atg[off:off + n], a1), (k, "R*g")
        assert torch.equal(G[off:off + n], G1), (k, "gradient")
        off += n


def test_uneven_groups_reconstruct_like_separate_contexts(orc):
    """Groups are independent problems (Sec. 2: the data term is slice-separable and the prior
    couples only the slices of a group): each keeps its own step constant, momentum and restart
    test, so 25 iterations of an uneven batch give, group by group, bitwise the iterates of a
    context holding that group alone (graph and eager launches), and follow the FP64 oracle's
    fast gradient method on that group."""
    specs = [(64, 2, 30), (128, 1, 50), (64, 1, 20)]
    iters = 25
    groups, sinos, thetas = [], [], []
    for k, (N, S, na) in enumerate(specs):
        p = synth.volume(S=S, N=N, n_angles=na, n_ellipsoids=4, seed=40 + k)
        groups.append(tm.Group(N=N, angles=list(p.theta), n_slices=S))
        sinos.append(p.sino.ravel())
        thetas.append(p.theta)
    big = tm.Context(groups)
    atg = big.build_operator(dev(np.concatenate(sinos)))
    xg = torch.zeros(atg.numel(), dtype=torch.float32, device="cuda")
    xe = torch.zeros_like(xg)
    sg = big.reconstruct(xg, atg, tm.Params(**PRIOR, max_iter=iters, use_graph=True))
    big.reconstruct(xe, atg, tm.Params(**PRIOR, max_iter=iters, use_graph=False))
    torch.cuda.synchronize()
    assert sg.iterations == iters and torch.equal(xg, xe)
    pr = orc.Prior(**PRIOR)
    off = 0
    for k, (N, S, na) in enumerate(specs):
        n = S * N * N
        ctx = tm.Context([groups[k]])
        a1 = ctx.build_operator(dev(sinos[k]))
        x1 = torch.zeros(n, dtype=torch.float32, device="cuda")
        ctx.reconstruct(x1, a1, tm.Params(**PRIOR, max_iter=iters))
        torch.cuda.synchronize()
        assert torch.equal(xg[off:off + n], x1), k
        g = sinos[k].reshape(S, na, N).astype(np.float64)
        K = orc.kernel(N, thetas[k], N)
        ref = orc.nesterov(np.zeros((S, N, N)), orc.adjoint(g, N, thetas[k]), float(np.sum(g * g)), K, pr,
                           orc.lipschitz(K, N, pr), iters)
        assert rel(host(xg[off:off + n], (S, N, N)), ref) < 1e-4, k
        off += n


def test_groups_of_one_side_share_launches(orc):
    """Consecutive groups of one image side (different angle counts and slice counts) run each
    pass as one launch over all their blocks: 25 iterations give, group by group, bitwise the
    iterates of a context holding that group alone, and an iteration launches one kernel per
    pass per run of such groups (runs: three groups of 64^2, two of 128^2, one of 64^2)."""
    specs = [(64, 2, 30), (64, 1, 20), (64, 3, 45), (128, 1, 50), (128, 2, 37), (64, 1, 24)]
    iters = 25
    groups, sinos = [], []
    for k, (N, S, na) in enumerate(specs):
        p = synth.volume(S=S, N=N, n_angles=na, n_ellipsoids=4, seed=60 + k)
        groups.append(tm.Group(N=N, angles=list(p.theta), n_slices=S))
        sinos.append(p.sino.ravel())
    big = tm.Context(groups)
    atg = big.build_operator(dev(np.concatenate(sinos)))
    xg = torch.zeros(atg.numel(), dtype=torch.float32, device="cuda")
    xe = torch.zeros_like(xg)
    big.reconstruct(xg, atg, tm.Params(**PRIOR, max_iter=iters, use_graph=True))
    n0 = big.launch_count()
    big.reconstruct(xe, atg, tm.Params(**PRIOR, max_iter=iters, use_graph=False))
    n1 = big.launch_count()
    big.reconstruct(xe.zero_(), atg, tm.Params(**PRIOR, max_iter=iters + 5, use_graph=False))
    n2 = big.launch_count()
    torch.cuda.synchronize()
    assert (n2 - n1) - (n1 - n0) == 5 * (4 + 4 + 4 + 1)  # three runs of four passes, and the finalize
    xe.zero_()
    big.reconstruct(xe, atg, tm.Params(**PRIOR, max_iter=iters, use_graph=False))
    torch.cuda.synchronize()
    assert torch.equal(xg, xe)
    off = 0
    for k, (N, S, na) in enumerate(specs):
        n = S * N * N
        ctx = tm.Context([groups[k]])
        a1 = ctx.build_operator(dev(sinos[k]))
        assert torch.equal(atg[off:off + n], a1), (k, "R*g")
        x1 = torch.zeros(n, dtype=torch.float32, device="cuda")
        ctx.reconstruct(x1, a1, tm.Params(**PRIOR, max_iter=iters))
        torch.cuda.synchronize()
        assert torch.equal(xg[off:off + n], x1), k
        off += n


def test_identical_groups_give_identical_results():
    p = synth.volume(S=2, N=64, n_angles=24, n_ellipsoids=4, seed=50)
    grp = tm.Group(N=64, angles=list(p.theta), n_slices=2)
    ctx = tm.Context([grp, grp, grp])
    sino = np.concatenate([p.sino.ravel()] * 3)
    atg = ctx.build_operator(dev(sino))
    x = dev(np.concatenate([synth.random_image(np.random.default_rng(4), (2, 64, 64)).ravel()] * 3))
    G = ctx.gradient(x, atg, tm.Params(**PRIOR))
    torch.cuda.synchronize()
    n = 2 * 64 * 64
    for k in (1, 2):
        assert torch.equal(atg[:n], atg[k * n:(k + 1) * n]), (k, "R*g")
        assert torch.equal(G[:n], G[k * n:(k + 1) * n]), (k, "gradient")


def test_overlapped_setup_equals_separate_calls(prob):
    atg, x0 = prob.ctx.build_operator_fbp(prob.d_sino)
    atg2 = prob.ctx.build_operator(prob.d_sino)
    x02 = prob.ctx.fbp(prob.d_sino)
    torch.cuda.synchronize()
    assert torch.equal(atg, atg2) and torch.equal(x0, x02)


def test_lanczos_upsampling(orc):
    rng = np.random.default_rng(9)
    for S, Nc in [(2, 32), (1, 100)]:
        c = rng.standard_normal((S, Nc, Nc)).astype(np.float32)
        ctx = tm.Context([tm.Group(N=64, angles=[0.0], n_slices=1)])
        f = host(ctx.upsample_lanczos3(dev(c), S, Nc), (S, 2 * Nc, 2 * Nc))
        ref = orc.lanczos_up(c.astype(np.float64))
        assert np.array_equal(f[:, ::2, ::2], c.astype(np.float64))
        assert np.max(np.abs(f - ref)) < 1e-5 * np.max(np.abs(ref))


def test_downsample_sino_bitwise(orc):
    rng = np.random.default_rng(10)
    g = rng.standard_normal((3, 7, 64)).astype(np.float32)
    ctx = tm.Context([tm.Group(N=64, angles=[0.0], n_slices=1)])
    for f in (2, 4):
        d = host(ctx.downsample_sino(dev(g), 3, 7, 64, f), (3, 7, 64 // f))
        assert np.array_equal(d, orc.downsample_sino(g.astype(np.float64), f))


@pytest.mark.parametrize("coarse_fp32", [False, True], ids=["fp64_setup", "fp32_coarse_setup"])
def test_hierarchical_levels_follow_oracle(orc, coarse_fp32):
    # three levels 64 -> 128 -> 256 (Sec. 2.3): coarse sinograms by bin subsampling, FBP at the
    # coarsest level, Lanczos-3 x2 upsampling between levels; the oracle runs the same chain (with
    # the FP64 R*g at every level, also when the coarse levels build theirs in FP32)
    N, S, na, levels = 256, 3, 60, 3
    iters = [25, 15, 8]
    p = synth.volume(S=S, N=N, n_angles=na, n_ellipsoids=6, seed=61)
    pr = orc.Prior(**PRIOR)
    x, ctxs, stats = tm.reconstruct_levels(N, p.theta, S, dev(p.sino), levels,
                                           [tm.Params(**PRIOR, max_iter=k) for k in iters],
                                           coarse_setup_fp32=coarse_fp32)
    assert [s.iterations for s in stats] == iters
    g = p.sino.astype(np.float64)
    xo = None
    for lev in range(levels):
        f = 1 << (levels - 1 - lev)
        Nl = N // f
        gl = g if f == 1 else orc.downsample_sino(g, f)
        K = orc.kernel(Nl, p.theta, Nl)
        atg = orc.adjoint(gl, Nl, p.theta)
        x0 = orc.fbp(gl, Nl, p.theta, math.pi) if xo is None else orc.lanczos_up(xo)
        L = orc.lipschitz(K, Nl, pr)
        xo = orc.nesterov(x0, atg, float(np.sum(gl ** 2)), K, pr, L, iters[lev])
    assert rel(host(x, xo.shape), xo) < 1e-3


def test_argument_errors():
    with pytest.raises(tm.TmbirError) as e:
        tm.Context([tm.Group(N=96, angles=[0.0, 1.0])])
    assert e.value.code == -2
    with pytest.raises(tm.TmbirError) as e:
        tm.Context([tm.Group(N=64, angles=[0.0], n_det=128)])
    assert e.value.code == -2
    # empty and degenerate geometries are refused, not run
    for bad in ([], [tm.Group(N=64, angles=[])], [tm.Group(N=64, angles=[0.0, 1.0], n_slices=0)],
                [tm.Group(N=64, angles=[0.0, float("nan")])], [tm.Group(N=64, angles=[0.0], span=0.0)]):
        with pytest.raises(tm.TmbirError) as e:
            tm.Context(bad)
        assert e.value.code == -1
    ctx = tm.Context([tm.Group(N=64, angles=[0.0, 1.0])])
    x = torch.zeros(64 * 64 + 1, device="cuda")
    with pytest.raises(tm.TmbirError) as e:
        ctx.normal_apply(x)  # operator not built yet
    assert e.value.code == -7
    sino = torch.zeros(2 * 64 + 4, device="cuda")
    with pytest.raises(tm.TmbirError) as e:
        ctx.build_operator(sino[1:], torch.zeros(64 * 64, device="cuda"))  # misaligned
    assert e.value.code == -1
    with pytest.raises(tm.TmbirError) as e:
        ctx.downsample_sino(sino, 1, 2, 64, 3)
    assert e.value.code == -1


def test_nonfinite_input_is_reported():
    p = synth.volume(S=1, N=64, n_angles=20, n_ellipsoids=3, seed=77)
    ctx = tm.Context([tm.Group(N=64, angles=list(p.theta))])
    atg = ctx.build_operator(dev(p.sino))
    x = torch.zeros(64 * 64, device="cuda")
    x[100] = float("nan")
    with pytest.raises(tm.TmbirError) as e:
        ctx.reconstruct(x, atg, tm.Params(max_iter=5))
    assert e.value.code == -6


def test_bounded_wait_gives_up_and_the_context_stays_usable():
    """A device wait that nothing satisfies gives up after its poll bound: the call reports
    TMBIR_ERR_TIMEOUT, no GPU fault or hang, and the context keeps working."""
    p = synth.volume(S=1, N=64, n_angles=20, n_ellipsoids=3, seed=77)
    ctx = tm.Context([tm.Group(N=64, angles=list(p.theta))])
    ctx.build_operator(dev(p.sino))
    x = dev(synth.random_image(np.random.default_rng(3), (64, 64), 0.5))
    before = host(ctx.normal_apply(x), (64, 64))
    ctx.wait_check(1 << 20, arrive=True)
    with pytest.raises(tm.TmbirError) as e:
        ctx.wait_check(1000, arrive=False)
    assert e.value.code == -5
    ctx.wait_check(1 << 20, arrive=True)
    after = host(ctx.normal_apply(x), (64, 64))
    assert np.array_equal(before, after)


def test_fp32_setup_for_coarse_levels(prob, orc):
    """tmbir_build_operator_fp32: R*g from the FP32 back-projection (within FP32 transform
    error of the oracle's sums), the same kernel, lambda_max and 1/2 g.g as the FP64 build."""
    ctx = tm.Context([tm.Group(N=prob.N, angles=list(prob.theta), n_slices=prob.S, span=prob.span)])
    atg32 = ctx.build_operator(prob.d_sino, fp64=False)
    assert rel(host(atg32, prob.atg.shape), prob.atg) < 1e-5
    assert torch.equal(ctx.kernel(0), prob.ctx.kernel(0))
    assert ctx.lambda_max()[0] == prob.ctx.lambda_max()[0]
    F64 = prob.ctx.objective(dev(prob.x), prob.d_atg, tm.Params(**PRIOR))
    F32 = ctx.objective(dev(prob.x), atg32, tm.Params(**PRIOR))
    assert abs(F32 - F64) <= 1e-5 * abs(F64)
