"""Learned warm start: the CUDA network against the FP64 oracle, and what training buys.

BF16 activations and weight copies bound the agreement: outputs and gradients within 2e-2
relative L2 of the oracle (FP64, plain loops).
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


def rel(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def random_params(orc, seed):
    rng = np.random.default_rng(seed)
    p = np.zeros(orc.cnn_param_count())
    for ws, bs, cin, cout in orc.cnn_layer_slices():
        p[ws] = rng.normal(0, math.sqrt(2.0 / (9 * cin)), ws.stop - ws.start)
        p[bs] = rng.normal(0, 0.05, bs.stop - bs.start)
    return p.astype(np.float32).astype(np.float64)


# Image widths against the 128-pixel rows of one tensor-core tile: 36 and 64 are one partial tile;
# 300 is two full tiles and a partial one (unmasked tiles and the halo handed from tile to tile);
# 2560 is twenty full tiles, the row width of the largest slices.  Heights 6, 12, 20 and 33 end
# the four-row tile groups full and partial.
@pytest.mark.parametrize("B,H,W", [(2, 20, 36), (2, 33, 64), (2, 12, 300), (1, 6, 2560)])
def test_forward_matches_oracle(orc, B, H, W):
    p = random_params(orc, 1)
    net = tm.CNN(H, W, max_batch=B)
    net.set_weights(p)
    x = np.random.default_rng(2).standard_normal((B, H, W)).astype(np.float32)
    out = net.net_forward(dev(x), B)
    torch.cuda.synchronize()
    ref = orc.cnn_forward(x.astype(np.float64), p)
    assert rel(out.cpu().numpy().reshape(ref.shape), ref) < 2e-2


def robust_params(orc, seed):
    """Hidden units that are clearly on or off: bias +-1 (+-3 in the first layer) dominates
    the weighted inputs, so no ReLU decision depends on the rounding of either side."""
    rng = np.random.default_rng(seed)
    p = np.zeros(orc.cnn_param_count())
    for l, (ws, bs, cin, cout) in enumerate(orc.cnn_layer_slices()):
        scale = 1.0 if l in (0, 3) else 0.1
        p[ws] = rng.normal(0, math.sqrt(2.0 / (9 * cin)), ws.stop - ws.start) * scale
        if l < 3:
            p[bs] = rng.choice([-1.0, 1.0], bs.stop - bs.start) * (3.0 if l == 0 else 1.0)
    return p.astype(np.float32).astype(np.float64)


def min_preactivation(orc, x, p):
    """Smallest |pre-activation| of the three hidden layers (FP64, 'same' 3x3 correlation)."""
    from scipy.signal import correlate2d

    layers = [(p[ws].reshape(cout, cin, 3, 3), p[bs]) for ws, bs, cin, cout in orc.cnn_layer_slices()]
    m = np.inf
    for img in x:
        a = img[None].astype(np.float64)
        for Wl, bl in layers[:3]:
            z = np.stack([sum(correlate2d(a[ci], Wl[co, ci], mode="same") for ci in range(a.shape[0])) + bl[co]
                          for co in range(Wl.shape[0])])
            m = min(m, float(np.abs(z).min()))
            a = np.maximum(z, 0)
    return m


def check_backward(orc, p, x, gout, tol):
    B, H, W = x.shape
    net = tm.CNN(H, W, max_batch=B)
    net.set_weights(p)
    gp, gin = net.net_backward(dev(x), dev(gout), B)
    torch.cuda.synchronize()
    rgp, rgin = orc.cnn_backward(x.astype(np.float64), p, gout.astype(np.float64))
    for ws, bs, cin, cout in orc.cnn_layer_slices():
        assert rel(gp[ws], rgp[ws]) < tol, ("weights", cin, cout, rel(gp[ws], rgp[ws]))
        assert rel(gp[bs], rgp[bs]) < tol, ("bias", cin, cout, rel(gp[bs], rgp[bs]))
    assert rel(gin.cpu().numpy().reshape(rgin.shape), rgin) < tol


@pytest.mark.parametrize("B,H,W", [(2, 18, 40), (2, 12, 300), (1, 6, 2560)])
def test_backward_matches_oracle(orc, B, H, W):
    # Every ReLU decision is the same on both sides (margin far above the BF16 error of a
    # pre-activation), so the gradients differ only by BF16 rounding of activations, gradients
    # and weight copies: 2^-9 per operand, a few 1e-3 after three layers and up to about 1e-2
    # in the bias sums, whose terms cancel (BF16 rounding modelled on the CPU: at most 9e-3).
    # Widths as in the forward test: one partial tile, two full tiles and a partial one, and
    # twenty full tiles.
    rng = np.random.default_rng(4)
    p = robust_params(orc, 3)
    x = rng.uniform(-0.5, 0.5, (B, H, W)).astype(np.float32)
    gout = rng.standard_normal((B, H, W)).astype(np.float32)
    assert min_preactivation(orc, x, p) > 0.1
    check_backward(orc, p, x, gout, 2e-2)


@pytest.mark.parametrize("B,H,W", [(2, 18, 40), (2, 12, 300)])
def test_backward_random_network(orc, B, H, W):
    # A random He-initialised network has pre-activations near zero, where BF16 rounding
    # flips the ReLU decision of a small fraction f of units; each flip moves a gradient term
    # by its full size, so the relative L2 error grows like sqrt(f) rather than like the unit
    # roundoff (BF16 rounding modelled on the CPU: 4e-2 to 8e-2 across the parameter blocks).
    p = random_params(orc, 3)
    rng = np.random.default_rng(4)
    x = rng.standard_normal((B, H, W)).astype(np.float32)
    gout = rng.standard_normal((B, H, W)).astype(np.float32)
    check_backward(orc, p, x, gout, 0.15)


def test_apply_is_residual(orc):
    # a zero network leaves the start unchanged: x + s * 0
    net = tm.CNN(16, 16, max_batch=1)
    net.set_weights(np.zeros(orc.cnn_param_count()))
    x = dev(np.random.default_rng(5).uniform(0, 1, (16, 16)))
    y = net.apply(x, 1)
    torch.cuda.synchronize()
    assert torch.equal(x, y)


def make_pairs(N, S, na, seeds, iters):
    """(FBP start, converged reconstruction, sinogram, theta) of several random volumes."""
    out = []
    for sd in seeds:
        p = synth.volume(S=S, N=N, n_angles=na, n_ellipsoids=6, seed=sd)
        ctx = tm.Context([tm.Group(N=N, angles=list(p.theta), n_slices=S)])
        sino = dev(p.sino)
        atg = ctx.build_operator(sino)
        fbp = ctx.fbp(sino)
        x = fbp.clone()
        ctx.reconstruct(x, atg, tm.Params(**PRIOR, max_iter=iters))
        torch.cuda.synchronize()
        out.append((ctx, fbp, x, atg))
    return out


def test_trained_network_improves_the_start():
    N, S, na = 64, 8, 30
    train = make_pairs(N, S, na, seeds=range(300, 306), iters=400)
    held = make_pairs(N, S, na, seeds=[400, 401], iters=400)
    net = tm.CNN(N, N, max_batch=S, seed=7)
    losses = []
    for epoch in range(40):
        for ctx, fbp, x, atg in train:
            losses.append(net.train_step(fbp, x, S, lr=2e-3))
    assert np.mean(losses[-len(train):]) < 0.5 * np.mean(losses[:len(train)])
    prm = tm.Params(**PRIOR)
    gains = []
    for ctx, fbp, xstar, atg in held:
        x0, used = net.warm_start(ctx, fbp, atg, prm)
        F_fbp = ctx.objective(fbp, atg, prm)
        F_cnn = ctx.objective(x0, atg, prm)
        F_star = ctx.objective(xstar, atg, prm)
        assert used and F_cnn < F_fbp
        # relative gap of the start: what the network removes before the first iteration
        gains.append((F_fbp - F_star) / (F_cnn - F_star))
        # and after 20 iterations from each start
        a, b = fbp.clone(), x0.clone()
        sa = ctx.reconstruct(a, atg, tm.Params(**PRIOR, max_iter=20))
        sb = ctx.reconstruct(b, atg, tm.Params(**PRIOR, max_iter=20))
        assert sb.objective < sa.objective
    assert min(gains) > 1.5
