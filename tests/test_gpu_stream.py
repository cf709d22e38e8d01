"""Host volumes streamed through the GPU in slabs (Sec. 2.4: partitions along the rotation axis
with halo slices for the 26-neighbour prior, copies overlapped with the kernels), through the C
ABI.  A slab context must give the resident context's R*g and iterates bit for bit (same kernels,
same pairing of slices in the setup transforms, partial sums reduced in the resident order), and
follow the FP64 oracle like the resident path does.
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


def pinned(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32).ravel()).pin_memory()


def host(t, shape):
    torch.cuda.synchronize()
    return t.double().cpu().numpy().reshape(shape)


class Volume:
    def __init__(self, N, S, na, span, slab, seed):
        self.N, self.S, self.na, self.span, self.slab = N, S, na, span, slab
        p = synth.volume(S=S, N=N, n_angles=na, n_ellipsoids=6, span=span, seed=seed)
        self.theta, self.sino = p.theta, p.sino
        self.res = tm.Context([tm.Group(N=N, angles=list(p.theta), n_slices=S, span=span)])
        self.slabctx = tm.Context([tm.Group(N=N, angles=list(p.theta), n_slices=slab, span=span)])
        self.d_atg, self.d_x0 = self.res.build_operator_fbp(dev(p.sino))
        self.h_atg, self.gtg, self.h_x0 = self.slabctx.stream_build_operator(pinned(p.sino), S, fbp=True)


@pytest.fixture(scope="module", params=[(64, 11, 37, math.pi, 4), (128, 6, 45, 2 * math.pi / 3, 2)],
                ids=["N64-11sl-slab4", "N128limited-6sl-slab2"])
def vol(request):
    N, S, na, span, slab = request.param
    return Volume(N, S, na, span, slab, seed=21)


def test_streamed_setup_equals_resident(vol):
    torch.cuda.synchronize()
    assert torch.equal(vol.h_atg, vol.d_atg.cpu())
    assert torch.equal(vol.h_x0, vol.d_x0.cpu())
    gtg = 0.5 * float(np.sum(vol.sino.astype(np.float64) ** 2))
    assert abs(vol.gtg - gtg) <= 1e-12 * gtg


@pytest.mark.parametrize("mode", ["fp32", "bf16_refined", "fp32_device_atg"])
def test_streamed_iterates_equal_resident(vol, mode):
    """Every iterate, the stats and the log of a streamed run equal the resident run's (the
    resident and the slab contexts both take one slice per pass-3b block at these sizes); R*g
    may stay in device memory while the iterates stream."""
    kw = dict(PRIOR, max_iter=12)
    if mode == "bf16_refined":
        # refinement needs a reference objective: a longer FP32 run of the resident volume
        xr = vol.d_x0.clone()
        Fref = vol.res.reconstruct(xr, vol.d_atg, tm.Params(**PRIOR, max_iter=200)).objective
        kw.update(bf16=True, refine_gap=0.5, F_ref=Fref)
    x = vol.d_x0.clone()
    st = vol.res.reconstruct(x, vol.d_atg, tm.Params(**kw))
    log = vol.res.get_log()
    hx = vol.h_x0.clone()
    atg = vol.d_atg if mode == "fp32_device_atg" else vol.h_atg
    sst = vol.slabctx.stream_reconstruct(hx, atg, vol.gtg, tm.Params(**kw))
    slog = vol.slabctx.get_log()
    torch.cuda.synchronize()
    assert torch.equal(hx, x.cpu())
    assert (sst.iterations, sst.restarts, sst.status) == (st.iterations, st.restarts, st.status)
    assert abs(sst.objective - st.objective) <= 1e-12 * abs(st.objective)
    assert len(slog) == len(log) == st.iterations
    for a, b in zip(slog, log):
        assert abs(a[0] - b[0]) <= 1e-12 * abs(b[0])
        assert a[1:] == b[1:]


def test_streamed_run_follows_oracle(vol, orc):
    pr = orc.Prior(**PRIOR)
    iters = 10
    g = vol.sino.astype(np.float64)
    K = orc.kernel(vol.N, vol.theta, vol.N)
    atg = orc.adjoint(g, vol.N, vol.theta)
    L = orc.lipschitz(K, vol.N, pr)
    hx = vol.h_x0.clone()
    st = vol.slabctx.stream_reconstruct(hx, vol.h_atg, vol.gtg, tm.Params(**PRIOR, max_iter=iters))
    assert st.iterations == iters and abs(st.L - L) <= 1e-5 * L
    x0 = vol.h_x0.double().numpy().reshape(vol.S, vol.N, vol.N)
    ref = orc.nesterov(x0, atg, float(np.sum(g ** 2)), K, pr, L, iters)
    assert rel(hx.double().numpy().reshape(ref.shape), ref) < 1e-4


def test_stream_gap_stop_and_one_slab(vol):
    """The gap rule ends a streamed run where it ends the resident one; a slab holding the whole
    volume is the resident run."""
    xr = vol.d_x0.clone()
    Fref = vol.res.reconstruct(xr, vol.d_atg, tm.Params(**PRIOR, max_iter=200)).objective
    kw = dict(PRIOR, max_iter=200, gap_tol=1e-2, F_ref=Fref)
    x = vol.d_x0.clone()
    st = vol.res.reconstruct(x, vol.d_atg, tm.Params(**kw))
    hx = vol.h_x0.clone()
    sst = vol.slabctx.stream_reconstruct(hx, vol.h_atg, vol.gtg, tm.Params(**kw))
    assert st.iterations < 200 and sst.iterations == st.iterations
    torch.cuda.synchronize()
    assert torch.equal(hx, x.cpu())
    whole = tm.Context([tm.Group(N=vol.N, angles=list(vol.theta), n_slices=vol.S, span=vol.span)])
    h_atg, gtg, _ = whole.stream_build_operator(pinned(vol.sino), vol.S)
    hx1 = vol.h_x0.clone()
    whole.stream_reconstruct(hx1, h_atg, gtg, tm.Params(**kw))
    assert torch.equal(hx1, x.cpu())


def test_stream_argument_errors(vol):
    lib = tm.load()
    import ctypes

    pr = tm.Params(**PRIOR, max_iter=2).c_struct()
    hx = vol.h_x0.clone()
    ws, nb = vol.slabctx._stream_work(vol.S)
    work = torch.empty(2 * hx.numel(), dtype=torch.float32, pin_memory=True)
    args = [vol.slabctx._h, vol.S, ctypes.c_void_p(hx.data_ptr()), ctypes.c_void_p(vol.h_atg.data_ptr()), vol.gtg,
            ctypes.c_void_p(work.data_ptr()), ctypes.c_void_p(ws)]
    assert lib.tmbir_stream_reconstruct(*args, 1024, ctypes.byref(pr), None) == -3  # workspace too small
    pr.resume = 1
    assert lib.tmbir_stream_reconstruct(*args, nb, ctypes.byref(pr), None) == -1  # resume refused
    two = tm.Context([tm.Group(N=vol.N, angles=list(vol.theta), n_slices=2, span=vol.span)] * 2)
    size = ctypes.c_size_t()
    assert lib.tmbir_stream_workspace_size(two._h, vol.S, ctypes.byref(size)) == -1  # one group only
    assert lib.tmbir_stream_workspace_size(vol.slabctx._h, 0, ctypes.byref(size)) == -1
