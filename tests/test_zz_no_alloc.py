"""tmbir_normal_apply_static: the normal operator with its scratch in the library's fixed
device array, for callers that cannot allocate device memory when they call (for example code
running inside a host application that owns the whole device-memory budget).  Its output must
match tmbir_normal_apply (the workspace-scratch entry point) on two calls in a row, also for
volumes whose spectra exceed the array (they run in slice chunks), and its first call must not
change the device's free memory: the array is committed when the context is created.  Kept in
its own file, collected last."""
import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2603_28756_gb300 as tm  # noqa: E402


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32).ravel()).cuda()


def test_static_scratch_matches_workspace_path_twice():
    specs = [(64, 3, 30), (128, 2, 40)]
    groups, sinos = [], []
    for k, (N, S, na) in enumerate(specs):
        p = synth.volume(S=S, N=N, n_angles=na, n_ellipsoids=4, seed=60 + k)
        groups.append(tm.Group(N=N, angles=list(p.theta), n_slices=S))
        sinos.append(p.sino.ravel())
    ctx = tm.Context(groups)
    ctx.build_operator(_dev(np.concatenate(sinos)))
    rng = np.random.default_rng(8)
    x = _dev(np.concatenate([synth.random_image(rng, (S, N, N)).ravel() for N, S, _ in specs]))
    ref = ctx.normal_apply(x)
    z = torch.empty_like(ref)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for k in range(2):
        ctx.normal_apply_static(x, out=z)
        torch.cuda.synchronize()
        if k == 0:
            # the array was committed by tmbir_create: the first call takes no device memory
            assert torch.cuda.mem_get_info()[0] == free0
        err = float(torch.linalg.norm((z - ref).double()) / torch.linalg.norm(ref.double()))
        assert err < 1e-5, err


def test_static_scratch_runs_volumes_beyond_the_array_in_chunks():
    N, S, na = 1024, 9, 16  # 9 * 1025 * 1024 complex values: more than the 8 Mi of the array
    p = synth.volume(S=S, N=N, n_angles=na, n_ellipsoids=4, seed=62)
    ctx = tm.Context([tm.Group(N=N, angles=list(p.theta), n_slices=S)])
    ctx.build_operator(_dev(p.sino))
    x = _dev(synth.random_image(np.random.default_rng(9), (S, N, N)))
    ref = ctx.normal_apply(x)
    z = ctx.normal_apply_static(x)
    torch.cuda.synchronize()
    err = float(torch.linalg.norm((z - ref).double()) / torch.linalg.norm(ref.double()))
    assert err < 1e-5, err


def test_static_scratch_two_groups_with_chunks():
    # 9 slices of 1024^2 (two chunks of the array, the second reusing the spectra of the first)
    # then 3 of 512^2 (one chunk, after the first group's chunks have used the array)
    specs = [(1024, 9, 16), (512, 3, 24)]
    groups, sinos = [], []
    for k, (N, S, na) in enumerate(specs):
        p = synth.volume(S=S, N=N, n_angles=na, n_ellipsoids=4, seed=70 + k)
        groups.append(tm.Group(N=N, angles=list(p.theta), n_slices=S))
        sinos.append(p.sino.ravel())
    ctx = tm.Context(groups)
    ctx.build_operator(_dev(np.concatenate(sinos)))
    rng = np.random.default_rng(10)
    x = _dev(np.concatenate([synth.random_image(rng, (S, N, N)).ravel() for N, S, _ in specs]))
    ref = ctx.normal_apply(x)
    for _ in range(2):
        z = ctx.normal_apply_static(x)
        torch.cuda.synchronize()
        off = 0
        for N, S, _ in specs:
            n = S * N * N
            a, b = z[off:off + n].double(), ref[off:off + n].double()
            err = float(torch.linalg.norm(a - b) / torch.linalg.norm(b))
            assert err < 1e-5, (N, err)
            off += n
