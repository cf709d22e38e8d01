"""Toeplitz-accelerated MBIR on one GB300: thin Python binding over the libtmbir C ABI.

Every computation runs in the CUDA library (``include/tmbir.h``); this module only
marshals arguments.  PyTorch provides device memory and the stream.  There is no CPU
fallback: if the library is missing or no GPU is present the calls raise.
"""
from __future__ import annotations

import ctypes
import math
import os
from dataclasses import dataclass, field

from .build import LIB, build  # noqa: F401

__all__ = ["CNN", "Context", "Group", "Params", "Stats", "TmbirError", "load", "SYMBOLS", "build", "reconstruct_levels"]

TMBIR_OK = 0
ERRORS = {
    -1: "TMBIR_ERR_ARG",
    -2: "TMBIR_ERR_SHAPE",
    -3: "TMBIR_ERR_WORKSPACE",
    -4: "TMBIR_ERR_CUDA",
    -5: "TMBIR_ERR_TIMEOUT",
    -6: "TMBIR_ERR_NONFINITE",
    -7: "TMBIR_ERR_STATE",
}


class TmbirError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{ERRORS.get(code, code)}: {msg}")
        self.code = code


class _Group(ctypes.Structure):
    _fields_ = [
        ("N", ctypes.c_int),
        ("n_det", ctypes.c_int),
        ("n_angles", ctypes.c_int),
        ("angles", ctypes.POINTER(ctypes.c_double)),
        ("span", ctypes.c_double),
        ("n_slices", ctypes.c_int),
    ]


class _Params(ctypes.Structure):
    _fields_ = [
        ("p", ctypes.c_double),
        ("q", ctypes.c_double),
        ("c", ctypes.c_double),
        ("sigma", ctypes.c_double),
        ("lambda_", ctypes.c_double),
        ("L", ctypes.c_double),
        ("max_iter", ctypes.c_int),
        ("gap_tol", ctypes.c_double),
        ("F_ref", ctypes.c_double),
        ("restart", ctypes.c_int),
        ("use_graph", ctypes.c_int),
        ("spectra", ctypes.c_int),
        ("refine_gap", ctypes.c_double),
        ("resume", ctypes.c_int),
        ("nonneg", ctypes.c_int),
    ]


class _Stats(ctypes.Structure):
    _fields_ = [
        ("iterations", ctypes.c_int),
        ("restarts", ctypes.c_int),
        ("status", ctypes.c_int),
        ("objective", ctypes.c_double),
        ("gap", ctypes.c_double),
        ("L", ctypes.c_double),
        ("grad_norm", ctypes.c_double),
    ]


SYMBOLS = [
    "tmbir_create", "tmbir_destroy", "tmbir_last_error", "tmbir_set_geometry", "tmbir_workspace_size",
    "tmbir_set_workspace", "tmbir_build_operator", "tmbir_fbp", "tmbir_reconstruct", "tmbir_get_log",
    "tmbir_normal_apply", "tmbir_gradient", "tmbir_step", "tmbir_objective", "tmbir_lambda_max", "tmbir_kernel",
    "tmbir_upsample_lanczos3", "tmbir_downsample_sino", "tmbir_sync", "tmbir_pass_times", "tmbir_launch_count",
    "tmbir_normal_apply_static", "tmbir_cnn_param_count", "tmbir_cnn_workspace_size", "tmbir_cnn_create",
    "tmbir_cnn_destroy", "tmbir_cnn_init", "tmbir_cnn_set_weights", "tmbir_cnn_get_weights", "tmbir_cnn_apply",
    "tmbir_cnn_train_step", "tmbir_cnn_net_forward", "tmbir_cnn_net_backward", "tmbir_warm_start",
    "tmbir_state_size", "tmbir_state_export", "tmbir_state_import", "tmbir_autotune", "tmbir_build_operator_fbp",
    "tmbir_wait_check", "tmbir_forward", "tmbir_adjoint", "tmbir_gradient_direct", "tmbir_sfu_rate",
    "tmbir_stream_workspace_size", "tmbir_stream_build_operator", "tmbir_stream_reconstruct",
    "tmbir_build_operator_fp32", "tmbir_set_angle_weights",
]

_lib = None


def load(path: str | None = None):
    """Load libtmbir.so (building it first if the sources are newer).  Raises if it cannot."""
    global _lib
    if _lib is not None:
        return _lib
    so = path or build()
    if not os.path.exists(so):
        raise RuntimeError(f"libtmbir.so not found at {so}; run paper_2603_28756_gb300.build.build()")
    L = ctypes.CDLL(so)
    vp, i, d, sz = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_size_t
    dp = ctypes.POINTER(ctypes.c_double)
    sig = {
        "tmbir_create": [ctypes.POINTER(vp), vp],
        "tmbir_destroy": [vp],
        "tmbir_set_geometry": [vp, i, ctypes.POINTER(_Group)],
        "tmbir_workspace_size": [vp, ctypes.POINTER(sz)],
        "tmbir_set_workspace": [vp, vp, sz],
        "tmbir_build_operator": [vp, vp, vp],
        "tmbir_build_operator_fp32": [vp, vp, vp],
        "tmbir_set_angle_weights": [vp, i, dp],
        "tmbir_fbp": [vp, vp, vp],
        "tmbir_reconstruct": [vp, vp, vp, ctypes.POINTER(_Params), ctypes.POINTER(_Stats)],
        "tmbir_get_log": [vp, dp, i, ctypes.POINTER(i)],
        "tmbir_normal_apply": [vp, vp, vp],
        "tmbir_gradient": [vp, vp, vp, ctypes.POINTER(_Params), vp],
        "tmbir_step": [vp, vp, vp, d, vp, ctypes.POINTER(_Params), d, vp, dp],
        "tmbir_objective": [vp, vp, vp, ctypes.POINTER(_Params), dp],
        "tmbir_lambda_max": [vp, dp],
        "tmbir_kernel": [vp, i, vp],
        "tmbir_upsample_lanczos3": [vp, vp, i, i, vp],
        "tmbir_downsample_sino": [vp, vp, i, i, i, i, vp],
        "tmbir_sync": [vp],
        "tmbir_pass_times": [vp, vp, vp, ctypes.POINTER(_Params), i, dp],
        "tmbir_launch_count": [vp, ctypes.POINTER(ctypes.c_longlong)],
        "tmbir_normal_apply_static": [vp, vp, vp],
        "tmbir_wait_check": [vp, ctypes.c_uint, i],
        "tmbir_cnn_param_count": [],
        "tmbir_cnn_workspace_size": [i, i, i, ctypes.POINTER(sz)],
        "tmbir_cnn_create": [ctypes.POINTER(vp), vp, i, i, i, vp, sz],
        "tmbir_cnn_destroy": [vp],
        "tmbir_cnn_init": [vp, ctypes.c_ulonglong],
        "tmbir_cnn_set_weights": [vp, ctypes.POINTER(ctypes.c_float)],
        "tmbir_cnn_get_weights": [vp, ctypes.POINTER(ctypes.c_float)],
        "tmbir_cnn_apply": [vp, vp, i, vp],
        "tmbir_cnn_train_step": [vp, vp, vp, i, ctypes.c_float, dp],
        "tmbir_cnn_net_forward": [vp, vp, i, vp],
        "tmbir_cnn_net_backward": [vp, vp, vp, i, ctypes.POINTER(ctypes.c_float), vp],
        "tmbir_warm_start": [vp, vp, vp, vp, ctypes.POINTER(_Params), vp, ctypes.POINTER(i)],
        "tmbir_state_size": [vp, ctypes.POINTER(sz)],
        "tmbir_state_export": [vp, vp],
        "tmbir_state_import": [vp, vp],
        "tmbir_autotune": [vp, vp, vp, ctypes.POINTER(_Params), ctypes.POINTER(i), ctypes.POINTER(i)],
        "tmbir_build_operator_fbp": [vp, vp, vp, vp],
        "tmbir_forward": [vp, vp, vp],
        "tmbir_adjoint": [vp, vp, vp],
        "tmbir_gradient_direct": [vp, vp, vp, ctypes.POINTER(_Params), vp, dp],
        "tmbir_sfu_rate": [vp, i, dp],
        "tmbir_stream_workspace_size": [vp, i, ctypes.POINTER(sz)],
        "tmbir_stream_build_operator": [vp, i, vp, vp, vp, vp, sz, dp],
        "tmbir_stream_reconstruct": [vp, i, vp, vp, d, vp, vp, sz, ctypes.POINTER(_Params), ctypes.POINTER(_Stats)],
    }
    for name, args in sig.items():
        f = getattr(L, name)
        f.argtypes = args
        f.restype = ctypes.c_int
    L.tmbir_last_error.restype = ctypes.c_char_p
    L.tmbir_last_error.argtypes = []
    _lib = L
    return L


def _check(code: int):
    if code != TMBIR_OK:
        raise TmbirError(code, _lib.tmbir_last_error().decode(errors="replace"))


@dataclass
class Group:
    """n_slices slices of N x N seen under `angles` (radians) covering `span` radians."""

    N: int
    angles: list
    n_slices: int = 1
    span: float = math.pi
    n_det: int | None = None


@dataclass
class Params:
    """qGGMRF prior and optimiser settings (see tmbir_params in include/tmbir.h)."""

    p: float = 1.2
    q: float = 2.0
    c: float = 0.01
    sigma: float = 0.1
    lam: float = 1.0
    L: float = 0.0
    max_iter: int = 50
    gap_tol: float = 0.0
    F_ref: float = 0.0
    restart: int = 0
    use_graph: bool = True
    bf16: bool = False  # BF16 storage of the intermediate spectrum
    refine_gap: float = 0.0  # with bf16: switch to FP32 spectra once the gap is <= refine_gap
    resume: bool = False  # continue the context's run (or an imported checkpoint)
    nonneg: bool = False  # project every iterate onto x >= 0

    def c_struct(self) -> _Params:
        return _Params(self.p, self.q, self.c, self.sigma, self.lam, self.L, self.max_iter, self.gap_tol, self.F_ref,
                       self.restart, 1 if self.use_graph else 0, 1 if self.bf16 else 0, self.refine_gap,
                       1 if self.resume else 0, 1 if self.nonneg else 0)


@dataclass
class Stats:
    iterations: int
    restarts: int
    status: int
    objective: float
    gap: float
    L: float
    grad_norm: float


def _ptr(t) -> int:
    import torch

    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError("expected a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError("tensor must be contiguous")
    return t.data_ptr()


class Context:
    """One libtmbir context bound to a CUDA stream, with a torch-allocated workspace."""

    def __init__(self, groups, stream=None, device="cuda"):
        import torch

        load()
        self.device = torch.device(device)
        self.stream = stream if stream is not None else torch.cuda.Stream(device=self.device)
        h = ctypes.c_void_p()
        _check(_lib.tmbir_create(ctypes.byref(h), ctypes.c_void_p(self.stream.cuda_stream)))
        self._h = h
        self.groups = [g if isinstance(g, Group) else Group(**g) for g in groups]
        self._angle_bufs = []
        arr = (_Group * len(self.groups))()
        for k, g in enumerate(self.groups):
            a = (ctypes.c_double * len(g.angles))(*[float(v) for v in g.angles])
            self._angle_bufs.append(a)
            arr[k] = _Group(g.N, g.n_det or g.N, len(g.angles), ctypes.cast(a, ctypes.POINTER(ctypes.c_double)),
                            float(g.span), g.n_slices)
        _check(_lib.tmbir_set_geometry(self._h, len(self.groups), arr))
        nbytes = ctypes.c_size_t()
        _check(_lib.tmbir_workspace_size(self._h, ctypes.byref(nbytes)))
        self.workspace_bytes = nbytes.value
        with torch.cuda.stream(self.stream):
            self.workspace = torch.empty(nbytes.value + 256, dtype=torch.uint8, device=self.device)
        base = self.workspace.data_ptr()
        aligned = (base + 255) // 256 * 256
        _check(_lib.tmbir_set_workspace(self._h, ctypes.c_void_p(aligned), nbytes.value))

    # shapes -----------------------------------------------------------------
    @property
    def n_slices(self) -> int:
        return sum(g.n_slices for g in self.groups)

    def image_numel(self) -> int:
        return sum(g.n_slices * g.N * g.N for g in self.groups)

    def sino_numel(self) -> int:
        return sum(g.n_slices * len(g.angles) * (g.n_det or g.N) for g in self.groups)

    def _empty(self, n):
        import torch

        with torch.cuda.stream(self.stream):
            return torch.empty(n, dtype=torch.float32, device=self.device)

    # stream ordering: the context stream is a PyTorch side stream (non-blocking), so every
    # call first makes it wait for the caller's current stream (inputs written there) and
    # afterwards makes the caller's stream wait for it (outputs read there); input tensors are
    # marked as used on the context stream so the caching allocator does not recycle them early.
    def _pre(self):
        import torch

        cur = torch.cuda.current_stream(self.device)
        if cur != self.stream:
            self.stream.wait_stream(cur)

    def _post(self, *tensors):
        import torch

        cur = torch.cuda.current_stream(self.device)
        if cur != self.stream:
            cur.wait_stream(self.stream)
            for t in tensors:
                if t is not None:
                    t.record_stream(self.stream)

    # calls --------------------------------------------------------------------
    def set_angle_weights(self, group: int, weights=None):
        """Per-angle data-term weights in [0, 1] for one group (None: all 1); the next
        build_operator rebuilds K, lambda_max, R*g and 1/2 g.g with them."""
        if weights is None:
            _check(_lib.tmbir_set_angle_weights(self._h, int(group), None))
            return
        w = (ctypes.c_double * len(weights))(*[float(v) for v in weights])
        if 0 <= group < len(self.groups) and len(weights) != len(self.groups[group].angles):
            raise ValueError("one weight per angle")
        _check(_lib.tmbir_set_angle_weights(self._h, int(group), w))

    def build_operator(self, sino, atg=None, fp64: bool = True):
        """K, its spectrum, lambda_max, 1/2 g.g and R*g (FP64, or FP32 with fp64=False)."""
        atg = self._empty(self.image_numel()) if atg is None else atg
        self._pre()
        fn = _lib.tmbir_build_operator if fp64 else _lib.tmbir_build_operator_fp32
        _check(fn(self._h, ctypes.c_void_p(_ptr(sino)), ctypes.c_void_p(_ptr(atg))))
        self._post(sino, atg)
        return atg

    def build_operator_fbp(self, sino, atg=None, x0=None):
        """build_operator and fbp overlapped on two streams; returns (atg, x0)."""
        atg = self._empty(self.image_numel()) if atg is None else atg
        x0 = self._empty(self.image_numel()) if x0 is None else x0
        self._pre()
        _check(_lib.tmbir_build_operator_fbp(self._h, ctypes.c_void_p(_ptr(sino)), ctypes.c_void_p(_ptr(atg)),
                                             ctypes.c_void_p(_ptr(x0))))
        self._post(sino, atg, x0)
        return atg, x0

    def fbp(self, sino, out=None):
        out = self._empty(self.image_numel()) if out is None else out
        self._pre()
        _check(_lib.tmbir_fbp(self._h, ctypes.c_void_p(_ptr(sino)), ctypes.c_void_p(_ptr(out))))
        self._post(sino, out)
        return out

    def reconstruct(self, x, atg, params: Params, want_stats: bool = True):
        st = _Stats()
        pr = params.c_struct()
        self._pre()
        _check(_lib.tmbir_reconstruct(self._h, ctypes.c_void_p(_ptr(x)), ctypes.c_void_p(_ptr(atg)), ctypes.byref(pr),
                                      ctypes.byref(st) if want_stats else None))
        self._post(x, atg)
        if not want_stats:
            return None
        return Stats(st.iterations, st.restarts, st.status, st.objective, st.gap, st.L, st.grad_norm)

    # host volumes (tmbir_stream_*): the context's one group is the slab ---------------------
    def _stream_work(self, n_slices: int):
        import torch

        nbytes = ctypes.c_size_t()
        _check(_lib.tmbir_stream_workspace_size(self._h, int(n_slices), ctypes.byref(nbytes)))
        if getattr(self, "_swork_key", None) != (n_slices, nbytes.value):
            with torch.cuda.stream(self.stream):
                self._swork = torch.empty(nbytes.value + 256, dtype=torch.uint8, device=self.device)
            self._swork_key = (n_slices, nbytes.value)
        base = self._swork.data_ptr()
        return (base + 255) // 256 * 256, nbytes.value

    def stream_build_operator(self, h_sino, n_slices: int, fbp: bool = False):
        """R*g (and the FBP start) of a host volume of n_slices slices, slab by slab.
        h_sino: a contiguous float32 CPU tensor (page-locked for overlapped copies).
        Returns (h_atg, gtg_half, h_x0 or None) as page-locked CPU tensors."""
        import torch

        g = self.groups[0]
        if h_sino.is_cuda or not h_sino.is_contiguous() or h_sino.dtype != torch.float32:
            raise TypeError("expected a contiguous float32 CPU tensor")
        if h_sino.numel() != n_slices * len(g.angles) * (g.n_det or g.N):
            raise ValueError("sinogram size does not match n_slices")
        nimg = n_slices * g.N * g.N
        h_atg = torch.empty(nimg, dtype=torch.float32, pin_memory=True)
        h_x0 = torch.empty(nimg, dtype=torch.float32, pin_memory=True) if fbp else None
        ws, nb = self._stream_work(n_slices)
        gtg = ctypes.c_double()
        self._pre()
        _check(_lib.tmbir_stream_build_operator(self._h, int(n_slices), ctypes.c_void_p(h_sino.data_ptr()),
                                                ctypes.c_void_p(h_atg.data_ptr()),
                                                ctypes.c_void_p(h_x0.data_ptr() if fbp else None),
                                                ctypes.c_void_p(ws), nb, ctypes.byref(gtg)))
        return h_atg, gtg.value, h_x0

    def stream_reconstruct(self, h_x, atg, gtg_half: float, params: Params):
        """tmbir_reconstruct on a host volume: h_x (x_0 in, the final iterate out) is a contiguous
        float32 CPU tensor of n_slices N^2 values; atg (R*g) the same on the CPU, or a CUDA tensor
        (read in place: only the iterates stream)."""
        import torch

        g = self.groups[0]
        if h_x.is_cuda or not h_x.is_contiguous() or h_x.dtype != torch.float32:
            raise TypeError("expected a contiguous float32 CPU tensor for the image")
        if not atg.is_contiguous() or atg.dtype != torch.float32:
            raise TypeError("expected a contiguous float32 tensor for R*g")
        h_atg = atg
        if h_x.numel() != h_atg.numel() or h_x.numel() % (g.N * g.N):
            raise ValueError("image sizes do not match")
        n_slices = h_x.numel() // (g.N * g.N)
        if getattr(self, "_hwork", None) is None or self._hwork.numel() != 2 * h_x.numel():
            self._hwork = torch.empty(2 * h_x.numel(), dtype=torch.float32, pin_memory=True)
        ws, nb = self._stream_work(n_slices)
        st = _Stats()
        pr = params.c_struct()
        self._pre()
        _check(_lib.tmbir_stream_reconstruct(self._h, int(n_slices), ctypes.c_void_p(h_x.data_ptr()),
                                             ctypes.c_void_p(h_atg.data_ptr()), float(gtg_half),
                                             ctypes.c_void_p(self._hwork.data_ptr()), ctypes.c_void_p(ws), nb,
                                             ctypes.byref(pr), ctypes.byref(st)))
        return Stats(st.iterations, st.restarts, st.status, st.objective, st.gap, st.L, st.grad_norm)

    def get_log(self, max_entries: int = 1 << 16):
        buf = (ctypes.c_double * (4 * max_entries))()
        n = ctypes.c_int()
        _check(_lib.tmbir_get_log(self._h, buf, max_entries, ctypes.byref(n)))
        return [tuple(buf[4 * k: 4 * k + 4]) for k in range(n.value)]

    def normal_apply(self, x, out=None):
        out = self._empty(x.numel()) if out is None else out
        self._pre()
        _check(_lib.tmbir_normal_apply(self._h, ctypes.c_void_p(_ptr(x)), ctypes.c_void_p(_ptr(out))))
        self._post(x, out)
        return out

    def normal_apply_static(self, x, out=None):
        """normal_apply with its scratch in the library's fixed device array (no allocation
        by the library; `out` is allocated here when not given)."""
        out = self._empty(x.numel()) if out is None else out
        self._pre()
        _check(_lib.tmbir_normal_apply_static(self._h, ctypes.c_void_p(_ptr(x)), ctypes.c_void_p(_ptr(out))))
        self._post(x, out)
        return out

    def forward(self, x, out=None):
        """R x by the type-2 NUFFT (FP32): [slice][angle][bin]."""
        out = self._empty(self.sino_numel()) if out is None else out
        self._pre()
        _check(_lib.tmbir_forward(self._h, ctypes.c_void_p(_ptr(x)), ctypes.c_void_p(_ptr(out))))
        self._post(x, out)
        return out

    def adjoint(self, sino, out=None):
        """R* g by the type-1 NUFFT (FP32)."""
        out = self._empty(self.image_numel()) if out is None else out
        self._pre()
        _check(_lib.tmbir_adjoint(self._h, ctypes.c_void_p(_ptr(sino)), ctypes.c_void_p(_ptr(out))))
        self._post(sino, out)
        return out

    def gradient_direct(self, x, sino, params: Params, out=None, want_objective: bool = False):
        """R*(R x - g) + lambda grad Phi(x) through the two NUFFTs (no Toeplitz structure); with
        want_objective also F(x) = 1/2 ||R x - g||^2 + lambda Phi(x)."""
        out = self._empty(x.numel()) if out is None else out
        pr = params.c_struct()
        F = ctypes.c_double()
        self._pre()
        _check(_lib.tmbir_gradient_direct(self._h, ctypes.c_void_p(_ptr(x)), ctypes.c_void_p(_ptr(sino)),
                                          ctypes.byref(pr), ctypes.c_void_p(_ptr(out)),
                                          ctypes.byref(F) if want_objective else None))
        self._post(x, sino, out)
        return (out, F.value) if want_objective else out

    def sfu_rate(self, iters: int = 4096) -> float:
        """Measured special-function operations per second (log2, exp2, reciprocal chains)."""
        out = ctypes.c_double()
        self._pre()
        _check(_lib.tmbir_sfu_rate(self._h, int(iters), ctypes.byref(out)))
        return out.value

    def wait_check(self, polls: int, arrive: bool):
        """Run the library's bounded device wait on its own: returns when the wait completes
        (arrive), raises TmbirError(TMBIR_ERR_TIMEOUT) when it gives up (nothing arrives)."""
        self._pre()
        _check(_lib.tmbir_wait_check(self._h, int(polls), 1 if arrive else 0))

    def gradient(self, x, atg, params: Params, out=None):
        out = self._empty(x.numel()) if out is None else out
        pr = params.c_struct()
        self._pre()
        _check(_lib.tmbir_gradient(self._h, ctypes.c_void_p(_ptr(x)), ctypes.c_void_p(_ptr(atg)), ctypes.byref(pr),
                                   ctypes.c_void_p(_ptr(out))))
        self._post(x, atg, out)
        return out

    def step(self, x, x_prev, beta, atg, params: Params, L, out=None):
        out = self._empty(x.numel()) if out is None else out
        pr = params.c_struct()
        parts = (ctypes.c_double * 5)()
        self._pre()
        _check(_lib.tmbir_step(self._h, ctypes.c_void_p(_ptr(x)), ctypes.c_void_p(_ptr(x_prev)), float(beta),
                               ctypes.c_void_p(_ptr(atg)), ctypes.byref(pr), float(L), ctypes.c_void_p(_ptr(out)),
                               parts))
        self._post(x, x_prev, atg, out)
        return out, list(parts)

    def objective(self, x, atg, params: Params) -> float:
        pr = params.c_struct()
        F = ctypes.c_double()
        self._pre()
        _check(_lib.tmbir_objective(self._h, ctypes.c_void_p(_ptr(x)), ctypes.c_void_p(_ptr(atg)), ctypes.byref(pr),
                                    ctypes.byref(F)))
        self._post(x, atg)
        return F.value

    def lambda_max(self):
        out = (ctypes.c_double * len(self.groups))()
        _check(_lib.tmbir_lambda_max(self._h, out))
        return list(out)

    def kernel(self, group: int = 0):
        import torch

        N = self.groups[group].N
        with torch.cuda.stream(self.stream):
            K = torch.empty((2 * N - 1) * (2 * N - 1), dtype=torch.float64, device=self.device)
        self._pre()
        _check(_lib.tmbir_kernel(self._h, group, ctypes.c_void_p(_ptr(K))))
        self._post(K)
        return K

    def upsample_lanczos3(self, coarse, n_slices: int, Nc: int, out=None):
        out = self._empty(n_slices * 4 * Nc * Nc) if out is None else out
        self._pre()
        _check(_lib.tmbir_upsample_lanczos3(self._h, ctypes.c_void_p(_ptr(coarse)), n_slices, Nc,
                                            ctypes.c_void_p(_ptr(out))))
        self._post(coarse, out)
        return out

    def downsample_sino(self, sino, n_slices: int, n_angles: int, n_det: int, factor: int, out=None):
        out = self._empty(n_slices * n_angles * (n_det // factor)) if out is None else out
        self._pre()
        _check(_lib.tmbir_downsample_sino(self._h, ctypes.c_void_p(_ptr(sino)), n_slices, n_angles, n_det, factor,
                                          ctypes.c_void_p(_ptr(out))))
        self._post(sino, out)
        return out

    def autotune(self, x, atg, params: Params):
        """Pick, by timing, the pass-3b slices per block and the slices per spectrum chunk of every
        group; returns the pass-3b choices (the chunk choices land in self.spec_chunks)."""
        zc = (ctypes.c_int * len(self.groups))()
        sc = (ctypes.c_int * len(self.groups))()
        pr = params.c_struct()
        self._pre()
        _check(_lib.tmbir_autotune(self._h, ctypes.c_void_p(_ptr(x)), ctypes.c_void_p(_ptr(atg)), ctypes.byref(pr), zc,
                                   sc))
        self._post(x, atg)
        self.spec_chunks = list(sc)
        return list(zc)

    def state_export(self, out=None):
        """Checkpoint of the last run (device uint8 tensor); x_k is the run's image."""
        import torch

        n = ctypes.c_size_t()
        _check(_lib.tmbir_state_size(self._h, ctypes.byref(n)))
        if out is None:
            with torch.cuda.stream(self.stream):
                out = torch.empty(n.value, dtype=torch.uint8, device=self.device)
        self._pre()
        _check(_lib.tmbir_state_export(self._h, ctypes.c_void_p(out.data_ptr())))
        self._post(out)
        return out

    def state_import(self, state):
        self._pre()
        _check(_lib.tmbir_state_import(self._h, ctypes.c_void_p(state.data_ptr())))
        self._post(state)

    def pass_times(self, x, atg, params: Params, iters: int):
        """Summed device ms of (pass 1, pass 2, pass 3a, pass 3b, finalize) over `iters` eager iterations."""
        pr = params.c_struct()
        out = (ctypes.c_double * 5)()
        self._pre()
        _check(_lib.tmbir_pass_times(self._h, ctypes.c_void_p(_ptr(x)), ctypes.c_void_p(_ptr(atg)), ctypes.byref(pr),
                                     iters, out))
        self._post(x, atg)
        return list(out)

    def launch_count(self) -> int:
        n = ctypes.c_longlong()
        _check(_lib.tmbir_launch_count(self._h, ctypes.byref(n)))
        return n.value

    def sync(self):
        _check(_lib.tmbir_sync(self._h))

    def close(self):
        if getattr(self, "_h", None):
            _lib.tmbir_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def reconstruct_levels(N: int, angles, n_slices: int, sino, levels: int, params, span: float = math.pi,
                       stream=None, device="cuda", start=None, ctxs=None, overlap_setup: bool = False,
                       coarse_setup_fp32: bool = False):
    """Hierarchical reconstruction (Sec. 2.3) through the C ABI.

    Level l = 0 .. levels-1 reconstructs n_slices slices of N / 2^(levels-1-l) pixels.  A
    level's sinogram keeps every angle and every f-th detector bin about the centre bin,
    divided by f (tmbir_downsample_sino, f = 2^(levels-1-l)); the coarsest level starts from
    its FBP image (or from `start`, a callable (ctx, sino_l, atg_l) -> image), every finer
    level from the Lanczos-3 x2 upsampling of the level below (tmbir_upsample_lanczos3).
    `params` is one Params per level.  `ctxs` (the list a previous call returned) reuses the
    level contexts and their workspaces.  With overlap_setup, every level's setup (its
    subsampled sinogram, kernel spectrum and R*g, which depend on the data only) is enqueued
    first on that level's own context stream, so the setups of the finer levels run while the
    coarser levels iterate; the contexts must then have distinct streams (created here when
    `ctxs` is None).  Without it all levels share one stream and run one after another.  With
    coarse_setup_fp32 the levels below the finest build their R*g in FP32
    (tmbir_build_operator_fp32); the finest level's is FP64 either way.
    Returns the finest image, the level contexts and the per-level Stats.
    """
    import torch

    if len(params) != levels:
        raise ValueError("one Params per level")
    if N % (1 << (levels - 1)):
        raise ValueError("N must be divisible by 2^(levels-1)")
    if ctxs is None:
        dev = torch.device(device)
        shared = stream if stream is not None else torch.cuda.Stream(device=dev)
        ctxs = [Context([Group(N=N >> (levels - 1 - lev), angles=list(angles), n_slices=n_slices, span=span)],
                        stream=torch.cuda.Stream(device=dev) if overlap_setup else shared, device=device)
                for lev in range(levels)]
    if overlap_setup and len({c.stream.cuda_stream for c in ctxs}) != levels:
        raise ValueError("overlap_setup needs one stream per level context")
    na = len(angles)
    caller = torch.cuda.current_stream(ctxs[0].device)

    def setup(lev):
        f = 1 << (levels - 1 - lev)
        Nl = N // f
        ctx = ctxs[lev]
        # per-level buffers live on the context, so repeated calls reuse them (and the
        # context's cached iteration graph, which is keyed on the buffers)
        if getattr(ctx, "_lv", None) is None:
            ctx._lv = {"x": ctx._empty(n_slices * Nl * Nl), "atg": ctx._empty(n_slices * Nl * Nl),
                       "sino": ctx._empty(n_slices * na * Nl) if f > 1 else None}
        lv = ctx._lv
        lv["sino_l"] = sino if f == 1 else ctx.downsample_sino(sino, n_slices, na, N, f, out=lv["sino"])
        ctx.build_operator(lv["sino_l"], lv["atg"], fp64=not (coarse_setup_fp32 and lev < levels - 1))

    if overlap_setup:
        for lev in range(levels):
            ctxs[lev].stream.wait_stream(caller)  # the sinogram is ready on the caller's stream
            with torch.cuda.stream(ctxs[lev].stream):
                setup(lev)
    stats = []
    x = None
    for lev in range(levels):
        ctx = ctxs[lev]
        with torch.cuda.stream(ctx.stream if overlap_setup else caller):
            if not overlap_setup:
                setup(lev)
            lv = ctx._lv
            if x is None:
                if start is not None:
                    lv["x"].copy_(start(ctx, lv["sino_l"], lv["atg"]))
                else:
                    ctx.fbp(lv["sino_l"], lv["x"])
            else:
                if overlap_setup:
                    ctx.stream.wait_stream(ctxs[lev - 1].stream)  # the coarser level's result
                ctx.upsample_lanczos3(x, n_slices, (N >> (levels - 1 - lev)) // 2, out=lv["x"])
            x = lv["x"]
            stats.append(ctx.reconstruct(x, lv["atg"], params[lev]))
    if overlap_setup:
        caller.wait_stream(ctxs[-1].stream)
    return x, ctxs, stats


class CNN:
    """The learned warm-start refiner (see tmbir_cnn_* in include/tmbir.h)."""

    def __init__(self, H: int, W: int, max_batch: int = 4, stream=None, device="cuda", seed: int = 1):
        import torch

        load()
        self.device = torch.device(device)
        self.stream = stream if stream is not None else torch.cuda.Stream(device=self.device)
        self.H, self.W, self.max_batch = H, W, max_batch
        nbytes = ctypes.c_size_t()
        _check(_lib.tmbir_cnn_workspace_size(max_batch, H, W, ctypes.byref(nbytes)))
        with torch.cuda.stream(self.stream):
            self.workspace = torch.empty(nbytes.value + 256, dtype=torch.uint8, device=self.device)
        aligned = (self.workspace.data_ptr() + 255) // 256 * 256
        h = ctypes.c_void_p()
        _check(_lib.tmbir_cnn_create(ctypes.byref(h), ctypes.c_void_p(self.stream.cuda_stream), max_batch, H, W,
                                     ctypes.c_void_p(aligned), nbytes.value))
        self._h = h
        self.n_params = _lib.tmbir_cnn_param_count()
        _check(_lib.tmbir_cnn_init(self._h, seed))

    _pre = Context._pre
    _post = Context._post

    def _empty(self, n):
        import torch

        with torch.cuda.stream(self.stream):
            return torch.empty(n, dtype=torch.float32, device=self.device)

    def set_weights(self, params):
        import numpy as np

        a = np.ascontiguousarray(params, dtype=np.float32)
        if a.size != self.n_params:
            raise ValueError(f"expected {self.n_params} parameters, got {a.size}")
        _check(_lib.tmbir_cnn_set_weights(self._h, a.ctypes.data_as(ctypes.POINTER(ctypes.c_float))))

    def get_weights(self):
        import numpy as np

        a = np.zeros(self.n_params, dtype=np.float32)
        _check(_lib.tmbir_cnn_get_weights(self._h, a.ctypes.data_as(ctypes.POINTER(ctypes.c_float))))
        return a

    def apply(self, x, batch: int, out=None):
        out = self._empty(x.numel()) if out is None else out
        self._pre()
        _check(_lib.tmbir_cnn_apply(self._h, ctypes.c_void_p(_ptr(x)), batch, ctypes.c_void_p(_ptr(out))))
        self._post(x, out)
        return out

    def train_step(self, x, target, batch: int, lr: float = 1e-3) -> float:
        loss = ctypes.c_double()
        self._pre()
        _check(_lib.tmbir_cnn_train_step(self._h, ctypes.c_void_p(_ptr(x)), ctypes.c_void_p(_ptr(target)), batch,
                                         float(lr), ctypes.byref(loss)))
        self._post(x, target)
        return loss.value

    def net_forward(self, x, batch: int):
        out = self._empty(x.numel())
        self._pre()
        _check(_lib.tmbir_cnn_net_forward(self._h, ctypes.c_void_p(_ptr(x)), batch, ctypes.c_void_p(_ptr(out))))
        self._post(x, out)
        return out

    def net_backward(self, x, gout, batch: int):
        import numpy as np

        gp = np.zeros(self.n_params, dtype=np.float32)
        gin = self._empty(x.numel())
        self._pre()
        _check(_lib.tmbir_cnn_net_backward(self._h, ctypes.c_void_p(_ptr(x)), ctypes.c_void_p(_ptr(gout)), batch,
                                           gp.ctypes.data_as(ctypes.POINTER(ctypes.c_float)),
                                           ctypes.c_void_p(_ptr(gin))))
        self._post(x, gout, gin)
        return gp, gin

    def warm_start(self, ctx: Context, fbp, atg, params: Params, out=None):
        """(x0, used_cnn): the refined start if its objective beats the FBP start's, else FBP."""
        out = ctx._empty(fbp.numel()) if out is None else out
        used = ctypes.c_int()
        pr = params.c_struct()
        ctx._pre()  # the library orders the network's stream after the context's
        _check(_lib.tmbir_warm_start(ctx._h, self._h, ctypes.c_void_p(_ptr(fbp)), ctypes.c_void_p(_ptr(atg)),
                                     ctypes.byref(pr), ctypes.c_void_p(_ptr(out)), ctypes.byref(used)))
        ctx._post(fbp, atg, out)
        self._post(fbp, out)
        return out, bool(used.value)

    def close(self):
        if getattr(self, "_h", None):
            _lib.tmbir_cnn_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
