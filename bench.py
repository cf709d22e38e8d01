"""Benchmark: gradient voxel-updates/s and time to a 1e-3 relative objective gap of the
Toeplitz MBIR path on GB300, through the C ABI.

Default workload (the largest single-GPU configuration): 512 slices of 2048^2, 128 angles
over [0, 2 pi/3) (missing wedge), 20 ellipsoids, Gaussian noise of 1 %.  One step is the
chosen form of the method, from the resident sinogram to the 1e-3 gap:
  levels 512^2 -> 1024^2 -> 2048^2 (Sec. 2.3): subsampled sinograms, setup per level
  (kernel spectrum, R*g, 1/2 g.g; Sec. 2.1), FBP start at the coarsest level (Sec. 2.2)
  refined by the learned network where that lowers the objective, Lanczos-3 x2 between
  levels, BF16 spectra with FP32 refinement, iterations in device-driven graph loops that
  stop at the gap.
value = the voxel-updates of all levels (slices x N_l^2 x iterations_l) / step time, summed
over ranks (each rank reconstructs its own independent batch: weak scaling, no collective on
the data path).  The iteration phase is also timed on its own, pass by pass, for the roofline.

`--workload batched-64x1024sq-256ang-100it` is the earlier fixed-work step: setup plus 100
iterations of one level.  `--impl reference` times the FP64 CPU oracle on the host cores on
a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

# kind "hier": one step = the chosen form to the gap; kind "fixed": setup + `iters` iterations
WORKLOADS = {
    "hier-512x2048sq-128ang-limited": dict(S=512, N=2048, na=128, span=2 * math.pi / 3, ne=20, kind="hier"),
    "batched-64x1024sq-256ang-100it": dict(S=64, N=1024, na=256, span=math.pi, ne=20, kind="fixed", iters=100),
    # the chosen form at the batched workload's size
    "hier-64x1024sq-256ang": dict(S=64, N=1024, na=256, span=math.pi, ne=20, kind="hier"),
    "single-1x128sq-90ang-50it": dict(S=1, N=128, na=90, span=math.pi, ne=10, kind="fixed", iters=50),
    # uneven batch: 16 groups of 16 slices, one per (N, angles) in {512, 1024, 1536, 2048} x
    # {64, 128, 180, 360}, in one context; FP32, one level, FBP start, to the 1e-3 gap
    "uneven-16x16sl-4sides-4angles": dict(S=256, N=2048, na=360, span=math.pi, ne=20, kind="uneven"),
    # learned warm start: trained on (FBP, converged) pairs at 1024^2 with 90..180 angles, evaluated
    # on 128 slices of 2560^2 with 150 angles (the CNN start against the FBP start, to the 1e-3 gap)
    "learned-128x2560sq-150ang": dict(S=128, N=2560, na=150, span=math.pi, ne=20, kind="learned"),
    # a host-resident volume streamed through the GPU in slabs (Sec. 2.4), the paper's nano-CT
    # shape (212 angles over [0, pi), 2448-bin detector rows on the 2560 grid) with 256 of its
    # 2048 slices: setup + `iters` FP32 iterations from and to host memory, against the same
    # iterations on the resident volume
    "streamed-256x2560sq-212ang": dict(S=256, N=2560, na=212, span=math.pi, ne=20, kind="streamed", iters=10,
                                       slab=16),
    # profiling cases: the image sides and angles of the workloads, a few GB on the device
    "profile-16x1024sq-256ang-20it": dict(S=16, N=1024, na=256, span=math.pi, ne=20, kind="fixed", iters=20),
    "profile-8x2048sq-128ang-limited-20it": dict(S=8, N=2048, na=128, span=2 * math.pi / 3, ne=20, kind="fixed",
                                                 iters=20),
}
DEFAULT = "hier-512x2048sq-128ang-limited"
UNEVEN_SIDES = (512, 1024, 1536, 2048)
UNEVEN_ANGLES = (64, 128, 180, 360)
UNEVEN_SLICES = 16
LEARN_TRAIN_N = 1024
LEARN_TRAIN_VOLUMES = 20  # volumes of LEARN_TRAIN_SLICES slices, each with its own angle count
LEARN_TRAIN_SLICES = 100
LEARN_TARGET_GAP = 1e-4  # training targets: the method run to this gap of each volume
LEARN_EPOCHS = 4
PRIOR = dict(p=1.2, q=2.0, c=0.01, sigma=0.1, lam=1.0)
METRIC = "gradient voxel-updates/s"

GAP = 1e-3
LEVELS = 3
COARSE_ITERS = (40, 15)  # iterations at N/4 and N/2 before the finest level (default, before tuning)
# candidates for the coarse iteration counts, chosen by the chosen form's measured time to the gap
COARSE_CANDIDATES = [(40, 15), (40, 30), (60, 30), (40, 50), (80, 60)]
FINEST_CAP = 400  # iteration cap of the finest level (the gap stops it first)
REF_ITERS = 600  # finest-level FP32 iterations after the hierarchy that give F_ref
PLAIN_CAP = 800  # iteration cap of the one-level forms
REFINE_GAP = 1e-2  # BF16 spectra until this gap, FP32 after
CNN_EPOCHS = 12
CNN_BATCH = 8
CNN_TARGET_ITERS = 300  # iterations that make a training target from an FBP start
CNN_TRAIN_SLICES = 128  # slices of the separate training volume
PASS_ITERS = 5  # eager iterations timed pass by pass


_t_start = time.perf_counter()


def progress(msg):
    """A timestamped progress line on stderr (the JSON line alone goes to stdout)."""
    print(f"[bench {time.perf_counter() - _t_start:7.1f}s] {msg}", file=sys.stderr, flush=True)


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def rank_seed(rank, base=1002):
    """Phantom seed of a rank: every rank reconstructs its own independent batch (weak scaling,
    no collective on the data path)."""
    return base + 17 * rank


def max_over_ranks(ms, world, device):
    """The slowest rank's time: each rank passes its own and every rank gets the maximum."""
    if world <= 1:
        return ms
    import torch

    t = torch.tensor([ms], dtype=torch.float64, device=device)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def job_rate(units_per_rank, steps, world, ms):
    """Whole-job throughput: the units all ranks processed over the slowest rank's time."""
    return world * units_per_rank * steps / (ms * 1e-3)


def make_problem(name, rank):
    import synth

    w = WORKLOADS[name]
    if w["kind"] == "uneven":
        return [synth.volume(S=UNEVEN_SLICES, N=N, n_angles=na, n_ellipsoids=w["ne"], span=w["span"],
                             seed=rank_seed(rank, 3000 + N + na)) for N in UNEVEN_SIDES for na in UNEVEN_ANGLES]
    base = 1003 if w["span"] < math.pi else 1002
    return synth.volume(S=w["S"], N=w["N"], n_angles=w["na"], n_ellipsoids=w["ne"], span=w["span"],
                        seed=rank_seed(rank, base))


class Clocks:
    """nvidia-smi samples of SM clock and throttle reasons while the timed region runs."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(gpu_index), f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.f,
                                      stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None

    def stop(self):
        if self.p is None:
            return None
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.p.kill()
        self.f.flush()
        rows = []
        with open(self.f.name) as fh:
            for line in fh:
                parts = [v.strip() for v in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.f.name)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        smax = max(float(r[2]) for r in rows if r[2].replace(".", "").isdigit())
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if "Active" in r[5 + k] and "Not" not in r[5 + k]})
        load = [v for v in sm if v > 0.5 * smax] or sm
        return {"sm_mhz": statistics.median(load), "sm_max_mhz": smax, "reasons": reasons, "samples": len(rows)}


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def kernel_traffic(kernel, workload):
    """DRAM bytes per launch from the committed ncu summary, if it matches the current kernel source."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as f:
            d = json.load(f)
        src = os.path.join(ROOT, "paper_2603_28756_gb300", "csrc", "toeplitz_kernels.cuh")
        h = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]
        e = d.get(workload, {}).get(kernel)
        if e and e.get("source_sha") == h:
            return e["dram_bytes_per_launch"]
    except Exception:
        pass
    return None


# ------------------------------------------------------------------------------ CPU baseline

_oracle_kernels = {}  # workload -> (K, its spectrum, seconds to build them)


def oracle_sample(name, slices, iters):
    """Seconds the FP64 oracle takes for `iters` fast-gradient iterations of `slices` slices at the
    workload's image side and angles (K (*) y by FFT convolution, the qGGMRF prior, the update;
    seeded images of that size).  The kernel K and its spectrum are built once per workload and
    not timed."""
    import numpy as np

    import oracle
    import synth

    w = WORKLOADS[name]
    N = w["N"]
    rng = np.random.default_rng(5)
    x0 = rng.uniform(0, 0.5, (slices, N, N))
    atg = rng.uniform(0, 1.0, (slices, N, N))
    pr = oracle.Prior(**PRIOR)
    if name not in _oracle_kernels:
        t0 = time.perf_counter()
        K = oracle.kernel(N, synth.angles(w["na"], w["span"]), N)
        _oracle_kernels[name] = (K, oracle.circulant_spectrum(K), time.perf_counter() - t0)
    K, Chat, t_setup = _oracle_kernels[name]
    L = 1.01 * 50.0 + pr.lam * 4.0 / pr.sigma ** 2
    t0 = time.perf_counter()
    oracle.nesterov(x0, atg, 1.0, K, pr, L, iters, Chat=Chat)
    return time.perf_counter() - t0, t_setup


def cpu_baseline(name, slices=1, iters=2, single_thread=True):
    """FP64 oracle on the host cores on a bounded sample of the workload's iteration phase:
    all cores, and (in a child process with one OpenMP thread) a single core."""
    w = WORKLOADS[name]
    N = w["N"]
    dt, t_setup = oracle_sample(name, slices, iters)
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    out = {
        "value": slices * N * N * iters / dt,
        "unit": "voxel-updates/s",
        "cores": cores,
        "kind": "oracle",
        "sample": f"{slices} of {w['S']} slices x {iters} iterations at {N}^2, {w['na']} angles; iteration phase "
                  f"only (kernel K and spectrum {t_setup:.1f} s excluded); numpy FFT single-threaded, prior in C with "
                  f"OpenMP",
    }
    if single_thread:
        # a child process whose OpenMP runtime starts with one thread; it takes the kernel K
        # from a file instead of building it again on one core
        import numpy as np

        env = dict(os.environ, OMP_NUM_THREADS="1")
        with tempfile.TemporaryDirectory() as td:
            kf = os.path.join(td, "K.npy")
            np.save(kf, _oracle_kernels[name][0])
            code = (f"import sys; sys.path.insert(0, {ROOT!r}); import numpy as np, oracle, bench; "
                    f"K = np.load({kf!r}); bench._oracle_kernels[{name!r}] = (K, oracle.circulant_spectrum(K), 0.0); "
                    f"print(bench.oracle_sample({name!r}, {slices}, {iters})[0])")
            try:
                r = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=600)
                out["single_thread"] = {"value": slices * N * N * iters / float(r.stdout.strip().splitlines()[-1]),
                                        "cores": 1}
            except Exception as e:  # reported, not hidden
                out["single_thread"] = {"error": str(e)[:200]}
    return out


# ------------------------------------------------------------------------------ learned start

def train_warm_start(tm, w, factor, stream):
    """The learned warm start for images of N / factor: trained on (FBP, reconstruction) pairs
    the method itself produces from a separate seeded volume (same geometry, other phantoms)."""
    import torch

    import synth

    S, N, na, span = min(w["S"], CNN_TRAIN_SLICES), w["N"], w["na"], w["span"]
    p = synth.volume(S=S, N=N, n_angles=na, n_ellipsoids=w["ne"], span=span, seed=7001)
    Nl = N // factor
    ctx = tm.Context([tm.Group(N=Nl, angles=list(p.theta), n_slices=S, span=span)], stream=stream)
    sino = torch.from_numpy(p.sino.ravel()).cuda()
    if factor > 1:
        sino = ctx.downsample_sino(sino, S, na, N, factor)
    atg = ctx.build_operator(sino)
    fbp = ctx.fbp(sino)
    target = fbp.clone()
    ctx.reconstruct(target, atg, tm.Params(**PRIOR, max_iter=CNN_TARGET_ITERS))
    net = tm.CNN(Nl, Nl, max_batch=CNN_BATCH, stream=stream, seed=11)
    plane = Nl * Nl
    losses = []
    t0 = time.perf_counter()
    for _ in range(CNN_EPOCHS):
        for b in range(0, S - CNN_BATCH + 1, CNN_BATCH):
            losses.append(net.train_step(fbp[b * plane:(b + CNN_BATCH) * plane],
                                         target[b * plane:(b + CNN_BATCH) * plane], CNN_BATCH, lr=1e-3))
    steps = max(1, S // CNN_BATCH)
    info = {"image": Nl, "pairs": S, "epochs": CNN_EPOCHS, "train_s": time.perf_counter() - t0,
            "loss_first_epoch": sum(losses[:steps]) / steps, "loss_last_epoch": sum(losses[-steps:]) / steps}
    del ctx
    return net, info


# ------------------------------------------------------------------------------ the chosen form

class Hier:
    """Level contexts (N/4, N/2, N), each on its own stream so that the setups of the finer levels
    run while the coarser levels iterate, and the per-level buffers of the chosen form."""

    def __init__(self, tm, w, theta):
        import torch

        self.tm, self.w, self.theta = tm, w, list(theta)
        S, N, span = w["S"], w["N"], w["span"]
        self.ctxs = [tm.Context([tm.Group(N=N >> (LEVELS - 1 - k), angles=self.theta, n_slices=S, span=span)],
                                stream=torch.cuda.Stream()) for k in range(LEVELS)]
        self.net = None

    def run(self, sino, prms, start_cnn=True, coarse_fp32=False):
        """The hierarchy through the C ABI: per level, stats of the level's reconstruct
        (coarse_fp32: the coarse levels build R*g in FP32)."""
        tm = self.tm

        def start(c, s_l, a_l):
            f0 = c.fbp(s_l)
            if not start_cnn or self.net is None:
                return f0
            x0, used = self.net.warm_start(c, f0, a_l, tm.Params(**PRIOR))
            self.used_cnn = used
            return x0

        self.used_cnn = False
        y, _, stats = tm.reconstruct_levels(self.w["N"], self.theta, self.w["S"], sino, LEVELS, prms,
                                            span=self.w["span"], ctxs=self.ctxs, start=start, overlap_setup=True,
                                            coarse_setup_fp32=coarse_fp32)
        self.x = y
        return stats

    def voxel_updates(self, stats):
        S, N = self.w["S"], self.w["N"]
        return sum(S * (N >> (LEVELS - 1 - k)) ** 2 * st.iterations for k, st in enumerate(stats))


def tune_coarse(H, sino, F_ref, stream, barrier, world):
    """The coarse-level iteration counts of the hierarchy (a cap per level, chosen by time to the
    gap; the paper's per-level counts were in a figure that is lost): each candidate runs the
    chosen form once to warm up and once timed; the fastest that reaches the gap is kept."""
    trials = {}
    for cand in COARSE_CANDIDATES:
        prms = chosen_params(F_ref, cand)
        H.run(sino, prms, coarse_fp32=True)
        ms, stats = timed(stream, barrier, world, lambda: H.run(sino, prms, coarse_fp32=True))
        trials[str(list(cand))] = {"ms": ms, "level_iterations": [st.iterations for st in stats],
                                   "reached": stats[-1].gap <= GAP}
    ok = [c for c in COARSE_CANDIDATES if trials[str(list(c))]["reached"]] or COARSE_CANDIDATES
    best = min(ok, key=lambda c: trials[str(list(c))]["ms"])
    return best, trials


def chosen_params(F_ref, coarse=None):
    prms = [tm_params(max_iter=k, bf16=True) for k in (coarse or COARSE_ITERS)]
    prms.append(tm_params(max_iter=FINEST_CAP, gap_tol=GAP, F_ref=F_ref, bf16=True, refine_gap=REFINE_GAP))
    return prms


def fp32_params(F_ref, finest_iters=FINEST_CAP, gap_tol=GAP, coarse=None):
    prms = [tm_params(max_iter=k) for k in (coarse or COARSE_ITERS)]
    prms.append(tm_params(max_iter=finest_iters, gap_tol=gap_tol, F_ref=F_ref))
    return prms


_tm = None


def tm_params(**kw):
    return _tm.Params(**PRIOR, **kw)


# ------------------------------------------------------------------------------ time to gap

def timed(stream, barrier, world, fn):
    """(device ms from the resident inputs to the end of fn, fn's result), max over ranks."""
    import torch

    barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    res = fn()
    e1.record(stream)
    barrier()
    return max_over_ranks(e0.elapsed_time(e1), world, "cuda"), res


def time_to_gap_hier(tm, H, sino, F_ref, F0, stream, barrier, world, step_ms, step_stats, coarse):
    """Every form from the resident sinogram until the device stops the finest level at gap <= 1e-3."""
    w = H.w
    S, N, span = w["S"], w["N"], w["span"]
    ctx = H.ctxs[-1]
    x, atg = ctx._lv["x"], ctx._lv["atg"]
    stop = dict(max_iter=PLAIN_CAP, gap_tol=GAP, F_ref=F_ref)
    forms = {}

    def one_level(use_graph, bf16):
        def run():
            if use_graph:
                ctx.build_operator_fbp(sino, atg, x)
            else:  # the plain form: one call after the other, eager launches
                ctx.build_operator(sino, atg)
                ctx.fbp(sino, x)
            return [ctx.reconstruct(x, atg, tm_params(**stop, use_graph=use_graph, bf16=bf16,
                                                      refine_gap=REFINE_GAP if bf16 else 0.0))]
        return run

    def hier(bf16, cnn):
        def run():
            prms = chosen_params(F_ref, coarse) if bf16 else fp32_params(F_ref, coarse=coarse)
            return H.run(sino, prms, start_cnn=cnn)
        return run

    runs = {
        "plain": (one_level(False, False), "FP32 spectra, FBP start, one level, eager launches", 1),
        "batched_graph": (one_level(True, False), "FP32 spectra, FBP start, one level, device-driven graph loop", 1),
        "bf16_refine": (one_level(True, True), f"BF16 spectra to gap {REFINE_GAP:g} then FP32, FBP start, one level, "
                                               "graph", 1),
        "hierarchical": (hier(False, False), f"levels N/4, N/2, N ({coarse[0]} and {coarse[1]} coarse iterations), "
                                             "FBP at N/4, Lanczos-3 between levels, FP32, graph", 1),
        "hierarchical_bf16": (hier(True, False), "as hierarchical, BF16 spectra (FP32 refinement at the finest level "
                                                 f"from gap {REFINE_GAP:g})", 1),
    }
    for name, (run, desc, reps) in runs.items():
        for _ in range(reps):
            ms, stats = timed(stream, barrier, world, run)
        progress(f"time to gap {name}: {ms:.1f} ms, {[st.iterations for st in stats]} iterations, gap {stats[-1].gap:.3g}")
        forms[name] = {"ms": ms, "finest_iterations": stats[-1].iterations, "gap_reached": stats[-1].gap,
                       "reached": stats[-1].gap <= GAP, "form": desc}
        if len(stats) > 1:
            forms[name]["level_iterations"] = [s.iterations for s in stats]
    forms["chosen"] = {"ms": step_ms, "finest_iterations": step_stats[-1].iterations,
                       "level_iterations": [s.iterations for s in step_stats], "gap_reached": step_stats[-1].gap,
                       "reached": step_stats[-1].gap <= GAP, "used_cnn": H.used_cnn,
                       "form": "the bench step: levels N/4, N/2, N (R*g in FP32 at the coarse levels, FP64 at N), "
                               "CNN-refined FBP start at N/4 (FBP fallback), "
                               f"BF16 spectra with FP32 refinement from gap {REFINE_GAP:g}, device-driven graph loops"}
    forms["single_slice"] = single_slice_form(tm, w, H.theta, sino, stream, barrier, world)
    return forms


def single_slice_form(tm, w, theta, sino, stream, barrier, world, sample=2):
    """The plain single-slice form (each slice alone: one-slice geometry, in-plane prior, its own
    F_ref, FBP start, one level, eager launches) on `sample` slices, scaled to the whole batch."""
    S, N, span, na = w["S"], w["N"], w["span"], w["na"]
    c1 = tm.Context([tm.Group(N=N, angles=list(theta), n_slices=1, span=span)], stream=stream)
    plane = N * N
    picks = list(range(0, S, max(1, S // sample)))[:sample]
    sl = [sino[z * na * N:(z + 1) * na * N] for z in picks]
    a1, x1 = c1._empty(plane), c1._empty(plane)
    refs = []
    for s in sl:
        c1.build_operator(s, a1)
        c1.fbp(s, x1)
        refs.append(c1.reconstruct(x1, a1, tm_params(max_iter=REF_ITERS)).objective)

    def run():
        sts = []
        for s, F in zip(sl, refs):
            c1.build_operator(s, a1)
            c1.fbp(s, x1)
            sts.append(c1.reconstruct(x1, a1, tm_params(max_iter=PLAIN_CAP, gap_tol=GAP, F_ref=F, use_graph=False)))
        return sts

    ms, sts = timed(stream, barrier, world, run)
    return {"ms": ms * S / len(sl), "extrapolated_from_slices": len(sl), "sample_ms": ms,
            "finest_iterations": [s.iterations for s in sts], "reached": all(s.gap <= GAP for s in sts),
            "form": f"plain FP32: each slice alone (8-neighbour in-plane prior, its own F_ref from {REF_ITERS} "
                    f"iterations), FBP start, one level, eager launches; {len(sl)} of {S} slices timed, scaled by "
                    f"{S / len(sl):g}"}


# ------------------------------------------------------------------------------ reference arm

def run_reference(args, rank, world):
    if rank != 0:
        return
    w = WORKLOADS[args.workload]
    cb = cpu_baseline(args.workload, single_thread=False)
    vals = []
    for _ in range(args.warmup):
        oracle_sample(args.workload, 1, 1)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        dt, _ = oracle_sample(args.workload, 1, 1)
        vals.append(w["N"] ** 2 / dt)
    el = time.perf_counter() - t0
    v = statistics.mean(vals)
    line = {
        "impl": "reference", "metric": METRIC, "value": v, "unit": "voxel-updates/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / max(args.steps, 1),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": config_of(args.workload),
        "cpu_baseline": dict(cb, value=v, sample=f"each step: 1 of {w['S']} slices x 1 iteration at {w['N']}^2, "
                                                 f"{w['na']} angles (oracle iteration phase)"),
        "e2e": {"value": v, "unit": "voxel-updates/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def config_of(name):
    w = WORKLOADS[name]
    c = {"workload": name, "slices": w["S"], "N": w["N"], "angles": w["na"], "span": w["span"]}
    if w["kind"] == "hier":
        c.update(levels=[w["N"] >> (LEVELS - 1 - k) for k in range(LEVELS)], gap=GAP)
    elif w["kind"] == "uneven":
        c.update(groups=[[N, na, UNEVEN_SLICES] for N in UNEVEN_SIDES for na in UNEVEN_ANGLES], gap=GAP)
    elif w["kind"] == "learned":
        c.update(gap=GAP, train={"N": LEARN_TRAIN_N, "pairs": LEARN_TRAIN_VOLUMES * LEARN_TRAIN_SLICES,
                                 "angles": [90, 180]})
    elif w["kind"] == "streamed":
        c.update(iterations=w["iters"], slab=w["slab"])
    else:
        c.update(iterations=w["iters"])
    return c


# ------------------------------------------------------------------------------ roofline

PASS_NAMES = ["pass1_rows_fwd", "pass2_columns", "pass3a_rows_inv", "pass3b_prior_update", "finalize"]


def pass_bytes(N):
    """Algorithmic HBM bytes per voxel-update of passes 1, 2, 3a, 3b (FP32 spectrum)."""
    B = (N + 1) / N
    return [8.0 + 8.0 * B, 16.0 * B, 8.0 * B + 4.0, 4.0 + 4 + 8 + 4]


# special-function operations per voxel of pass 3b: 13 neighbour pairs (each unordered pair of the
# 26-neighbourhood once) x (log2, exp2, reciprocal)
SFU_OPS_PER_VOXEL = 13 * 3


def roofline_of(pt, iters, S, N, workload, sfu_rate=None):
    """Per-pass fractions and the roofline line of the slowest pass.  Passes 1, 2, 3a are bound by
    HBM (the algorithmic bytes of pass_bytes over the CUDA-event time, against the measured copy
    bandwidth); pass 3b also against the measured special-function rate, and its line takes the
    tighter of the two ceilings."""
    peak, peak_kind = measured_peaks()
    bpv = pass_bytes(N)
    per = {}
    vox = S * N * N
    for k in range(4):
        sec = pt[k] / iters * 1e-3
        ach = bpv[k] * vox / sec / 1e9
        per[PASS_NAMES[k]] = {"ms": pt[k] / iters, "achieved_gbs": ach, "frac": ach / peak,
                              "algorithmic_bytes_per_voxel": bpv[k]}
    if sfu_rate:
        sec = pt[3] / iters * 1e-3
        per[PASS_NAMES[3]]["sfu"] = {"achieved_gops": SFU_OPS_PER_VOXEL * vox / sec / 1e9,
                                     "peak_gops": sfu_rate / 1e9,
                                     "frac": SFU_OPS_PER_VOXEL * vox / sec / sfu_rate,
                                     "ops_per_voxel": SFU_OPS_PER_VOXEL}
    top = max(range(4), key=lambda k: pt[k])
    name = PASS_NAMES[top]
    ach = per[name]["achieved_gbs"]
    roof = {"kernel": name, "bound": "hbm", "achieved": ach, "peak": peak, "unit": "GB/s", "frac": ach / peak,
            "peak_source": f"{peak_kind} (copy bandwidth)", "algorithmic_bytes_per_voxel": bpv[top],
            "traffic": kernel_traffic(name, workload), "per_pass": per}
    if "sfu" in per[name]:
        # the special-function ceiling is the lower one when its time floor is longer
        sf = per[name]["sfu"]
        if SFU_OPS_PER_VOXEL / sfu_rate > bpv[top] / (peak * 1e9):
            roof.update({"bound": "alu", "achieved": sf["achieved_gops"], "peak": sf["peak_gops"], "unit": "Gop/s",
                         "frac": sf["frac"], "peak_source": "measured: tmbir_sfu_rate (log2/exp2/reciprocal chains)",
                         "hbm": {"achieved": ach, "peak": peak, "unit": "GB/s", "frac": ach / peak}})
    return roof


# ------------------------------------------------------------------------------ main

def main():
    global _tm
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default=DEFAULT, choices=sorted(WORKLOADS))
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-graph", action="store_true", help="launch the iterations eagerly (profiling)")
    ap.add_argument("--no-gap", action="store_true", help="skip the time-to-gap forms")
    ap.add_argument("--no-tune", action="store_true",
                    help="keep the default coarse iteration counts instead of timing the candidates (profiling)")
    args = ap.parse_args()
    rank, world, local = dist_env()
    if args.impl == "reference":
        return run_reference(args, rank, world)

    import torch

    import paper_2603_28756_gb300 as tm

    _tm = tm
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    w = WORKLOADS[args.workload]
    t_gen = time.perf_counter()
    prob = make_problem(args.workload, rank)
    t_gen = time.perf_counter() - t_gen
    progress(f"inputs generated ({t_gen:.1f} s)")
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        if w["kind"] == "uneven":
            run_uneven(args, tm, prob, stream, rank, world, local, barrier, {"input_generation_s": t_gen})
        elif w["kind"] == "learned":
            run_learned(args, tm, w, prob, stream, rank, world, local, barrier, {"input_generation_s": t_gen})
        elif w["kind"] == "streamed":
            run_streamed(args, tm, w, prob, stream, rank, world, local, barrier, {"input_generation_s": t_gen})
        else:
            run_ours(args, tm, w, prob, stream, rank, world, local, barrier, {"input_generation_s": t_gen})
    if world > 1:
        torch.distributed.destroy_process_group()


def run_ours(args, tm, w, prob, stream, rank, world, local, barrier, extra):
    """Everything of our arm, with the bench stream current: every C-ABI call orders itself after
    it and the events recorded on it bracket the work."""
    import torch

    S, N, na, span = w["S"], w["N"], w["na"], w["span"]
    sino = torch.from_numpy(prob.sino.ravel()).cuda()

    if w["kind"] == "hier":
        H = Hier(tm, w, prob.theta)
        ctx = H.ctxs[-1]
        # F_ref: the hierarchy in FP32, then REF_ITERS more finest-level iterations
        t0 = time.perf_counter()
        ref_stats = H.run(sino, fp32_params(0.0, finest_iters=REF_ITERS, gap_tol=0.0), start_cnn=False)
        F_ref = ref_stats[-1].objective
        log = ctx.get_log(REF_ITERS)
        F0 = ctx.objective(torch.zeros_like(H.x), ctx._lv["atg"], tm_params())
        progress(f"F_ref {F_ref:.9g}")
        extra["F_ref"] = {"value": F_ref, "F0": F0, "finest_iterations": REF_ITERS,
                          "change_last_half_in_gap_units": (log[REF_ITERS // 2 - 1][0] - F_ref) / (F0 - F_ref),
                          "s": time.perf_counter() - t0}
        # launch shapes of every level by timing (pass-3b slices per block, spectrum chunk, rows
        # per block of the row passes where a side has variants)
        extra["autotune"] = [{"N": c.groups[0].N, "pass3_slices_per_block": c.autotune(c._lv["x"], c._lv["atg"],
                                                                                       tm_params()),
                              "spectrum_chunk": c.spec_chunks} for c in H.ctxs]
        # the learned start at the coarsest level (outside the timed region)
        try:
            H.net, extra["warm_start_training"] = train_warm_start(tm, w, 1 << (LEVELS - 1), stream)
        except Exception as e:  # reported, not hidden: the step then starts from FBP
            extra["warm_start_training"] = {"error": str(e)[:300]}
        progress(f"warm start trained: {extra['warm_start_training']}")
        if args.no_tune:
            coarse, extra["coarse_iteration_tuning"] = COARSE_ITERS, "skipped (--no-tune)"
        else:
            coarse, extra["coarse_iteration_tuning"] = tune_coarse(H, sino, F_ref, stream, barrier, world)
        progress(f"coarse iterations {coarse}: {extra['coarse_iteration_tuning']}")
        prms = chosen_params(F_ref, coarse)
        if args.no_graph:  # profiling: every iteration's kernels launched one by one
            for prm in prms:
                prm.use_graph = False
        state = {}

        def step():
            state["stats"] = H.run(sino, prms, coarse_fp32=True)

        def units():
            return H.voxel_updates(state["stats"])
    else:
        ctx = tm.Context([tm.Group(N=N, angles=list(prob.theta), n_slices=S, span=span)], stream=stream)
        with torch.cuda.stream(stream):
            atg = torch.empty(S * N * N, dtype=torch.float32, device="cuda")
            x = torch.empty_like(atg)
        prm = tm_params(max_iter=w["iters"], use_graph=not args.no_graph)
        ctx.build_operator(sino, atg)
        ctx.fbp(sino, x)
        extra["autotune_pass3_slices_per_block"] = ctx.autotune(x, atg, prm)

        def step():
            ctx.build_operator_fbp(sino, atg, x)
            ctx.reconstruct(x, atg, prm, want_stats=False)

        def units():
            return S * N * N * w["iters"]

    # tmbir_launch_count is the process-wide host count plus the context's device-side graph
    # count; a context that runs no graph gives the host count alone
    host_ctx = tm.Context([tm.Group(N=64, angles=[0.0], n_slices=1)], stream=stream)
    all_ctxs = [ctx] if w["kind"] == "fixed" else H.ctxs

    def launch_total():
        host = host_ctx.launch_count()
        return host + sum(c.launch_count() - host for c in all_ctxs)

    torch.cuda.synchronize()
    for _ in range(args.warmup):
        step()
    barrier()
    clocks = Clocks(local)
    n0 = launch_total()
    step_units = []
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier()
    torch.cuda.nvtx.range_push("bench_timed_steps")  # lets a profiler select the timed launches
    e0.record(stream)
    for _ in range(args.steps):
        step()
        step_units.append(units())
    e1.record(stream)
    barrier()
    torch.cuda.nvtx.range_pop()
    clk = clocks.stop()
    progress(f"timed steps done: {e0.elapsed_time(e1) / args.steps:.1f} ms per step")
    launches = launch_total() - n0
    ms = max_over_ranks(e0.elapsed_time(e1), world, "cuda")
    vox = sum(step_units) / len(step_units)
    value = job_rate(vox, args.steps, world, ms)

    # iteration phase of the finest level, eager, pass by pass on the context stream
    xf = ctx._lv["x"] if w["kind"] == "hier" else x
    af = ctx._lv["atg"] if w["kind"] == "hier" else atg
    it_pass = PASS_ITERS if w["kind"] == "hier" else w["iters"]
    ctx.fbp(sino, xf)
    pt = ctx.pass_times(xf, af, tm_params(), it_pass)
    pt16 = ctx.pass_times(xf, af, tm_params(bf16=True), it_pass)
    it_ms = sum(pt)
    sfu = ctx.sfu_rate()
    roof = roofline_of(pt, it_pass, S, N, args.workload, sfu)
    progress(f"pass times (ms per iteration) {[round(v / it_pass, 3) for v in pt]}, bf16 {[round(v / it_pass, 3) for v in pt16]}")
    iteration_phase = {
        "level": f"{N}^2 x {S} slices", "iterations": it_pass,
        "voxel_updates_per_s": S * N * N * it_pass / (it_ms * 1e-3), "ms_per_iteration": it_ms / it_pass,
        "ms_per_pass": dict(zip(PASS_NAMES, [v / it_pass for v in pt])),
        "bf16_ms_per_iteration": sum(pt16) / it_pass,
        "bf16_ms_per_pass": dict(zip(PASS_NAMES, [v / it_pass for v in pt16])),
    }

    direct = gradient_comparison(ctx, xf, af, sino, stream, barrier)
    progress(f"direct vs Toeplitz gradient: {direct}")

    # one step broken down by stage (outside the timed region)
    breakdown = None
    if w["kind"] == "hier":
        breakdown = stage_breakdown(tm, H, sino, prms, stream, barrier)
    else:
        barrier()
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
        ev[0].record(stream)
        ctx.build_operator(sino, atg)
        ev[1].record(stream)
        ctx.fbp(sino, x)
        ev[2].record(stream)
        barrier()
        breakdown = {"build_operator_data": ev[0].elapsed_time(ev[1]), "fbp": ev[1].elapsed_time(ev[2])}

    # end to end through the C ABI with host buffers: H2D sinogram, the step, D2H image
    h_sino = torch.from_numpy(prob.sino.ravel()).pin_memory()
    xout = H.x if w["kind"] == "hier" else x
    h_x = torch.empty(xout.numel(), dtype=torch.float32).pin_memory()
    d_sino = torch.empty_like(sino)
    e2e_units = []

    def e2e_step():
        with torch.cuda.stream(stream):
            d_sino.copy_(h_sino, non_blocking=True)
        if w["kind"] == "hier":
            state["stats"] = H.run(d_sino, prms, coarse_fp32=True)
            e2e_units.append(units())
            out = H.x
        else:
            ctx.build_operator_fbp(d_sino, atg, x)
            ctx.reconstruct(x, atg, prm, want_stats=False)
            e2e_units.append(units())
            out = x
        with torch.cuda.stream(stream):
            h_x.copy_(out, non_blocking=True)

    e2e_step()  # warm (the sinogram buffer differs from the timed steps')
    e2e_units.clear()
    barrier()
    f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    f0.record(stream)
    for _ in range(args.steps):
        e2e_step()
    f1.record(stream)
    barrier()
    e2e_ms = max_over_ranks(f0.elapsed_time(f1), world, "cuda")
    e2e_value = job_rate(sum(e2e_units) / len(e2e_units), args.steps, world, e2e_ms)
    progress(f"e2e {e2e_ms / args.steps:.1f} ms per step")

    gap_info = None
    if not args.no_gap:
        if w["kind"] == "hier":
            gap_info = {"gap": GAP, "F_ref": extra["F_ref"],
                        "forms": time_to_gap_hier(tm, H, sino, extra["F_ref"]["value"], extra["F_ref"]["F0"], stream,
                                                  barrier, world, ms / args.steps, state["stats"],
                                                  [s.iterations for s in state["stats"][:-1]])}

    if rank == 0:
        cfg = config_of(args.workload)
        cfg.update({"parallelism": f"replicas{world}", "l2": "working set > L2 (no explicit flush)"})
        if w["kind"] == "hier":
            cfg.update({"step": "chosen form to the 1e-3 gap: 3 levels (coarse R*g in FP32), CNN start with FBP "
                                "fallback, BF16 spectra with FP32 refinement, device-driven graph loops",
                        "coarse_iterations": [s.iterations for s in state["stats"][:-1]],
                        "refine_gap": REFINE_GAP,
                        "level_iterations": [s.iterations for s in state["stats"]]})
        else:
            cfg.update({"step": "build_operator_fbp (R*g and FBP overlapped) + reconstruct(graph)"})
        line = {
            "metric": METRIC,
            "value": value,
            "unit": "voxel-updates/s",
            "n_gpus": world,
            "steps": args.steps,
            "warmup": args.warmup,
            "ms_per_step": ms / args.steps,
            "higher_is_better": True,
            "scaling": "weak",
            "vs_baseline": None,
            "dtype": "f32",
            "data": "synthetic",
            "config": cfg,
            "voxel_updates_per_step": vox,
            "iteration_phase": iteration_phase,
            "toeplitz_vs_direct_gradient": direct,
            "step_breakdown_ms": breakdown,
            "roofline": roof,
            "e2e": {"value": e2e_value, "unit": "voxel-updates/s", "h2d_bytes_per_step": sino.numel() * 4,
                    "d2h_bytes_per_step": xout.numel() * 4},
            "gpu_launches": launches,
            "time_to_gap": gap_info,
            "clocks": clk,
        }
        line.update(extra)
        if not args.no_cpu_baseline:
            line["cpu_baseline"] = cpu_baseline(args.workload)
        print(json.dumps(line), flush=True)


def run_uneven(args, tm, probs, stream, rank, world, local, barrier, extra):
    """The uneven batch (16 geometry groups of 16 slices) in one context: every iteration runs the
    groups' passes from one device-driven graph loop; each group has its own step constant and
    momentum, the stop rule is the whole batch's gap.  One step = setup (R*g, FBP) + iterations to
    the 1e-3 gap.  Per-size throughput from contexts holding the four groups of one side."""
    import torch

    groups = [tm.Group(N=p.N, angles=list(p.theta), n_slices=UNEVEN_SLICES, span=p.span) for p in probs]
    ctx = tm.Context(groups, stream=stream)
    sino = torch.from_numpy(__import__("numpy").concatenate([p.sino.ravel() for p in probs])).cuda()
    atg, x = ctx.build_operator_fbp(sino)
    extra["autotune_pass3_slices_per_block"] = ctx.autotune(x, atg, tm_params())
    extra["autotune_spectrum_chunk"] = ctx.spec_chunks
    t0 = time.perf_counter()
    ref = ctx.reconstruct(x, atg, tm_params(max_iter=REF_ITERS))
    log = ctx.get_log(REF_ITERS)
    F0 = ctx.objective(torch.zeros_like(x), atg, tm_params())
    F_ref = ref.objective
    extra["F_ref"] = {"value": F_ref, "F0": F0, "iterations": REF_ITERS,
                      "change_last_half_in_gap_units": (log[REF_ITERS // 2 - 1][0] - F_ref) / (F0 - F_ref),
                      "s": time.perf_counter() - t0}
    progress(f"F_ref {F_ref:.9g}")
    per_iter = sum(g.n_slices * g.N * g.N for g in groups)
    prm = tm_params(max_iter=PLAIN_CAP, gap_tol=GAP, F_ref=F_ref)
    state = {}

    def step(s_in=sino):
        ctx.build_operator_fbp(s_in, atg, x)
        state["st"] = ctx.reconstruct(x, atg, prm)
        return per_iter * state["st"].iterations

    host_ctx = tm.Context([tm.Group(N=64, angles=[0.0], n_slices=1)], stream=stream)
    for _ in range(args.warmup):
        step()
    barrier()
    clocks = Clocks(local)
    n0 = ctx.launch_count()
    h0 = host_ctx.launch_count()
    units = []
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier()
    e0.record(stream)
    for _ in range(args.steps):
        units.append(step())
    e1.record(stream)
    barrier()
    clk = clocks.stop()
    launches = ctx.launch_count() - n0
    ms = max_over_ranks(e0.elapsed_time(e1), world, "cuda")
    vox = sum(units) / len(units)
    value = job_rate(vox, args.steps, world, ms)
    progress(f"timed steps: {ms / args.steps:.1f} ms, {state['st'].iterations} iterations, host launches "
             f"{host_ctx.launch_count() - h0}")
    # iteration phase of the whole batch, and per image side (its four groups alone)
    pt = ctx.pass_times(x, atg, tm_params(), PASS_ITERS)
    per_size = {}
    roof = None
    for N in UNEVEN_SIDES:
        idx = [k for k, g in enumerate(groups) if g.N == N]
        sub = tm.Context([groups[k] for k in idx], stream=stream)
        off, parts = 0, []
        for k, g in enumerate(groups):
            n = g.n_slices * len(g.angles) * g.N
            if k in idx:
                parts.append(sino[off:off + n])
            off += n
        s_sub = torch.cat(parts)
        a_sub, x_sub = sub.build_operator_fbp(s_sub)
        sub.autotune(x_sub, a_sub, tm_params())
        pts = sub.pass_times(x_sub, a_sub, tm_params(), PASS_ITERS)
        nvox = sum(groups[k].n_slices * N * N for k in idx)
        per_size[str(N)] = {"voxel_updates_per_s": nvox * PASS_ITERS / (sum(pts) * 1e-3),
                            "ms_per_iteration": sum(pts) / PASS_ITERS,
                            "ms_per_pass": dict(zip(PASS_NAMES, [v / PASS_ITERS for v in pts]))}
        if N == max(UNEVEN_SIDES):
            roof = roofline_of(pts, PASS_ITERS, nvox // (N * N), N, args.workload, ctx.sfu_rate())
        del sub
    progress(f"per size {json.dumps(per_size)}")
    # end to end with host buffers
    h_sino = torch.from_numpy(__import__("numpy").concatenate([p.sino.ravel() for p in probs])).pin_memory()
    h_x = torch.empty(x.numel(), dtype=torch.float32).pin_memory()
    d_sino = torch.empty_like(sino)
    barrier()
    f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    f0.record(stream)
    e_units = []
    for _ in range(args.steps):
        d_sino.copy_(h_sino, non_blocking=True)
        e_units.append(step(d_sino))
        h_x.copy_(x, non_blocking=True)
    f1.record(stream)
    barrier()
    e2e_ms = max_over_ranks(f0.elapsed_time(f1), world, "cuda")
    if rank == 0:
        cfg = {"workload": args.workload, "groups": [[g.N, len(g.angles), g.n_slices] for g in groups],
               "slices": sum(g.n_slices for g in groups), "gap": GAP, "parallelism": f"replicas{world}",
               "l2": "working set > L2 (no explicit flush)",
               "step": "build_operator_fbp + reconstruct (FP32, FBP start, one level, graph loop) to the 1e-3 gap"}
        line = {
            "metric": METRIC, "value": value, "unit": "voxel-updates/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic", "config": cfg,
            "voxel_updates_per_step": vox, "iterations_to_gap": state["st"].iterations,
            "iteration_phase": {"voxel_updates_per_s": per_iter * PASS_ITERS / (sum(pt) * 1e-3),
                                "ms_per_iteration": sum(pt) / PASS_ITERS,
                                "ms_per_pass": dict(zip(PASS_NAMES, [v / PASS_ITERS for v in pt])),
                                "per_size": per_size},
            "roofline": roof,
            "e2e": {"value": job_rate(sum(e_units) / len(e_units), args.steps, world, e2e_ms),
                    "unit": "voxel-updates/s", "h2d_bytes_per_step": sino.numel() * 4,
                    "d2h_bytes_per_step": x.numel() * 4},
            "gpu_launches": launches, "clocks": clk,
        }
        line.update(extra)
        if not args.no_cpu_baseline:
            line["cpu_baseline"] = cpu_baseline(args.workload)
        print(json.dumps(line), flush=True)


def learned_training_set(tm, w, stream, rank):
    """(FBP, converged) pairs at LEARN_TRAIN_N^2: LEARN_TRAIN_VOLUMES seeded volumes, each with an
    angle count drawn from 90..180 over [0, pi), reconstructed by the method itself (FP32, to
    LEARN_TARGET_GAP of an F_ref from twice as many iterations)."""
    import numpy as np
    import torch

    import synth

    rng = np.random.default_rng(rank_seed(rank, 7100))
    fbps, targets, info = [], [], []
    for v in range(LEARN_TRAIN_VOLUMES):
        na = int(rng.integers(90, 181))
        p = synth.volume(S=LEARN_TRAIN_SLICES, N=LEARN_TRAIN_N, n_angles=na, n_ellipsoids=w["ne"], span=math.pi,
                         seed=rank_seed(rank, 7200 + v))
        ctx = tm.Context([tm.Group(N=LEARN_TRAIN_N, angles=list(p.theta), n_slices=LEARN_TRAIN_SLICES)],
                         stream=stream)
        sino = torch.from_numpy(p.sino.ravel()).cuda()
        atg, f0 = ctx.build_operator_fbp(sino)
        x = f0.clone()
        F_ref = ctx.reconstruct(x, atg, tm_params(max_iter=600)).objective
        x.copy_(f0)
        st = ctx.reconstruct(x, atg, tm_params(max_iter=600, gap_tol=LEARN_TARGET_GAP, F_ref=F_ref))
        fbps.append(f0)
        targets.append(x)
        info.append((na, st.iterations))
        del ctx
    return torch.cat(fbps), torch.cat(targets), info


def run_learned(args, tm, w, prob, stream, rank, world, local, barrier, extra):
    """The learned warm start at a size it was not trained on: the network trained at
    1024^2 on pairs with 90..180 angles, then applied to 2560^2 slices with 150 angles; the step
    is setup + CNN-refined start (FBP fallback) + iterations to the 1e-3 gap, compared with the
    FBP start."""
    import torch

    S, N, na, span = w["S"], w["N"], w["na"], w["span"]
    t0 = time.perf_counter()
    fbp_t, tgt_t, info = learned_training_set(tm, w, stream, rank)
    extra["training_set"] = {"pairs": fbp_t.numel() // LEARN_TRAIN_N ** 2, "image": LEARN_TRAIN_N,
                             "angle_counts_and_iterations": info, "s": time.perf_counter() - t0}
    progress(f"training set {extra['training_set']}")
    net = tm.CNN(LEARN_TRAIN_N, LEARN_TRAIN_N, max_batch=CNN_BATCH, stream=stream, seed=11)
    plane = LEARN_TRAIN_N ** 2
    npairs = fbp_t.numel() // plane
    losses = []
    t0 = time.perf_counter()
    gen = torch.Generator().manual_seed(5)
    for _ in range(LEARN_EPOCHS):
        order = torch.randperm(npairs // CNN_BATCH, generator=gen).tolist()
        ep = []
        for b in order:
            sl = slice(b * CNN_BATCH * plane, (b + 1) * CNN_BATCH * plane)
            ep.append(net.train_step(fbp_t[sl], tgt_t[sl], CNN_BATCH, lr=1e-3))
        losses.append(sum(ep) / len(ep))
    extra["training"] = {"epochs": LEARN_EPOCHS, "batch": CNN_BATCH, "loss_per_epoch": losses,
                         "s": time.perf_counter() - t0}
    progress(f"trained {extra['training']}")
    del fbp_t, tgt_t
    weights = net.get_weights()
    del net
    # evaluation at 2560^2: a network of that image size with the trained weights
    ev = tm.CNN(N, N, max_batch=4, stream=stream, seed=11)
    ev.set_weights(weights)
    ctx = tm.Context([tm.Group(N=N, angles=list(prob.theta), n_slices=S, span=span)], stream=stream)
    sino = torch.from_numpy(prob.sino.ravel()).cuda()
    atg, f0 = ctx.build_operator_fbp(sino)
    x = f0.clone()
    t0 = time.perf_counter()
    F_ref = ctx.reconstruct(x, atg, tm_params(max_iter=REF_ITERS)).objective
    log = ctx.get_log(REF_ITERS)
    F0 = ctx.objective(torch.zeros_like(x), atg, tm_params())
    extra["F_ref"] = {"value": F_ref, "F0": F0, "iterations": REF_ITERS,
                      "change_last_half_in_gap_units": (log[REF_ITERS // 2 - 1][0] - F_ref) / (F0 - F_ref),
                      "s": time.perf_counter() - t0}
    progress(f"F_ref {F_ref:.9g}")
    stop = tm_params(max_iter=PLAIN_CAP, gap_tol=GAP, F_ref=F_ref)
    state = {}

    def step_cnn():
        ctx.build_operator_fbp(sino, atg, f0)
        _, state["used"] = ev.warm_start(ctx, f0, atg, tm_params(), out=x)
        state["st"] = ctx.reconstruct(x, atg, stop)
        return S * N * N * state["st"].iterations

    def step_fbp():
        ctx.build_operator_fbp(sino, atg, x)
        state["st_fbp"] = ctx.reconstruct(x, atg, stop)
        return S * N * N * state["st_fbp"].iterations

    for _ in range(args.warmup):
        step_cnn()
    barrier()
    clocks = Clocks(local)
    units = []
    ms, _ = timed(stream, barrier, world, lambda: [units.append(step_cnn()) for _ in range(args.steps)])
    clk = clocks.stop()
    ms_fbp, _ = timed(stream, barrier, world, step_fbp)
    F_fbp = ctx.objective(f0, atg, tm_params())
    ev.warm_start(ctx, f0, atg, tm_params(), out=x)
    F_cnn = ctx.objective(x, atg, tm_params())
    progress(f"cnn start {ms / args.steps:.1f} ms ({state['st'].iterations} it, used {state['used']}), "
             f"fbp start {ms_fbp:.1f} ms ({state['st_fbp'].iterations} it)")
    if rank == 0:
        cfg = config_of(args.workload)
        cfg.update({"parallelism": f"replicas{world}", "l2": "working set > L2 (no explicit flush)",
                    "step": "build_operator_fbp + CNN-refined start (FBP fallback) + reconstruct (FP32, graph) to "
                            "the 1e-3 gap", "train_image": LEARN_TRAIN_N})
        vox = sum(units) / len(units)
        line = {
            "metric": METRIC, "value": job_rate(vox, args.steps, world, ms), "unit": "voxel-updates/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": cfg, "voxel_updates_per_step": vox,
            "time_to_gap": {"gap": GAP, "F_ref": extra.pop("F_ref"), "forms": {
                "learned": {"ms": ms / args.steps, "iterations": state["st"].iterations, "used_cnn": state["used"],
                            "start_gap": (F_cnn - F_ref) / (F0 - F_ref)},
                "fbp": {"ms": ms_fbp, "iterations": state["st_fbp"].iterations,
                        "start_gap": (F_fbp - F_ref) / (F0 - F_ref)},
                "iterations_saved": state["st_fbp"].iterations - state["st"].iterations}},
            "clocks": clk,
            "e2e": None,
        }
        line.update(extra)
        print(json.dumps(line), flush=True)


def host_link(stream, nbytes=1 << 30, reps=3):
    """Page-locked host <-> device copy rates (GB/s, best of reps, CUDA events): one direction at a
    time on one stream, host-to-device on two streams at once, and both directions at once."""
    import torch

    h = [torch.empty(nbytes, dtype=torch.uint8, pin_memory=True) for _ in range(2)]
    d = [torch.empty(nbytes, dtype=torch.uint8, device="cuda") for _ in range(2)]
    s2 = torch.cuda.Stream()

    def rate(fn, moved):
        best = 0.0
        for _ in range(reps):
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fn()
            s2.wait_stream(stream)
            stream.wait_stream(s2)
            e1.record(stream)
            e1.synchronize()
            best = max(best, moved / (e0.elapsed_time(e1) * 1e-3) / 1e9)
        return best

    def two(first, second):
        def fn():
            s2.wait_stream(stream)
            first()
            with torch.cuda.stream(s2):
                second()
        return fn

    return {
        "h2d": rate(lambda: d[0].copy_(h[0], non_blocking=True), nbytes),
        "d2h": rate(lambda: h[0].copy_(d[0], non_blocking=True), nbytes),
        "h2d_two_streams": rate(two(lambda: d[0].copy_(h[0], non_blocking=True),
                                    lambda: d[1].copy_(h[1], non_blocking=True)), 2 * nbytes),
        "both_directions": rate(two(lambda: d[0].copy_(h[0], non_blocking=True),
                                    lambda: h[1].copy_(d[1], non_blocking=True)), 2 * nbytes),
    }


def run_streamed(args, tm, w, prob, stream, rank, world, local, barrier, extra):
    """A volume in host memory streamed through the GPU slab by slab: one step is the streamed
    setup (R*g, 1/2 g.g and the FBP start) and `iters` streamed FP32 iterations, every input read
    from and every output written to page-locked host memory.  The same iterations on the
    resident volume give the streaming overhead, and their final iterates are compared."""
    import torch

    S, N, na, span, slab, iters = w["S"], w["N"], w["na"], w["span"], w["slab"], w["iters"]
    ctx = tm.Context([tm.Group(N=N, angles=list(prob.theta), n_slices=slab, span=span)], stream=stream)
    h_sino = torch.from_numpy(prob.sino.ravel()).pin_memory()
    h_x = torch.empty(S * N * N, dtype=torch.float32, pin_memory=True)
    prm = tm_params(max_iter=iters)
    state = {}

    def step():
        h_atg, gtg, h_x0 = ctx.stream_build_operator(h_sino, S, fbp=True)
        h_x.copy_(h_x0)
        state["st"] = ctx.stream_reconstruct(h_x, h_atg, gtg, prm)
        state["atg"], state["gtg"], state["x0"] = h_atg, gtg, h_x0
        return S * N * N * state["st"].iterations

    for _ in range(args.warmup):
        step()
    barrier()
    clocks = Clocks(local)
    units = []
    n0 = ctx.launch_count()
    ms, _ = timed(stream, barrier, world, lambda: [units.append(step()) for _ in range(args.steps)])
    launches = ctx.launch_count() - n0
    clk = clocks.stop()
    # the iteration phase alone, streamed and resident
    h_x.copy_(state["x0"])
    ms_it, _ = timed(stream, barrier, world, lambda: ctx.stream_reconstruct(h_x, state["atg"], state["gtg"], prm))
    x_streamed = h_x.clone()
    # the same with R*g kept in device memory (only the iterates stream)
    d_atg = state["atg"].cuda()
    h_x.copy_(state["x0"])
    ms_it_dev, _ = timed(stream, barrier, world, lambda: ctx.stream_reconstruct(h_x, d_atg, state["gtg"], prm))
    same_dev = bool(torch.equal(h_x, x_streamed))
    del d_atg
    res = tm.Context([tm.Group(N=N, angles=list(prob.theta), n_slices=S, span=span)], stream=stream)
    atg = res.build_operator(h_sino.cuda())
    atg_same = bool(torch.equal(atg.cpu(), state["atg"]))
    x = state["x0"].cuda()
    res.reconstruct(x.clone(), atg, prm)
    ms_res, _ = timed(stream, barrier, world, lambda: res.reconstruct(x, atg, prm))
    diff = float((x.cpu() - x_streamed).abs().max()) / max(float(x_streamed.abs().max()), 1e-30)
    del res, atg, x
    link = host_link(stream)
    progress(f"host link GB/s {link}")
    nslab = (S + slab - 1) // slab
    plane = N * N * 4
    h2d_it = (2 * (S + 2 * (nslab - 1)) + S) * plane  # x_k and x_{k-1} with the halo slices, R*g
    d2h_it = S * plane
    progress(f"streamed step {ms / args.steps:.1f} ms; iterations streamed {ms_it / iters:.1f} ms (R*g on the "
             f"device {ms_it_dev / iters:.1f} ms), resident "
             f"{ms_res / iters:.1f} ms per iteration; max |difference| / max |x| = {diff:.2e}")
    if rank == 0:
        cfg = config_of(args.workload)
        cfg.update({"parallelism": f"replicas{world}", "l2": "working set > L2 (no explicit flush)",
                    "step": "stream_build_operator (R*g, FBP) + stream_reconstruct, host volume in slabs of "
                            f"{slab} slices", "stand_in_for": "2048 x 2448^2 nano-CT volume, 212 angles"})
        vox = sum(units) / len(units)
        val = job_rate(vox, args.steps, world, ms)
        sino_b = S * na * N * 4
        line = {
            "metric": METRIC, "value": val, "unit": "voxel-updates/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic", "config": cfg, "voxel_updates_per_step": vox,
            "streaming": {
                "slab": slab, "slabs": nslab,
                "streamed_ms_per_iteration": ms_it / iters, "resident_ms_per_iteration": ms_res / iters,
                "streamed_atg_on_device_ms_per_iteration": ms_it_dev / iters,
                "atg_on_device_iterates_equal": same_dev,
                "overhead": ms_it / ms_res,
                "host_copies_per_iteration_bytes": {"h2d": h2d_it, "d2h": d2h_it},
                "copy_GBps_per_iteration": (h2d_it + d2h_it) / (ms_it / iters) / 1e6,
                "host_link_GBps": link,
                # the copies alone at the measured rates (both directions at once): the streamed
                # iteration's floor when it is copy-bound
                "copy_floor_ms_per_iteration": (h2d_it + d2h_it) / (link["both_directions"] * 1e9) * 1e3,
                "max_abs_difference_vs_resident_over_max_abs_x": diff,
                "atg_bitwise_equal_to_resident": atg_same,
                "host_bytes_for_the_2048_slice_volume": 5 * 2048 * plane,
            },
            "clocks": clk,
            "e2e": {"value": val, "unit": "voxel-updates/s", "h2d_bytes_per_step": sino_b + iters * h2d_it,
                    "d2h_bytes_per_step": 2 * S * plane + iters * d2h_it},
            "gpu_launches": launches,
        }
        line.update(extra)
        print(json.dumps(line), flush=True)


def gradient_comparison(ctx, x, atg, sino, stream, barrier, reps=3):
    """Sec. 3.1's comparison at the workload's finest level: one gradient through the Toeplitz
    passes (R*R as the 2N x 2N FFT convolution, R*g precomputed) against the direct gradient
    R*(R x - g) through the two NUFFTs; device ms of each and their relative L2 difference."""
    import torch

    prm = tm_params()
    gt = ctx.gradient(x, atg, prm)
    gd = ctx.gradient_direct(x, sino, prm)

    def time_it(fn):
        barrier()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            fn()
        e1.record(stream)
        barrier()
        return e0.elapsed_time(e1) / reps

    t_toep = time_it(lambda: ctx.gradient(x, atg, prm, out=gt))
    t_dir = time_it(lambda: ctx.gradient_direct(x, sino, prm, out=gd))
    d = torch.linalg.norm((gd - gt).double())
    return {"toeplitz_ms": t_toep, "direct_ms": t_dir, "direct_over_toeplitz": t_dir / t_toep,
            "relative_l2_difference": float(d / torch.linalg.norm(gt.double())),
            # the gradient is the difference of R*R x and R*g, which nearly cancel near a
            # solution; on the scale of R*g the difference is the operators' own error
            "difference_over_atg_norm": float(d / torch.linalg.norm(atg.double()))}


def stage_breakdown(tm, H, sino, prms, stream, barrier):
    """Device ms of each stage of one chosen-form step (events between the C-ABI calls)."""
    import torch

    w = H.w
    S, N, na = w["S"], w["N"], w["na"]
    marks = []

    def mark(name):
        ev = torch.cuda.Event(enable_timing=True)
        ev.record(stream)
        marks.append((name, ev))

    barrier()
    mark("start")
    x = None
    for lev in range(LEVELS):
        f = 1 << (LEVELS - 1 - lev)
        Nl = N // f
        c = H.ctxs[lev]
        lv = c._lv
        s_l = sino if f == 1 else c.downsample_sino(sino, S, na, N, f, out=lv["sino"])
        c.build_operator(s_l, lv["atg"], fp64=lev == LEVELS - 1)  # as the chosen form
        mark(f"L{lev} setup")
        if x is None:
            f0 = c.fbp(s_l)
            mark(f"L{lev} fbp")
            if H.net is not None:
                x0, _ = H.net.warm_start(c, f0, lv["atg"], tm.Params(**PRIOR))
                lv["x"].copy_(x0)
            else:
                lv["x"].copy_(f0)
            mark(f"L{lev} warm_start")
        else:
            c.upsample_lanczos3(x, S, Nl // 2, out=lv["x"])
            mark(f"L{lev} upsample")
        x = lv["x"]
        c.reconstruct(x, lv["atg"], prms[lev])
        mark(f"L{lev} iterations")
    barrier()
    return {name: marks[k - 1][1].elapsed_time(ev) for k, (name, ev) in enumerate(marks) if k > 0}


if __name__ == "__main__":
    main()
