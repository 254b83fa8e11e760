"""Benchmark: chi0 (tetra x band-pair x q x omega) evals/s on one GB300.

Default workload: the large mixed-precision run -- an 80-band seeded tight-binding model on a
72^3 k mesh (2,239,488 tetrahedra, complex64 eigenvectors, 19.1 GB), 128 on-grid q points and
256 frequencies in [0, 2] eV.  One step = the dynamic chi0 (Re and Im, Eqs. 1-3) of a stated
subset of the 128 q points (``--nq``, default 1) at all 256 frequencies, every stage in the
CUDA library: tensor-core overlaps (split-BF16, three pieces), carving and frequency-resolved
weights (FP32 with FP64 near-degenerate branches), reduction.  ``value`` is that mixed form
with inputs resident in HBM; the all-FP64 GPU form is timed on the same inputs and reported
beside it with the normwise error between the two; the FP64 CPU oracle is timed on a bounded,
seeded sample of the builtin tetrahedra of the same q (``cpu_baseline``), and the GPU forms run
on the same sample are compared with it (``error.vs_oracle``).  After the timed steps the
Kramers-Kronig route (Im alone on a grid over the whole spectrum, Re by the transform) is
timed on the same q and compared with the direct form (``kk_route``; ``--no-kk`` skips it).

Other workloads (``--workload``): cr (Cr-like 9-band static, 48^3, 256 q), free (free-electron
Lindhard), fese (FeSe-like dynamic, 512 w), sweep (40-band window sweep, static).

``--impl reference`` times the oracle alone (host cores) on the same metric.  Under torchrun
every rank runs its own replica of the workload (independent q sets: no data-path
collective); rank 0 prints the JSON line.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_1407_3444_gb300 import workloads as wl  # noqa: E402

METRIC = "chi0 (tetra x band-pair x q x omega) evals/s, mixed vs all-FP64 GPU at 1e-6 rel"
LARGE_NQ = 128  # q points of the large run (a step takes a stated subset)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-tune", action="store_true",
                    help="skip chi0_tune (launch-shape autotuner) before the warm-up steps")
    ap.add_argument("--tune", action="store_true", help="run chi0_tune on the large run too (skipped by default)")
    ap.add_argument("--overlap", default="auto", choices=["auto", "fp32", "bf16x3", "bf16x6", "tf32"],
                    help="matrix elements of the mixed form: auto = three-piece split-BF16 on the tensor cores "
                         "for the 80-band run, FP32 on the CUDA cores for the small windows of the others")
    ap.add_argument("--workload", default="large", choices=["large", "cr", "free", "fese", "sweep"],
                    help="large: 80-band 72^3 dynamic (default); cr: Cr-like 9-orbital static; free: "
                         "free-electron Lindhard; fese: FeSe-like dynamic; sweep: 40-band window sweep (static)")
    ap.add_argument("--nw", type=int, default=0, help="dynamic workloads: the first NW frequencies only")
    ap.add_argument("--nq", type=int, default=None,
                    help="q points per step (large: a subset of its 128, default 1; others: the workload's)")
    ap.add_argument("--n", type=int, default=None, help="k mesh cubes per axis (cubic workloads)")
    ap.add_argument("--fp64-steps", type=int, default=1)
    ap.add_argument("--e2e-steps", type=int, default=5)
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--cpu-sample-q", type=int, default=None,
                    help="static workloads: q points of the oracle's timed sample (default 8; 2 per "
                         "--impl reference step)")
    ap.add_argument("--cpu-sample-w", type=int, default=16, help="dynamic workloads: frequencies of the oracle sample")
    ap.add_argument("--cpu-tets", type=int, default=None,
                    help="large: tetrahedra of the oracle sample (default 192; 48 per --impl reference step)")
    ap.add_argument("--tets", type=int, default=0,
                    help="large: the step on a seeded sample of TETS of the mesh's tetrahedra (the full mesh's mix "
                         "of final tetrahedra at a fraction of its size, for profiler counters); nominal evals "
                         "scale by TETS / ntet")
    ap.add_argument("--no-kk", action="store_true",
                    help="dynamic workloads: skip the Kramers-Kronig route's timing (Im alone on a grid over the "
                         "whole spectrum, Re by the transform), reported beside the direct principal value")
    ap.add_argument("--profile-out", default="")
    return ap.parse_args()


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def reduce_max(x: float) -> float:
    """Maximum of a host value over the ranks of the default process group (the timing rule:
    the whole job is as slow as its slowest rank); identity without a group."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return x
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(world_size: int, units_per_rank: float, max_ms: float) -> float:
    """Units all ranks processed per second (every rank runs its own replica)."""
    return world_size * units_per_rank / (max_ms * 1e-3)


def overlap_mode(args):
    if args.overlap != "auto":
        return args.overlap
    return "bf16x6" if args.workload == "large" else "fp32"


def make_workload(args, nproc):
    """The selected workload (the five synthetic stand-ins of the paper's materials)."""
    k = args.workload
    if k == "cr":
        return wl.cr_like(n=args.n or 48, nq=args.nq or 256, nproc=nproc)
    if k == "free":
        return wl.free_electron(n=args.n or 16, nq=args.nq or 32)
    if k == "fese":
        nq = args.nq or 64
        n = (args.n, args.n, max(1, args.n // 4)) if args.n else (64, 64, 16)
        W = wl.fese_like(n=n, nq=64, nproc=nproc,
                         qfracs=[np.array([0.5, 0.5, 0.0]) * (j + 1) / 64 for j in range(64)][:nq])
    elif k == "sweep":
        W = wl.band_sweep(n=args.n or 32, nq=args.nq or 128, nproc=nproc)
        W.omega = None  # the static sweep (the dynamic one: chi0_dynamic on the same plan)
        return W
    else:
        W = wl.large_mixed(n=args.n or 72, nq=LARGE_NQ, nproc=nproc)
        W.meta["nq_total"] = len(W.qs)
        W.qs = W.qs[:args.nq or 1]
    if args.nw:
        W.omega = W.omega[:args.nw]
    return W


def workload_config(W, args):
    names = {"cr": "Cr-like 9-orbital static chi0 (Gamma-X-M-Gamma, explicit k+q eigen-data, E_F at 6/9)",
             "free": "free-electron static Lindhard chi0 (open [-pi,pi]^3 mesh, |M|^2 = 1, 32 q along (100))",
             "fese": "FeSe-like 10-orbital dynamic chi0 (Gamma-M, explicit k+q, 512 w in [0,2] eV, E_F at 6/10)",
             "sweep": "40-band random model, static chi0, on-grid q with per-q band windows 4..40",
             "large": "80-band random model, dynamic chi0 (Re and Im), on-grid q, w in [0,2] eV, E_F at half filling"}
    nw = 1 if W.omega is None else len(W.omega)
    inb = sum((q.Cq.nbytes if q.Cq is not None else 0) + (q.Eq.nbytes if q.Eq is not None else 0) for q in W.qs)
    inb += W.E.nbytes + (W.C.nbytes if W.C is not None else 0)
    qs = "%d q" % len(W.qs)
    if "nq_total" in W.meta:
        qs = "q points 1..%d of its %d per step" % (len(W.qs), W.meta["nq_total"])
    ovl = overlap_mode(args)
    return {
        "workload": "%s: %s k mesh (%d tetrahedra), %d bands, %s, %d w" % (
            names[args.workload], "x".join(str(x) for x in W.n), W.ntet, W.nb, qs, nw),
        "ntet": W.ntet, "nbands": W.nb, "nq": len(W.qs), "nomega": nw,
        "nominal_evals_per_step": W.nominal_evals(),
        "evec_dtype": str(W.C.dtype) if W.C is not None else None,
        "overlap": {"fp32": "FP32 on the CUDA cores", "bf16x3": "tensor cores, BF16 2 pieces, 3 products",
                    "bf16x6": "tensor cores, BF16 3 pieces, 6 products", "tf32": "tensor cores, TF32"}[ovl],
        "l2": "inputs larger than L2 (%.1f GB of eigen-data read per step)" % (inb / 1e9),
    }


def tet_sample(W, count, seed):
    """A seeded sample of the builtin tetrahedra as an explicit list (corners, volumes)."""
    rng = np.random.default_rng(seed)
    ids = np.sort(rng.choice(W.ntet, size=min(count, W.ntet), replace=False))
    return wl.builtin_tetra(W.n, ids)


def sample_freqs(W, nw_sample):
    return np.unique(np.linspace(0, len(W.omega) - 1, nw_sample).round().astype(int))


def cpu_sample(W, nq_sample, nthreads, nw_sample=16, tets=None):
    """The oracle on a bounded sample.  With ``tets``: the first q of the step, those tetrahedra,
    nw_sample frequencies spread over the grid.  Without: q points 1 .. nq_sample (whole
    tetrahedron set; q 0 is Gamma on the paths), the first nw_sample frequencies (dynamic)."""
    import oracle
    oracle.build()
    if tets is not None:
        tet, vol = tets
        idx = sample_freqs(W, nw_sample)
        q = W.qs[0]
        t0 = time.perf_counter()
        vals = [oracle.chi0_q(W, q, omega=W.omega[idx], nthreads=nthreads, tet=tet, tvol=vol)]
        dt = time.perf_counter() - t0
        lo, hi = q.window or W.window
        return vals, dt, len(tet) * (hi - lo) ** 2 * len(idx)
    qs = W.qs[1:1 + nq_sample] if len(W.qs) > 1 else W.qs[:1]
    om = None if W.omega is None else W.omega[:nw_sample]
    t0 = time.perf_counter()
    vals = [oracle.chi0_q(W, q, omega=om, nthreads=nthreads) for q in qs]
    dt = time.perf_counter() - t0
    evals = sum(W.ntet * ((q.window or W.window)[1] - (q.window or W.window)[0]) ** 2 for q in qs) * (
        1 if om is None else len(om))
    return vals, dt, evals


# ------------------------------------------------------------------------------ clocks
class Clocks:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.idx = gpu_index
        self.p = None
        self.path = os.path.join(tempfile.gettempdir(), "chi0_bench_clocks_%d.csv" % os.getpid())

    def start(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.idx), "--query-gpu=" + self.QUERY,
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except Exception:
            self.p.kill()
        self.f.close()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() in ("active", "0x1") or v.lower().startswith("active"):
                    reasons.add(nm)
        try:
            os.remove(self.path)
        except OSError:
            pass
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        try:
            return json.load(open(p)), "measured"
        except Exception:
            pass
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


def arithmetic_peaks(chi0):
    """FP32 and FP64 FMA and tcgen05 TF32 / BF16 MMA throughput of this GPU, measured by the
    library's micro-kernels (chi0_peak) with CUDA events, before the timed region."""
    out = {}
    for name, kind, iters in (("fp32_fma_tflops", chi0.CHI0_PEAK_FP32_FMA, 20000),
                              ("fp64_fma_tflops", chi0.CHI0_PEAK_FP64_FMA, 300),
                              ("tf32_mma_tflops", chi0.CHI0_PEAK_TF32_MMA, 100000),
                              ("bf16_mma_tflops", chi0.CHI0_PEAK_BF16_MMA, 200000)):
        try:
            out[name] = chi0.chi0_peak(kind, iters)[0]
        except Exception as e:  # reported, not hidden
            out[name] = None
            out.setdefault("errors", []).append("%s: %s" % (name, e))
    out["source"] = "chi0_peak micro-kernels in this run (CUDA events, every SM busy)"
    return out


# Executed FP32 operations (FFMA counted twice, FADD, FMUL) per final tetrahedron of the mixed
# static weight kernels on the Cr-like 48^3 workload (ncu instruction counters of k_static +
# k_static_tab, before the long-series queue was compacted over the call: the same arithmetic
# per piece now runs in k_tab_eval).  Their DRAM bytes per final tetrahedron (3.58 then) are
# not reported: the kernels have changed since the counters were taken.
FLOPS_PER_PIECE_MIXED = 202.6
TRAFFIC_PER_PIECE_MIXED = None
# The same for the dynamic weight kernel per final tetrahedron over one pass of 256 frequencies
# (ncu instruction counters of k_dynamic on a seeded sample of 16384 tetrahedra of the 80-band
# 72^3 mesh, one q: the full mesh's mix of pieces; the FP64 kernel's FP64 operations likewise).
# DRAM bytes: not taken from the sample (its scattered tetrahedra defeat the caches that the
# whole mesh uses); on whole meshes they fall per final tetrahedron as the mesh grows (29.3 B at
# 24^3, 16.4 B at 48^3), so no per-unit figure scales to the 72^3 launch: None until counted there.
FLOPS_PER_PIECE_DYN32 = 2987.4
FLOPS_PER_PIECE_DYN64 = 6346.5
TRAFFIC_PER_PIECE_DYN32 = None


def run_step(P, W):
    """One pass of the whole path over the step's q points (static or dynamic)."""
    return P.static() if W.omega is None else P.dynamic(W.omega)


def to_host(out):
    if isinstance(out, tuple):
        return tuple(o.cpu().numpy() if hasattr(o, "cpu") else o for o in out)
    return out.cpu().numpy() if hasattr(out, "cpu") else out


def rel_err(a, b):
    """Normwise error per q (max over w of |a - b| / max over w of |b|), max over q; Re and Im
    separately for dynamic results (the larger of the two is returned)."""
    if isinstance(a, tuple):
        return max(rel_err(x, y) for x, y in zip(a, b))
    a = np.atleast_2d(np.asarray(a, dtype=np.float64).T).T if np.ndim(a) == 1 else np.asarray(a)
    b = np.atleast_2d(np.asarray(b, dtype=np.float64).T).T if np.ndim(b) == 1 else np.asarray(b)
    a = a.reshape(a.shape[0], -1)
    b = b.reshape(b.shape[0], -1)
    scale = np.max(np.abs(b), axis=1)
    scale = np.where(scale > 0, scale, 1.0)
    return float(np.max(np.max(np.abs(a - b), axis=1) / scale))


def sample_desc(args, W, tets, dt):
    if tets is not None:
        return ("q point 1 of the step, %d seeded tetrahedra of the %d-tetrahedron mesh, %d of the %d w, "
                "%.1f s" % (len(tets[0]), W.ntet, len(sample_freqs(W, args.cpu_sample_w)), len(W.omega), dt))
    return "q points 1..%d of the workload (all %d tetrahedra%s), %.1f s" % (
        args.cpu_sample_q, W.ntet, "" if W.omega is None else ", first %d w" % args.cpu_sample_w, dt)


# ------------------------------------------------------------------------------ main
def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    nproc = wl.default_nproc()
    W = make_workload(args, nproc)
    tets = None
    if args.workload == "large":
        tets = tet_sample(W, args.cpu_tets or 48, wl.SEED_BASE + 77)
        args.cpu_sample_w = min(args.cpu_sample_w, 8)
    if args.cpu_sample_q is None:
        args.cpu_sample_q = 2 if W.omega is None else 1
    cores = len(os.sched_getaffinity(0))
    times = []
    evals = 0
    for s in range(args.warmup + args.steps):
        _, dt, ev = cpu_sample(W, args.cpu_sample_q, cores, args.cpu_sample_w, tets)
        if s >= args.warmup:
            times.append(dt)
            evals = ev
    T = sum(times) / len(times)
    v = evals / T
    line = {"metric": METRIC, "value": v, "unit": "evals/s", "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": T * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": workload_config(W, args),
            "cpu_baseline": {"value": v, "unit": "evals/s", "cores": cores, "kind": "oracle",
                             "sample": sample_desc(args, W, tets, T)},
            "e2e": {"value": v, "unit": "evals/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def run_ours(args):
    ws, rank, local = dist_env()
    nproc = max(1, wl.default_nproc() // max(1, ws))
    ovl = overlap_mode(args)
    # inputs (and the oracle sample) before any CUDA call: the generator uses a spawn pool
    W = make_workload(args, nproc)
    tets = tet_sample(W, args.cpu_tets or 192, wl.SEED_BASE + 77) if args.workload == "large" else None
    if args.cpu_sample_q is None:
        args.cpu_sample_q = 8 if W.omega is None else 1
    cpu = None
    if rank == 0 and not args.no_cpu:
        cores = len(os.sched_getaffinity(0))
        vals, dt, ev = cpu_sample(W, args.cpu_sample_q, cores, args.cpu_sample_w, tets)
        cpu = {"value": ev / dt, "unit": "evals/s", "cores": cores, "kind": "oracle",
               "sample": sample_desc(args, W, tets, dt)}
        oracle_vals = vals
    import torch
    import torch.distributed as dist
    from paper_1407_3444_gb300 import chi0

    torch.cuda.set_device(local)
    if ws > 1:
        dist.init_process_group("nccl")

    def barrier():
        if ws > 1:
            dist.barrier()

    stream = torch.cuda.current_stream()
    peaks_run = arithmetic_peaks(chi0)
    dev = chi0.DeviceInputs(W)
    sub = tet_sample(W, args.tets, wl.SEED_BASE + 78) if args.tets else None
    Pm = chi0.Plan(W, precision="mixed", device=True, profile=True, staged=dev, overlap=ovl, tetra=sub)
    nominal = W.nominal_evals() * (len(sub[1]) / W.ntet if sub is not None else 1.0)
    tuned = None
    if args.workload == "large" and not args.tune:
        tuned = {"skipped": "the autotuner times one whole step per candidate launch shape (about a minute on "
                            "this run); --tune runs it"}
    elif not args.no_tune:  # untimed: picks the weight kernel's block shape and grid, and the
        tuned = Pm.tune(W.omega)  # tensor-core corner packing, on one call of the step
    for _ in range(args.warmup):
        run_step(Pm, W)
    torch.cuda.synchronize()
    s0 = Pm.stats()
    clocks = Clocks(local)
    clocks.start()
    barrier()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        out_m = run_step(Pm, W)
    e1.record(stream)
    torch.cuda.synchronize()
    barrier()
    ck = clocks.stop()
    ms = reduce_max(e0.elapsed_time(e1) / args.steps)
    s1 = Pm.stats()
    value = whole_job_rate(ws, nominal, ms)

    def stage_ms(s_a, s_b, k):
        n = s_b.launches[k] - s_a.launches[k]
        return (s_b.time_ms[k] - s_a.time_ms[k]) / n if n else None

    launches = s1.kernels - s0.kernels
    pieces_timed = s1.pieces - s0.pieces
    w_eval = 1.0 if W.omega is None else len(W.omega) / max(1, -(-len(W.omega) // chi0.DYNAMIC_MAX_NW))
    nonzero_rate = whole_job_rate(ws, pieces_timed / args.steps * w_eval, ms)
    stages = {name: stage_ms(s0, s1, k) for name, k in (
        ("overlap", chi0.CHI0_K_OVERLAP), ("weights", chi0.CHI0_K_STATIC), ("dynamic", chi0.CHI0_K_DYNAMIC),
        ("reduce", chi0.CHI0_K_REDUCE), ("bands", chi0.CHI0_K_BANDS), ("dos", chi0.CHI0_K_DOS))}
    counters = Pm.counters()
    counters_step = {"final_tetrahedra": pieces_timed // args.steps,
                     "box_pieces": (s1.box_pieces - s0.box_pieces) // args.steps,
                     "fp64_branch_evals": (s1.fp64_evals - s0.fp64_evals) // args.steps}
    mixed = to_host(out_m)

    # all-FP64 GPU form on the same resident inputs
    fp64 = None
    ms64 = None
    err_mixed = None
    dyn64_ms = None
    pieces64 = None
    if args.fp64_steps > 0:
        Pd = chi0.Plan(W, precision="fp64", device=True, profile=True, staged=dev, tetra=sub)
        torch.cuda.synchronize()
        d0 = Pd.stats()
        f0 = torch.cuda.Event(enable_timing=True)
        f1 = torch.cuda.Event(enable_timing=True)
        f0.record(stream)
        for _ in range(args.fp64_steps):
            out_d = run_step(Pd, W)
        f1.record(stream)
        torch.cuda.synchronize()
        d1 = Pd.stats()
        ms64 = f0.elapsed_time(f1) / args.fp64_steps
        fp64 = to_host(out_d)
        err_mixed = rel_err(mixed, fp64)
        dyn64_ms = stage_ms(d0, d1, chi0.CHI0_K_DYNAMIC if W.omega is not None else chi0.CHI0_K_STATIC)
        pieces64 = (d1.pieces - d0.pieces) / max(1, (d1.launches[chi0.CHI0_K_DYNAMIC if W.omega is not None
                                                                   else chi0.CHI0_K_STATIC]
                                                      - d0.launches[chi0.CHI0_K_DYNAMIC if W.omega is not None
                                                                    else chi0.CHI0_K_STATIC]))
        Pd.close()

    # the Kramers-Kronig route (Im alone on a uniform grid of the step's spacing that covers the
    # spectrum, Re by the transform), timed after the step's timed region, against the direct form
    kk = None
    if W.omega is not None and not args.no_kk and len(W.omega) > 1:
        du = float(W.omega[1] - W.omega[0])
        uniform = np.allclose(np.diff(W.omega), du, rtol=1e-9, atol=0) and W.omega[0] == 0.0
        if uniform:
            lo_w, hi_w = W.window
            span = float(W.E[:, hi_w - 1].max() - W.E[:, lo_w].min())
            nkk = int(np.ceil(span / du)) + 2
            wmax = (nkk - 1) * du
            Pm.dynamic_kk(wmax, nkk)
            torch.cuda.synchronize()
            k0 = torch.cuda.Event(enable_timing=True)
            k1 = torch.cuda.Event(enable_timing=True)
            k0.record(stream)
            rk, ik = Pm.dynamic_kk(wmax, nkk)
            k1.record(stream)
            torch.cuda.synchronize()
            kms = k0.elapsed_time(k1) / len(W.qs)
            nwo = len(W.omega)
            rk = rk.cpu().numpy()[:, :nwo]
            ik = ik.cpu().numpy()[:, :nwo]
            mre, mim = mixed
            kk = {"ms_per_q": kms, "direct_ms_per_q": ms / len(W.qs), "nkk": nkk, "wmax": wmax,
                  "passes": -(-nkk // chi0.DYNAMIC_MAX_NW),
                  "speedup_vs_direct": (ms / len(W.qs)) / kms,
                  "re_vs_direct": rel_err(rk, mre), "im_vs_direct": rel_err(ik, mim),
                  "note": "Im on u_j = j dw up to the largest band-pair energy of the window (the step's "
                          "spacing), Re by the transform of the piecewise-linear Im; the step's q"}

    # the GPU forms on the oracle's tetrahedron sample (large run): same q, same frequencies
    gpu_on_sample = None
    if tets is not None and cpu is not None:
        idx = sample_freqs(W, args.cpu_sample_w)
        gpu_on_sample = {}
        for prec in ("mixed", "fp64"):
            Ps = chi0.Plan(W, precision=prec, device=True, staged=dev, tetra=tets, qs=W.qs[:1],
                           overlap=ovl if prec == "mixed" else "fp32")
            re, im = Ps.dynamic(W.omega)
            gpu_on_sample[prec] = (re.cpu().numpy()[:, idx], im.cpu().numpy()[:, idx])
            Ps.close()

    # end to end through the public API with host buffers (pinned), copies inside
    e2e = None
    if args.e2e_steps > 0:
        # the plan is built, and called once on a staged set, in untimed steps.  The K timed
        # steps then run as a pipeline: the region opens with the staging of step 1's
        # eigen-data from pinned host memory (chi0_plan_stage: the H2D copies, on the plan's
        # copy stream), and each step stages the next step's data (but the last) before its
        # own call, which takes its staged set, computes and reads the results back.  Every
        # step's copies lie inside the region; all but the first run alongside the previous
        # step's kernels.
        host = chi0.HostInputs(W, pinned=True)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        Ph = chi0.Plan(W, precision="mixed", device=False, staged=host, overlap=ovl, tetra=sub)
        torch.cuda.synchronize()
        plan_ms = (time.perf_counter() - t0) * 1e3
        Ph.stage(host)  # (allocates the plan's second set of eigen-data buffers)
        run_step(Ph, W)
        K = args.e2e_steps
        t_stage = t_call = 0.0
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        Ph.stage(host)
        for s in range(K):
            ta = time.perf_counter()
            if s + 1 < K:
                Ph.stage(host)
            tb = time.perf_counter()
            out_h = run_step(Ph, W)
            t_stage += tb - ta
            t_call += time.perf_counter() - tb
        torch.cuda.synchronize()
        T = (time.perf_counter() - t0) / K
        Ph.close()
        e2e = {"value": nominal / T, "unit": "evals/s", "h2d_bytes_per_step": host.nbytes(),
               "d2h_bytes_per_step": int(sum(o.nbytes for o in out_h) if isinstance(out_h, tuple) else out_h.nbytes),
               "ms_per_step": T * 1e3, "steps": K, "rel_diff_vs_device": rel_err(out_h, mixed),
               "ms_stage_call": [t_stage / K * 1e3, t_call / K * 1e3], "plan_ms_untimed": plan_ms,
               "api": "chi0_plan and one call (untimed), then chi0_plan_stage (host eigen-data of step 1) "
                      "and per step chi0_plan_stage (step i + 1) + chi0_dynamic/chi0_static (step i, "
                      "host results)"}
        del host

    peaks, kind = measured_peaks()
    sms = torch.cuda.get_device_properties(local).multi_processor_count
    fp32_pk = peaks_run.get("fp32_fma_tflops")
    fp64_pk = peaks_run.get("fp64_fma_tflops")
    if W.omega is None:
        k_ms = stage_ms(s0, s1, chi0.CHI0_K_STATIC)
        launches_w = s1.launches[chi0.CHI0_K_STATIC] - s0.launches[chi0.CHI0_K_STATIC]
        fpu, tpu, kname = (FLOPS_PER_PIECE_MIXED if args.workload == "cr" else None,
                           TRAFFIC_PER_PIECE_MIXED if args.workload == "cr" else None,
                           "static weights (k_static + k_static_tab, mixed)")
        uname = "final tetrahedron"
    else:
        k_ms = stage_ms(s0, s1, chi0.CHI0_K_DYNAMIC)
        launches_w = s1.launches[chi0.CHI0_K_DYNAMIC] - s0.launches[chi0.CHI0_K_DYNAMIC]
        at72 = args.workload == "large" and (args.n or 72) == 72
        fpu, tpu, kname = (FLOPS_PER_PIECE_DYN32 if at72 else None,
                           TRAFFIC_PER_PIECE_DYN32 if at72 else None,
                           "dynamic weights (k_dynamic + box sums/evaluation, mixed)")
        uname = "final tetrahedron over a pass of <= 256 w"
    units = pieces_timed / max(1, launches_w)
    ach = fpu * units / (k_ms * 1e-3) / 1e12 if (fpu and k_ms) else None
    roof = {"bound": "alu", "achieved": ach, "peak": fp32_pk, "unit": "TFLOP/s",
            "frac": ach / fp32_pk if (ach is not None and fp32_pk) else None,
            "traffic": tpu * units if tpu else None, "kernel": kname, "kernel_ms": k_ms,
            "units_per_launch": units, "unit_name": uname, "flops_per_unit": fpu,
            "final_tetrahedra_per_s_per_sm": units / (k_ms * 1e-3) / sms if k_ms else None,
            "peak_source": "measured FP32 FMA peak of this GPU (chi0_peak, this run)"}
    roof64 = None
    if dyn64_ms and pieces64:
        f64 = FLOPS_PER_PIECE_DYN64 if (W.omega is not None and args.workload == "large"
                                        and (args.n or 72) == 72) else None
        a64 = f64 * pieces64 / (dyn64_ms * 1e-3) / 1e12 if f64 else None
        roof64 = {"bound": "alu", "achieved": a64, "peak": fp64_pk, "unit": "TFLOP/s (FP64)",
                  "frac": a64 / fp64_pk if (a64 is not None and fp64_pk) else None,
                  "kernel_ms": dyn64_ms, "units_per_launch": pieces64, "flops_per_unit": f64,
                  "peak_source": "measured FP64 FMA peak of this GPU (chi0_peak, this run)"}
    # the overlap kernel: HBM bytes (eigenvector blocks at k and k+q read, |M|^2 written) and the
    # tensor-core products (8 w^2 norb flops per corner for the complex GEMM, times the products
    # of the split form)
    ovl_ms = stages["overlap"]
    ovl_roof = None
    if ovl_ms and W.C is not None:
        nc, no = W.ncorner, W.norb
        lo, hi = W.qs[0].window or W.window
        w = hi - lo
        kq = W.qs[0].Cq.itemsize if W.qs[0].Cq is not None else 8
        ovl_bytes = nc * no * w * (8 + kq) + nc * w * w * 4
        prods = {"bf16x6": 6, "bf16x3": 3, "tf32": 1, "fp32": 0}[ovl]
        tflop = 8.0 * w * w * no * nc * prods / (ovl_ms * 1e-3) / 1e12 if prods else None
        tpk = peaks_run.get("tf32_mma_tflops" if ovl == "tf32" else "bf16_mma_tflops")
        ovl_roof = {"bound": "hbm", "achieved": ovl_bytes / (ovl_ms * 1e-3) / 1e9,
                    "peak": float(peaks.get("hbm_gbs", 6800.0)), "unit": "GB/s", "bytes_per_launch": ovl_bytes,
                    "kernel_ms": ovl_ms, "kernel": "k_overlap_tc" if prods else "k_overlap_small / k_overlap",
                    "tensor_tflops": tflop, "tensor_peak_tflops": tpk,
                    "tensor_frac": tflop / tpk if (tflop and tpk) else None}
        ovl_roof["frac"] = ovl_roof["achieved"] / ovl_roof["peak"]

    if rank == 0:
        err_oracle = None
        if cpu is not None:
            if tets is not None:
                ref = tuple(np.asarray(oracle_vals[0][k])[None, :] for k in (0, 1))
                err_oracle = {"mixed_gpu": rel_err(gpu_on_sample["mixed"], ref),
                              "fp64_gpu": rel_err(gpu_on_sample["fp64"], ref),
                              "sample": "the cpu_baseline sample (explicit tetrahedron list, same q, same w)"}
            else:
                nq = len(oracle_vals)
                i0 = 1 if len(W.qs) > 1 else 0

                def sample(x):
                    if isinstance(x, tuple):
                        return tuple(y[i0:i0 + nq, :args.cpu_sample_w] for y in x)
                    return x[i0:i0 + nq]

                ref = (tuple(np.array([v[k] for v in oracle_vals]) for k in (0, 1))
                       if W.omega is not None else np.array(oracle_vals))
                err_oracle = {"mixed_gpu": rel_err(sample(mixed), ref), "q_points": nq}
                if fp64 is not None:
                    err_oracle["fp64_gpu"] = rel_err(sample(fp64), ref)
        dtype = "f32+f64" if ovl == "fp32" else "%s+f32+f64" % ovl
        line = {"metric": METRIC, "value": value, "unit": "evals/s", "n_gpus": ws, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": dtype, "data": "synthetic",
                "config": dict(workload_config(W, args), **({"tetra_sample": len(sub[1])} if sub is not None else {})),
                "fp64_gpu": ({"value": nominal / (ms64 * 1e-3), "unit": "evals/s", "ms_per_step": ms64,
                              "mixed_speedup": ms64 / ms} if ms64 else None),
                "error": {"mixed_vs_fp64_gpu_max_rel": err_mixed, "vs_oracle": err_oracle},
                "roofline": roof, "roofline_fp64": roof64, "roofline_overlap": ovl_roof,
                "stage_ms_per_q": stages, "peaks_run": peaks_run, "kk_route": kk,
                "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": int(launches), "tuned": tuned,
                "nonzero": {"value": nonzero_rate, "unit": "(final tetrahedron, w) evaluations/s"},
                "counters_per_step": counters_step, "counters": counters, "clocks": ck, "peaks_source": kind}
        print(json.dumps(line), flush=True)
        if args.profile_out:
            with open(args.profile_out, "w") as f:
                json.dump(line, f, indent=1)
    Pm.close()
    if ws > 1:
        dist.destroy_process_group()
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
