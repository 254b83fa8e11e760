"""Benchmark: chi0 (tetra x band-pair x q x omega) evals/s on one GB300.

Default workload: the Cr-like 9-orbital static run (48^3 k mesh, 663,552 tetrahedra,
9 bands, 256 q on Gamma-X-M-Gamma with explicit k+q eigen-data).  One step = chi0
for all 256 q through the C-ABI, every stage (overlaps, carving + weights, reduction)
in the CUDA library.  ``value`` is the mixed-precision form with inputs resident in
HBM; the all-FP64 GPU form is timed on the same inputs and reported beside it with
the normwise error between the two, and the FP64 CPU oracle is timed on a bounded
sample of the same workload (``cpu_baseline``).

``--impl reference`` times the oracle alone (host cores) on the same metric.
Under torchrun every rank runs its own replica of the workload (independent q sets:
no data-path collective); rank 0 prints the JSON line.
"""
from __future__ import annotations

import argparse
import json
import math
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


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-tune", action="store_true",
                    help="skip chi0_tune (launch-shape autotuner) before the warm-up steps")
    ap.add_argument("--overlap", default="fp32", choices=["fp32", "bf16x3", "bf16x6", "tf32"],
                    help="matrix elements of the mixed form: FP32 on the CUDA cores (default) or the "
                         "tensor cores (BF16 split in two pieces / three pieces, or one TF32 product)")
    ap.add_argument("--workload", default="cr", choices=["cr", "free", "fese", "sweep", "large"],
                    help="cr: Cr-like 9-orbital static (default); free: free-electron Lindhard; fese: "
                         "FeSe-like dynamic; sweep: 40-band window sweep (static); large: 80-band 72^3 dynamic")
    ap.add_argument("--nw", type=int, default=0,
                    help="dynamic workloads: use the first NW frequencies of the workload's grid "
                         "(a bounded sample of the 80-band 72^3 run)")
    ap.add_argument("--nq", type=int, default=None, help="q points per step (default: the workload's)")
    ap.add_argument("--n", type=int, default=None, help="k mesh cubes per axis (cubic workloads)")
    ap.add_argument("--cpu-sample-w", type=int, default=16, help="frequencies in the CPU sample (dynamic)")
    ap.add_argument("--fp64-steps", type=int, default=2)
    ap.add_argument("--e2e-steps", type=int, default=2)
    ap.add_argument("--cpu-sample-q", type=int, default=None,
                    help="q points of the oracle's timed sample (default: static workloads 8 for the "
                         "cpu_baseline, ~10-15 s on 16 cores, and 2 per --impl reference step; dynamic 1)")
    ap.add_argument("--no-cpu", action="store_true")
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
        return wl.fese_like(n=n, nq=64, nproc=nproc,
                            qfracs=[np.array([0.5, 0.5, 0.0]) * (j + 1) / 64 for j in range(64)][:nq])
    if k == "sweep":
        W = wl.band_sweep(n=args.n or 32, nq=args.nq or 128, nproc=nproc)
        W.omega = None  # the static sweep (the dynamic one: chi0_dynamic on the same plan)
        return W
    W = wl.large_mixed(n=args.n or 72, nq=args.nq or 128, nproc=nproc)
    if args.nw:
        W.omega = W.omega[:args.nw]
    return W


def workload_config(W, args):
    names = {"cr": "Cr-like 9-orbital static chi0 (Gamma-X-M-Gamma, explicit k+q eigen-data, E_F at 6/9)",
             "free": "free-electron static Lindhard chi0 (open [-pi,pi]^3 mesh, |M|^2 = 1, 32 q along (100))",
             "fese": "FeSe-like 10-orbital dynamic chi0 (Gamma-M, explicit k+q, 512 w in [0,2] eV, E_F at 6/10)",
             "sweep": "40-band random model, static chi0, on-grid q with per-q band windows 4..40",
             "large": "80-band random model, dynamic chi0, on-grid q, 256 w in [0,2] eV"}
    nw = 1 if W.omega is None else len(W.omega)
    inb = sum((q.Cq.nbytes if q.Cq is not None else 0) + (q.Eq.nbytes if q.Eq is not None else 0) for q in W.qs)
    inb += W.E.nbytes + (W.C.nbytes if W.C is not None else 0)
    return {
        "workload": "%s: %s k mesh (%d tetrahedra), %d bands, %d q, %d w" % (
            names[args.workload], "x".join(str(x) for x in W.n), W.ntet, W.nb, len(W.qs), nw),
        "ntet": W.ntet, "nbands": W.nb, "nq": len(W.qs), "nomega": nw,
        "nominal_evals_per_step": W.nominal_evals(),
        "evec_dtype": str(W.C.dtype) if W.C is not None else None,
        "overlap": {"fp32": "FP32 on the CUDA cores", "bf16x3": "tensor cores, BF16 2 pieces, 3 products",
                    "bf16x6": "tensor cores, BF16 3 pieces, 6 products", "tf32": "tensor cores, TF32"}[args.overlap],
        "l2": "inputs larger than L2 (%.1f GB of eigen-data read per step)" % (inb / 1e9),
    }


def cpu_sample(W, nq_sample, nthreads, nw_sample=16):
    """Oracle on q points 1 .. nq_sample (whole tetrahedron set; q 0 is Gamma on the paths);
    dynamic workloads: the first nw_sample frequencies."""
    import oracle
    oracle.build()
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


# FP32 FMA lanes: 152 SMs x 128 lanes x 2 flop per FMA at the maximum SM clock
def fp32_peak_tflops(sm_mhz):
    return 152 * 128 * 2 * sm_mhz * 1e6 / 1e12


# FP32 operations (FFMA counted twice, FADD, FMUL) of the mixed static weight kernels per
# final tetrahedron on the Cr-like 48^3 workload, from ncu's instruction counters of
# k_static + k_static_tab (one q of an 8-q run, 13.65 M final tetrahedra per launch); and
# their DRAM bytes per final tetrahedron.
FLOPS_PER_PIECE_MIXED = 202.6
TRAFFIC_PER_PIECE_MIXED = 3.58
# The same for k_dynamic per (final tetrahedron, frequency) on the FeSe-like model (ncu
# counters of the four k_dynamic launches of one step on its 32x32x8 mesh, 2 q x 512 w:
# 1.40 M final tetrahedra x 256 w per launch).
FLOPS_PER_PIECE_W_DYN = 169.3
TRAFFIC_PER_PIECE_W_DYN = None  # counted (0.0139 B) on the kernel before its piece buffering


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


# ------------------------------------------------------------------------------ main
def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    nproc = wl.default_nproc()
    W = make_workload(args, nproc)
    if args.cpu_sample_q is None:
        args.cpu_sample_q = 2 if W.omega is None else 1
    cores = len(os.sched_getaffinity(0))
    times = []
    evals = 0
    for s in range(args.warmup + args.steps):
        _, dt, ev = cpu_sample(W, args.cpu_sample_q, cores, args.cpu_sample_w)
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
                             "sample": "q points 1..%d of the workload, all tetrahedra%s" % (
                                 args.cpu_sample_q, "" if W.omega is None else ", first %d w" % args.cpu_sample_w)},
            "e2e": {"value": v, "unit": "evals/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def run_ours(args):
    ws, rank, local = dist_env()
    nproc = max(1, wl.default_nproc() // max(1, ws))
    # inputs (and the oracle sample) before any CUDA call: the generator uses a spawn pool
    W = make_workload(args, nproc)
    if args.cpu_sample_q is None:
        args.cpu_sample_q = 8 if W.omega is None else 1
    cpu = None
    if rank == 0 and not args.no_cpu:
        cores = len(os.sched_getaffinity(0))
        vals, dt, ev = cpu_sample(W, args.cpu_sample_q, cores, args.cpu_sample_w)
        cpu = {"value": ev / dt, "unit": "evals/s", "cores": cores, "kind": "oracle",
               "sample": "q points 1..%d of the workload (all %d tetrahedra%s), %.1f s"
                         % (args.cpu_sample_q, W.ntet, "" if W.omega is None else ", first %d w" % args.cpu_sample_w,
                            dt)}
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
    dev = chi0.DeviceInputs(W)
    Pm = chi0.Plan(W, precision="mixed", device=True, profile=True, staged=dev, overlap=args.overlap)
    Pd = chi0.Plan(W, precision="fp64", device=True, profile=False, staged=dev) if args.fp64_steps > 0 else None
    nominal = W.nominal_evals()
    tuned = None
    if not args.no_tune:  # untimed: picks the weight kernel's block shape and grid, and the
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
    def stage_ms(k):
        n = s1.launches[k] - s0.launches[k]
        return (s1.time_ms[k] - s0.time_ms[k]) / n if n else None

    k_static_ms = stage_ms(chi0.CHI0_K_STATIC)
    launches = s1.kernels - s0.kernels
    pieces_timed = s1.pieces - s0.pieces
    # non-empty work: final tetrahedra times the frequencies each is evaluated on, per second
    w_eval = 1.0 if W.omega is None else len(W.omega) / max(1, -(-len(W.omega) // chi0.DYNAMIC_MAX_NW))
    nonzero_rate = whole_job_rate(ws, pieces_timed / args.steps * w_eval, ms)
    static_launches = s1.launches[chi0.CHI0_K_STATIC] - s0.launches[chi0.CHI0_K_STATIC]
    stages = {name: stage_ms(k) for name, k in (("overlap", chi0.CHI0_K_OVERLAP), ("weights", chi0.CHI0_K_STATIC),
                                                 ("dynamic", chi0.CHI0_K_DYNAMIC),
                                                 ("reduce", chi0.CHI0_K_REDUCE), ("bands", chi0.CHI0_K_BANDS),
                                                 ("dos", chi0.CHI0_K_DOS))}
    counters = Pm.counters()
    mixed = to_host(out_m)

    # all-FP64 GPU form on the same resident inputs
    fp64 = None
    ms64 = None
    err_mixed = None
    if Pd is not None:
        run_step(Pd, W)
        torch.cuda.synchronize()
        f0 = torch.cuda.Event(enable_timing=True)
        f1 = torch.cuda.Event(enable_timing=True)
        f0.record(stream)
        for _ in range(args.fp64_steps):
            out_d = run_step(Pd, W)
        f1.record(stream)
        torch.cuda.synchronize()
        ms64 = f0.elapsed_time(f1) / args.fp64_steps
        fp64 = to_host(out_d)
        err_mixed = rel_err(mixed, fp64)

    # end to end through the public API with host buffers (pinned), copies inside
    e2e = None
    if args.e2e_steps > 0:
        host = chi0.HostInputs(W, pinned=True)
        t_e2e = []
        for s in range(args.e2e_steps + 1):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            Ph = chi0.Plan(W, precision="mixed", device=False, staged=host)
            out_h = run_step(Ph, W)
            Ph.close()
            t1 = time.perf_counter()
            if s > 0:
                t_e2e.append(t1 - t0)
        T = sum(t_e2e) / len(t_e2e)
        e2e = {"value": nominal / T, "unit": "evals/s", "h2d_bytes_per_step": host.nbytes(),
               "d2h_bytes_per_step": int(sum(o.nbytes for o in out_h) if isinstance(out_h, tuple) else out_h.nbytes),
               "ms_per_step": T * 1e3, "rel_diff_vs_device": rel_err(out_h, mixed)}
        del host

    peaks, kind = measured_peaks()
    smax = float(peaks.get("sm_max_mhz", 2070.0))
    pk = fp32_peak_tflops(smax)
    peak_src = "derived: 152 SMs x 128 FP32 lanes x 2 flop x %.0f MHz (max SM clock)" % smax
    if W.omega is None:
        pieces_per_launch = pieces_timed / max(1, static_launches)
        ach = (FLOPS_PER_PIECE_MIXED * pieces_per_launch / (k_static_ms * 1e-3) / 1e12
               if k_static_ms and args.workload == "cr" else None)
        roof = {"bound": "alu", "achieved": ach, "peak": pk, "unit": "TFLOP/s",
                "frac": ach / pk if ach is not None else None,
                "traffic": (TRAFFIC_PER_PIECE_MIXED * pieces_per_launch
                            if TRAFFIC_PER_PIECE_MIXED and args.workload == "cr" else None),
                "kernel": "static weights (k_static + k_static_tab, mixed)",
                "kernel_ms": k_static_ms, "units_per_launch": pieces_per_launch,
                "flops_per_unit": FLOPS_PER_PIECE_MIXED, "unit_name": "final tetrahedron",
                "peak_source": peak_src}
    else:
        # k_dynamic: one launch = one pass of <= 256 frequencies over every final tetrahedron
        dyn_launches = s1.launches[chi0.CHI0_K_DYNAMIC] - s0.launches[chi0.CHI0_K_DYNAMIC]
        k_dyn_ms = stage_ms(chi0.CHI0_K_DYNAMIC)
        pieces_per_launch = pieces_timed / max(1, dyn_launches)
        w_per_launch = len(W.omega) / max(1, -(-len(W.omega) // chi0.DYNAMIC_MAX_NW))
        units = pieces_per_launch * w_per_launch
        ach = (FLOPS_PER_PIECE_W_DYN * units / (k_dyn_ms * 1e-3) / 1e12
               if k_dyn_ms and FLOPS_PER_PIECE_W_DYN and args.workload == "fese" else None)
        roof = {"bound": "alu", "achieved": ach, "peak": pk, "unit": "TFLOP/s",
                "frac": ach / pk if ach is not None else None,
                "traffic": (TRAFFIC_PER_PIECE_W_DYN * units
                            if TRAFFIC_PER_PIECE_W_DYN and args.workload == "fese" else None),
                "kernel": "dynamic weights (k_dynamic, mixed)",
                "kernel_ms": k_dyn_ms, "units_per_launch": units,
                "flops_per_unit": FLOPS_PER_PIECE_W_DYN, "unit_name": "(final tetrahedron, w)",
                "peak_source": peak_src}
    # the overlap kernel is bound by HBM: eigenvector blocks at k (complex64 copy) and at k+q
    # (complex128 inputs) read once, |M|^2 written once
    ovl_ms = stages["overlap"]
    ovl = None
    if ovl_ms and W.C is not None:
        nc, no, w = W.ncorner, W.norb, W.nb
        kq = W.qs[0].Cq.itemsize if W.qs[0].Cq is not None else 8
        ovl_bytes = nc * no * w * (8 + kq) + nc * w * w * 4
        ovl = {"bound": "hbm", "achieved": ovl_bytes / (ovl_ms * 1e-3) / 1e9, "peak": float(peaks.get("hbm_gbs", 6800.0)),
               "unit": "GB/s", "bytes_per_launch": ovl_bytes, "kernel_ms": ovl_ms}
        ovl["frac"] = ovl["achieved"] / ovl["peak"]

    if rank == 0:
        err_oracle = None
        if cpu is not None:
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
        line = {"metric": METRIC, "value": value, "unit": "evals/s", "n_gpus": ws, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
                "config": workload_config(W, args),
                "fp64_gpu": ({"value": nominal / (ms64 * 1e-3), "unit": "evals/s", "ms_per_step": ms64,
                              "mixed_speedup": ms64 / ms} if ms64 else None),
                "error": {"mixed_vs_fp64_gpu_max_rel": err_mixed, "vs_oracle": err_oracle},
                "roofline": roof, "roofline_overlap": ovl, "stage_ms_per_q": stages,
                "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": int(launches), "tuned": tuned,
                "nonzero": {"value": nonzero_rate, "unit": "(final tetrahedron, w) evaluations/s"},
                "counters": counters, "clocks": ck, "peaks_source": kind}
        print(json.dumps(line), flush=True)
        if args.profile_out:
            with open(args.profile_out, "w") as f:
                json.dump(line, f, indent=1)
    Pm.close()
    if Pd is not None:
        Pd.close()
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
