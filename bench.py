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
    ap.add_argument("--nq", type=int, default=256)
    ap.add_argument("--n", type=int, default=48)
    ap.add_argument("--fp64-steps", type=int, default=2)
    ap.add_argument("--e2e-steps", type=int, default=2)
    ap.add_argument("--cpu-sample-q", type=int, default=1)
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--profile-out", default="")
    return ap.parse_args()


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def make_workload(args, nproc):
    return wl.cr_like(n=args.n, nq=args.nq, nproc=nproc)


def workload_config(W, args):
    return {
        "workload": "Cr-like 9-orbital static chi0: %d^3 k mesh (%d tetrahedra), 9 bands, %d q on "
                    "Gamma-X-M-Gamma with explicit k+q eigen-data, E_F at 6/9 filling" % (args.n, W.ntet, len(W.qs)),
        "ntet": W.ntet, "nbands": W.nb, "nq": len(W.qs), "nomega": 1,
        "nominal_evals_per_step": W.nominal_evals(),
        "evec_dtype": str(W.C.dtype),
        "l2": "inputs larger than L2 (explicit k+q eigen-data %.1f GB per step)" % (
            sum(q.Cq.nbytes + q.Eq.nbytes for q in W.qs) / 1e9),
    }


def cpu_sample(W, nq_sample, nthreads):
    """Oracle on q points 1 .. nq_sample (whole tetrahedron set; q 0 is Gamma)."""
    import oracle
    oracle.build()
    t0 = time.perf_counter()
    vals = [oracle.chi0_q(W, q, nthreads=nthreads) for q in W.qs[1:1 + nq_sample]]
    dt = time.perf_counter() - t0
    evals = W.ntet * (W.window[1] - W.window[0]) ** 2 * nq_sample
    return np.array(vals), dt, evals


# ------------------------------------------------------------------------------ clocks
class Clocks:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.idx = gpu_index
        self.p = None
        self.path = os.path.join(ROOT, "gpurun_out", "bench_clocks_%d.csv" % os.getpid())

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
# final tetrahedron on this workload, from the ncu instruction counters of
# profiles/static_weights_cr_like_48.md; and their DRAM bytes per final tetrahedron.
FLOPS_PER_PIECE_MIXED = 207.0
TRAFFIC_PER_PIECE_MIXED = None


# ------------------------------------------------------------------------------ main
def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    nproc = wl.default_nproc()
    W = make_workload(args, nproc)
    cores = len(os.sched_getaffinity(0))
    times = []
    evals = 0
    for s in range(args.warmup + args.steps):
        _, dt, ev = cpu_sample(W, args.cpu_sample_q, cores)
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
                             "sample": "q points 1..%d of the workload, all tetrahedra" % args.cpu_sample_q},
            "e2e": {"value": v, "unit": "evals/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def run_ours(args):
    ws, rank, local = dist_env()
    nproc = max(1, wl.default_nproc() // max(1, ws))
    # inputs (and the oracle sample) before any CUDA call: the generator uses a spawn pool
    W = make_workload(args, nproc)
    cpu = None
    if rank == 0 and not args.no_cpu:
        cores = len(os.sched_getaffinity(0))
        vals, dt, ev = cpu_sample(W, args.cpu_sample_q, cores)
        cpu = {"value": ev / dt, "unit": "evals/s", "cores": cores, "kind": "oracle",
               "sample": "q points 1..%d of the workload (all %d tetrahedra, 81 pairs), %.1f s"
                         % (args.cpu_sample_q, W.ntet, dt)}
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
    Pm = chi0.Plan(W, precision="mixed", device=True, profile=True, staged=dev)
    Pd = chi0.Plan(W, precision="fp64", device=True, profile=False, staged=dev) if args.fp64_steps > 0 else None
    nominal = W.nominal_evals()
    for _ in range(args.warmup):
        Pm.static()
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
        out_m = Pm.static()
    e1.record(stream)
    torch.cuda.synchronize()
    barrier()
    ck = clocks.stop()
    ms = e0.elapsed_time(e1) / args.steps
    if ws > 1:
        t = torch.tensor([ms], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    s1 = Pm.stats()
    value = ws * nominal / (ms * 1e-3)
    def stage_ms(k):
        n = s1.launches[k] - s0.launches[k]
        return (s1.time_ms[k] - s0.time_ms[k]) / n if n else None

    k_static_ms = stage_ms(chi0.CHI0_K_STATIC)
    launches = s1.kernels - s0.kernels
    pieces_timed = s1.pieces - s0.pieces
    static_launches = s1.launches[chi0.CHI0_K_STATIC] - s0.launches[chi0.CHI0_K_STATIC]
    stages = {name: stage_ms(k) for name, k in (("overlap", chi0.CHI0_K_OVERLAP), ("weights", chi0.CHI0_K_STATIC),
                                                 ("reduce", chi0.CHI0_K_REDUCE), ("bands", chi0.CHI0_K_BANDS),
                                                 ("dos", chi0.CHI0_K_DOS))}
    counters = Pm.counters()
    mixed = out_m.cpu().numpy()

    # all-FP64 GPU form on the same resident inputs
    fp64 = None
    ms64 = None
    err_mixed = None
    if Pd is not None:
        Pd.static()
        torch.cuda.synchronize()
        f0 = torch.cuda.Event(enable_timing=True)
        f1 = torch.cuda.Event(enable_timing=True)
        f0.record(stream)
        for _ in range(args.fp64_steps):
            out_d = Pd.static()
        f1.record(stream)
        torch.cuda.synchronize()
        ms64 = f0.elapsed_time(f1) / args.fp64_steps
        fp64 = out_d.cpu().numpy()
        err_mixed = float(np.max(np.abs(mixed - fp64) / np.abs(fp64)))

    # end to end through the public API with host buffers (pinned), copies inside
    e2e = None
    if args.e2e_steps > 0:
        host = chi0.HostInputs(W, pinned=True)
        t_e2e = []
        for s in range(args.e2e_steps + 1):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            Ph = chi0.Plan(W, precision="mixed", device=False, staged=host)
            out_h = Ph.static()
            Ph.close()
            t1 = time.perf_counter()
            if s > 0:
                t_e2e.append(t1 - t0)
        T = sum(t_e2e) / len(t_e2e)
        e2e = {"value": nominal / T, "unit": "evals/s", "h2d_bytes_per_step": host.nbytes(),
               "d2h_bytes_per_step": int(out_h.nbytes), "ms_per_step": T * 1e3,
               "max_abs_diff_vs_device": float(np.max(np.abs(out_h - mixed)))}
        del host

    peaks, kind = measured_peaks()
    smax = float(peaks.get("sm_max_mhz", 2070.0))
    pieces_per_launch = pieces_timed / max(1, static_launches)
    pk = fp32_peak_tflops(smax)
    ach = FLOPS_PER_PIECE_MIXED * pieces_per_launch / (k_static_ms * 1e-3) / 1e12 if k_static_ms else None
    roof = {"bound": "alu", "achieved": ach, "peak": pk, "unit": "TFLOP/s",
            "frac": ach / pk if ach is not None else None,
            "traffic": TRAFFIC_PER_PIECE_MIXED * pieces_per_launch if TRAFFIC_PER_PIECE_MIXED else None,
            "kernel": "static weights (k_static + k_static_f64 + k_static_tab, mixed)",
            "kernel_ms": k_static_ms, "units_per_launch": pieces_per_launch,
            "flops_per_unit": FLOPS_PER_PIECE_MIXED, "unit_name": "final tetrahedron",
            "peak_source": "derived: 152 SMs x 128 FP32 lanes x 2 flop x %.0f MHz (max SM clock)" % smax}
    # the overlap kernel is bound by HBM: eigenvector blocks at k (complex64 copy) and at k+q
    # (complex128 inputs) read once, |M|^2 written once
    ovl_ms = stages["overlap"]
    ovl = None
    if ovl_ms:
        nc, no, w = W.ncorner, W.norb, W.nb
        ovl_bytes = nc * no * w * (8 + 16) + nc * w * w * 4
        ovl = {"bound": "hbm", "achieved": ovl_bytes / (ovl_ms * 1e-3) / 1e9, "peak": float(peaks.get("hbm_gbs", 6800.0)),
               "unit": "GB/s", "bytes_per_launch": ovl_bytes, "kernel_ms": ovl_ms}
        ovl["frac"] = ovl["achieved"] / ovl["peak"]

    if rank == 0:
        err_oracle = None
        if cpu is not None:
            nq = len(oracle_vals)
            err_oracle = {"mixed_gpu": float(np.max(np.abs(mixed[1:1 + nq] - oracle_vals) / np.abs(oracle_vals))),
                          "q_points": nq}
            if fp64 is not None:
                err_oracle["fp64_gpu"] = float(np.max(np.abs(fp64[1:1 + nq] - oracle_vals) / np.abs(oracle_vals)))
        line = {"metric": METRIC, "value": value, "unit": "evals/s", "n_gpus": ws, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
                "config": workload_config(W, args),
                "fp64_gpu": ({"value": nominal / (ms64 * 1e-3), "unit": "evals/s", "ms_per_step": ms64,
                              "mixed_speedup": ms64 / ms} if ms64 else None),
                "error": {"mixed_vs_fp64_gpu_max_rel": err_mixed, "vs_oracle": err_oracle},
                "roofline": roof, "roofline_overlap": ovl, "stage_ms_per_q": stages,
                "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": int(launches),
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
