"""Benchmark: histories/s of the transport hot path on one B300 (or N, weak
scaling with disjoint history ranges per rank), printed as one JSON line.

Default workload: the 20 cm two-region time-dependent slab (1e7 histories,
50 time bins x 200 spatial bins, one group), FP32 flights with position and
time kept exact in FP64 where they cross a cell face or a census edge (FP32
offsets from those in between) and an FP64 tally reduction; the variant with
FP64 position and time accumulated every flight is reported beside it.  A
step is one full run (every history of the
workload through source, flights, tally, collisions and the batch
statistics).  Inputs (problem tables) are resident in HBM before timing; the
per-step L2 flush writes a 256 MiB buffer.

``--impl reference`` times the CPU oracle (FP64, all host cores) on a bounded
sample of the same workload and prints the same line with "impl": "reference".
"""
import argparse
import hashlib
import json
import math
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2409_04668_b300 import workloads as W  # noqa: E402

METRIC = "histories/sec and tally figure of merit (1/sigma^2 T), 1 B300"
WORKLOADS = {
    "c1": (W.c1_slab, 100_000),
    "c2": (W.c2_two_region, 10_000_000),
    "c3": (W.c3_channel, 100_000_000),
    "c4": (W.c4_deep, 100_000_000),
    "c5": (None, 0),          # 256 independent problems in one batched run
}


def history_offset(rank, step, n_hist, max_steps=1000):
    """First history id a rank runs at a step: every rank owns a disjoint
    block of max_steps consecutive runs, so ranks never repeat a history and
    the union over ranks is as many independent histories as one long run."""
    return (rank * max_steps + step) * n_hist


def job_value(local_ms, n_hist, steps, world, reduce_max=None):
    """Whole-job histories/s: all ranks' histories over the slowest rank's
    time (reduce_max(x) returns the maximum of x over ranks)."""
    slowest = reduce_max(local_ms) if reduce_max else local_ms
    return n_hist * steps * world / (slowest / 1e3), slowest


def peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {"hbm_gbs": 6400.0, "bf16_tflops": 1800.0, "fallback": True}


class Clocks:
    """nvidia-smi sampling during the timed region."""

    def __init__(self, gpu_index):
        self.samples = []
        self.proc = None
        self.gpu = gpu_index

    def __enter__(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={q}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.samples.append([v.strip() for v in line.split(",")])

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        if not self.samples:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(s[1]) for s in self.samples if len(s) > 2 and s[1].replace(".", "").isdigit()]
        mx = [float(s[2]) for s in self.samples if len(s) > 2 and s[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for s in self.samples:
            for k, nm in enumerate(names):
                if len(s) > 5 + k and s[5 + k].lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": sorted(reasons),
                "samples": len(self.samples)}


def oracle_sample(prob, seconds, threads, seed=1, offset=0):
    """Runs the CPU oracle on growing history counts until `seconds` of wall
    time have been spent; returns (histories, segments, wall_s)."""
    from oracle import oracle as O
    n, done, segs, t_all = 20_000, 0, 0, 0.0
    while t_all < seconds:
        t0 = time.perf_counter()
        r = O.run(prob, n, seed=seed, offset=offset + done, batches=max(2, min(32, n // 1000)),
                  threads=threads)
        dt = time.perf_counter() - t0
        done += n
        segs += r["counts"]["segments"]
        t_all += dt
        n = int(min(max(n * 2, 20_000), max(20_000, n * (seconds - t_all) / max(dt, 1e-3))))
        if seconds - t_all < 0.5:
            break
    return done, segs, t_all


def run_reference(args, prob, n_hist):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    threads = os.cpu_count() or 1
    per_step = max(1.0, min(20.0, 120.0 / max(1, args.steps + args.warmup)))
    vals, segs_all, hist_all, t_all = [], 0, 0, 0.0
    for s in range(args.warmup + args.steps):
        h, sg, dt = oracle_sample(prob, per_step, threads, offset=s * 10_000_000)
        if s >= args.warmup:
            vals.append(h / dt)
            hist_all += h
            segs_all += sg
            t_all += dt
    value = hist_all / t_all
    cpu = {"value": value, "unit": "histories/s", "cores": threads, "kind": "oracle",
           "sample": f"{hist_all} histories of {prob.name} in {t_all:.1f} s on {threads} host threads "
                     f"(FP64 oracle, {segs_all / t_all:.3g} segments/s)"}
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "histories/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * t_all / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": prob.name, "histories_per_step": int(hist_all / args.steps),
                       "l2": "n/a (host)"},
            "cpu_baseline": cpu,
            "e2e": {"value": value, "unit": "histories/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="c2", choices=sorted(WORKLOADS))
    ap.add_argument("--histories", type=int, default=0)
    ap.add_argument("--precision", default="fp32_local", choices=["fp32", "fp32_local", "fp64"],
                    help="fp32_local (default): FP32 flights with FP64 positions and times "
                         "only where they cross a cell face or a census edge; fp32: FP64 "
                         "position and time accumulated every flight; fp64: all FP64")
    ap.add_argument("--batches", type=int, default=0, help="batches per run (0: library default)")
    ap.add_argument("--block", type=int, default=0, help="threads per CTA (0: library default)")
    ap.add_argument("--pc-target", type=int, default=0,
                    help="population control in the timed run: particles per batch after "
                         "each comb (0: off; the run then uses the global tally)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--no-fom", action="store_true", help="skip the learned-vs-analog FOM leg")
    ap.add_argument("--profile-deep", choices=["table", "per_event"], default=None,
                    help="only a compact deep-box run for an ncu capture: FP64 pilot, then "
                         "one FP32 cell-local run of 1e5 histories with learned windows "
                         "(baked table or per event); its first tracker launch is the only "
                         "cell-local one")
    ap.add_argument("--no-fom-per-event", action="store_true",
                    help="skip the deep box with the windows evaluated per event (a position "
                         "network fitted to the folded table, on the tensor cores)")
    ap.add_argument("--no-extra-workloads", action="store_true",
                    help="skip the 60^3 channel (HBM roofline) and the 256 batched problems")
    ap.add_argument("--no-variants", action="store_true",
                    help="skip the same workload in the other modes (cell-local FP32, "
                         "collision estimator, implicit capture)")
    args = ap.parse_args()

    if args.workload == "c5":
        run_batched_bench(args)
        return
    if args.profile_deep:
        profile_deep(args.profile_deep)
        return
    make, n_default = WORKLOADS[args.workload]
    prob = make()
    n_hist = args.histories or n_default
    if args.impl == "reference":
        run_reference(args, prob, n_hist)
        return

    import torch
    import torch.distributed as dist
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_2409_04668_b300 import mcdc as M

    prec = {"fp32": M.PREC_FP32, "fp32_local": M.PREC_FP32_LOCAL, "fp64": M.PREC_FP64}[args.precision]
    P = M.Problem(prob, precision=prec, block_size=args.block, pc_target=args.pc_target)
    dev = torch.device("cuda", local)
    mean = torch.empty(P.n_bins, dtype=torch.float64, device=dev)
    rel = torch.empty(P.n_bins, dtype=torch.float64, device=dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()

    def step(s):
        return P.run_ex(n_hist, seed=1, offset=history_offset(rank, s, n_hist), batches=args.batches,
                        mean=mean, relerr=rel,
                        stream=stream.cuda_stream, want_scalar=True, want_stats=True)

    for s in range(args.warmup):
        step(s)
        flush.fill_(float(s))
    torch.cuda.synchronize()

    kernel_ms, stats_all, scal_all = [], [], []
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    with Clocks(local) as clk:
        t0 = time.perf_counter()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for s in range(args.steps):
            st, sc = step(args.warmup + s)
            kernel_ms.append(st["kernel_ms"])
            stats_all.append(st)
            scal_all.append(sc)
            flush.fill_(float(s))
        e1.record(stream)
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
        # ---- end to end through the public API with host buffers: create
        # (uploads the tables), run with host outputs (D2H), destroy.  Inside
        # the sampled region: stopping nvidia-smi leaves the driver slow for a
        # while (creates 0.05 -> 0.3 ms, runs +0.25 ms measured), which is not
        # the library's cost
        nb = P.n_bins
        # pinned host buffers for the read-back (the channel's 3e7-bin mean
        # and error are 484 MB: an end-to-end step took 175 ms into pageable
        # buffers and 96 ms into pinned ones, against 79 ms on the device)
        h_mean = torch.zeros(nb, dtype=torch.float64).pin_memory()
        h_rel = torch.zeros(nb, dtype=torch.float64).pin_memory()
        h2d = int(prob.material.nbytes + 8 * (prob.sigma_t.size * 2 + prob.transfer.size +
                                              prob.speed.size + prob.src_pdf.size +
                                              (0 if prob.edges is None else prob.edges.size)))
        e2e_steps = max(1, min(3, args.steps))
        torch.cuda.synchronize()
        te0 = time.perf_counter()
        for s in range(e2e_steps):
            with M.Problem(prob, precision=prec, block_size=args.block,
                           pc_target=args.pc_target) as Q:
                Q.run_ex(n_hist, seed=1, offset=history_offset(rank, 500 + s, n_hist),
                         batches=args.batches, mean=h_mean, relerr=h_rel, want_stats=False)
        te = time.perf_counter() - te0
    def reduce_max(x):
        t = torch.tensor([x], dtype=torch.float64, device=dev)
        if world > 1:
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
        return float(t.item())

    value, region_ms = job_value(e0.elapsed_time(e1), n_hist, args.steps, world, reduce_max)
    segs = sum(s["segments"] for s in stats_all) / args.steps
    ms_step = region_ms / args.steps
    k_ms = float(np.mean(kernel_ms))

    e2e_val = n_hist * e2e_steps * world / te

    pk = peaks()
    measured_fp64 = M.measure_fp64_pipe()
    fom = None
    if scal_all and scal_all[-1] and scal_all[-1][1] > 0:
        fom = 1.0 / (scal_all[-1][1] ** 2 * (ms_step / 1e3))
    line = {
        "metric": METRIC, "value": value, "unit": "histories/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": {M.PREC_FP32: "f32+f64", M.PREC_FP32_LOCAL: "f32 (f64 faces and census edges)",
                  M.PREC_FP64: "f64"}[prec], "data": "synthetic",
        "config": {"workload": prob.name, "histories_per_step": n_hist, "precision": args.precision,
                   "tally_mode": ["auto", "shared", "global"][stats_all[-1]["tally_mode"]],
                   "n_batches": stats_all[-1]["n_batches"], "block": stats_all[-1]["block_size"],
                   "bank_per_cta": stats_all[-1]["bank_per_cta"],
                   "ctas_per_sm": stats_all[-1]["ctas_per_sm"],
                   "l2": "flushed between steps (256 MiB write)", "parallelism": f"replicas{world}"},
        "segments_per_sec": segs * args.steps * world / (region_ms / 1e3),
        "segments_per_history": segs / n_hist,
        "fom_region": fom,
        "region_relerr": scal_all[-1][1] if scal_all[-1] else None,
        "kernel_ms": k_ms,
        "clocks": clk.summary(),
        "e2e": {"value": e2e_val, "unit": "histories/s", "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": 2 * 8 * nb},
        "gpu_launches": None,
        "roofline": None,
    }
    launches_per_step = 2 if stats_all[-1]["tally_mode"] == 1 else 3 * stats_all[-1]["n_batches"] + 1
    if args.pc_target > 0:
        # per time step one tracker launch and four comb kernels (none after
        # the last), a fold pair per batch slice, one finalize
        T = len(prob.edges) - 1
        launches_per_step = T + 4 * (T - 1) + 2 * stats_all[-1]["n_batches"] + 1
    line["gpu_launches"] = launches_per_step * args.steps
    # roofline of the tracker from its per-flight algorithmic figures
    seg_rate = segs / (k_ms / 1e3)
    line["roofline"] = roofline(prob, seg_rate, pk, stats_all[-1]["tally_mode"], args.precision,
                                measured_fp64)
    if world == 1 and not args.no_variants:
        line["variants"] = variants(M, prob, n_hist, args, mean, rel, stream)
    if rank == 0 and world == 1 and not args.no_extra_workloads and args.workload == "c2":
        line["c3"] = channel_block(M, prec, args, pk, measured_fp64)
        line["c5"] = batched_block(M, prec, args)
    if rank == 0 and not args.no_fom and world == 1:
        line["fom"] = fom_over_pilots(M, prec, None)
        line["fom_shallow"] = fom_over_pilots(M, prec, W.c4_shallow(), match_relerr=0.04)
        if not args.no_fom_per_event:
            pe = fom_over_pilots(M, prec, None, per_event=True)
            for f in ("fom", "fom_incl_fit", "fom_incl_pilot"):
                if line["fom"].get(f"learned_{f}_median"):
                    pe[f"{f}_median_table_over_per_event"] = (
                        line["fom"][f"learned_{f}_median"] / max(pe[f"learned_{f}_median"], 1e-300))
            line["fom_per_event"] = pe
    if rank == 0 and not args.no_cpu_baseline and world == 1:
        h, sg, dt = oracle_sample(prob, args.cpu_seconds, os.cpu_count() or 1, offset=10**12)
        line["cpu_baseline"] = {"value": h / dt, "unit": "histories/s", "cores": os.cpu_count(),
                                "kind": "oracle",
                                "sample": f"{h} histories of {prob.name} ({sg / dt:.3g} segments/s) "
                                          f"in {dt:.1f} s, FP64 oracle on all host threads"}
    if world > 1:
        dist.destroy_process_group()
    P.close()
    if rank == 0:
        print(json.dumps(line), flush=True)


def channel_block(M, prec, args, pk, measured_fp64, n_hist=100_000_000):
    """The 60^3 channel (7 groups, 20 time bins, 3.02e7 tally bins, 242 MB of
    FP64 tally, larger than L2) at its full 1e8 histories: device-timed
    histories/s and segments/s, and the HBM roofline of the tracker at 16
    algorithmic bytes per segment (an FP64 read-modify-write of a tally bin)
    against the measured copy bandwidth.  The time is that of the run's
    launches (tracker and the slice fold), so the achieved figure is a
    slight underestimate of the tracker's own."""
    import torch
    prob = W.c3_channel()
    stream = torch.cuda.current_stream()
    with M.Problem(prob, precision=prec) as P:
        for s in range(args.warmup):
            P.run_ex(n_hist, seed=1, offset=history_offset(0, 800 + s, n_hist),
                     stream=stream.cuda_stream)
        ms, segs, st = [], 0, None
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        for s in range(args.steps):
            st, sc = P.run_ex(n_hist, seed=1, offset=history_offset(0, 820 + s, n_hist),
                              stream=stream.cuda_stream)
            ms.append(st["kernel_ms"])
            segs += st["segments"]
        e1.record(stream)
        torch.cuda.synchronize()
        region_ms = e0.elapsed_time(e1)
    k_s = float(np.sum(ms)) / 1e3
    seg_rate = segs / k_s
    out = {"workload": prob.name, "histories_per_step": n_hist, "steps": args.steps,
           "histories_per_s": n_hist * args.steps / (region_ms / 1e3),
           "histories_per_s_kernels": n_hist * args.steps / k_s,
           "segments_per_s": seg_rate, "segments_per_history": segs / (n_hist * args.steps),
           "ms_per_step": region_ms / args.steps, "kernel_ms": k_s * 1e3 / args.steps,
           "tally_mode": ["auto", "shared", "global"][st["tally_mode"]],
           "n_batches": st["n_batches"], "region_relerr": sc[1],
           "l2": "tally (242 MB) larger than L2",
           "roofline": roofline(prob, seg_rate, pk, st["tally_mode"], args.precision)}
    if args.precision == "fp32" and measured_fp64 is not None:
        # the same flights seen from the FP64 pipe: 16 operations per 3-D flight
        add, cvt = measured_fp64
        mix = 2.0 / (1.0 / add + 1.0 / cvt) / 1e12
        out["fp64_pipe"] = {"achieved_T_ops_per_s": seg_rate * 16 / 1e12,
                            "frac_of_measured_pipe": seg_rate * 16 / 1e12 / mix}
    return out


def batched_block(M, prec, args):
    """The 256 independent problems (meshes 16^3..64^3, 1..7 groups, 1e4..1e7
    histories, 3.3e8 in all) in one batched run per step: histories/s and
    segments/s over the run's device time."""
    probs, hist = W.c5_batch()
    handles = [M.Problem(p, precision=prec) for p in probs]
    try:
        # the first call autotunes the launch shape and captures the run's
        # graph; later calls replay it
        _, first_ms = _timed(lambda: M.run_batched(handles, hist, 1, batches=16))
        for s in range(1, max(2, args.warmup)):
            M.run_batched(handles, hist, 1 + s, batches=16)
        ms, segs, tot = [], 0, []
        for s in range(args.steps):
            (st, _), wall = _timed(lambda: M.run_batched(handles, hist, 100 + s, batches=16))
            ms.append(st["kernel_ms"])
            tot.append(wall)
            segs += st["segments"]
    finally:
        for h in handles:
            h.close()
    t = float(np.sum(ms)) / 1e3
    return {"workload": "c5_batched_256_problems", "problems": len(probs),
            "histories_per_step": int(sum(hist)), "steps": args.steps,
            "histories_per_s": sum(hist) * args.steps / t, "segments_per_s": segs / t,
            "ms_per_step": 1e3 * t / args.steps,
            "wall_ms_per_step": 1e3 * float(np.mean(tot)),
            "host_overhead_ms_per_step": 1e3 * (float(np.mean(tot)) - t / args.steps),
            "first_call_wall_ms": 1e3 * first_ms,
            "block": st["block_size"], "ctas_per_sm": st["ctas_per_sm"]}


def run_batched_bench(args):
    """256 independent 3-D problems of uneven size (meshes 16^3..64^3, 1..7
    groups, 1e4..1e7 histories) in one batched run per step."""
    import torch
    from paper_2409_04668_b300 import mcdc as M
    probs, hist = W.c5_batch()
    if args.impl == "reference":
        # the oracle on a bounded sample: the 16 smallest problems
        idx = np.argsort(hist)[:16]
        from oracle import oracle as O
        t0 = time.perf_counter()
        done = 0
        for i in idx:
            n = int(min(hist[i], 20_000))
            O.run(probs[i], n, seed=1, batches=4, threads=os.cpu_count() or 1)
            done += n
        dt = time.perf_counter() - t0
        v = done / dt
        print(json.dumps({"impl": "reference", "metric": METRIC, "value": v, "unit": "histories/s",
                          "n_gpus": 1, "steps": 1, "warmup": 0, "ms_per_step": dt * 1e3,
                          "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                          "dtype": "f64", "data": "synthetic",
                          "config": {"workload": "c5_batched_256_problems"},
                          "cpu_baseline": {"value": v, "unit": "histories/s", "kind": "oracle",
                                           "cores": os.cpu_count(),
                                           "sample": f"{done} histories of the 16 smallest problems"},
                          "e2e": {"value": v, "unit": "histories/s", "h2d_bytes_per_step": 0,
                                  "d2h_bytes_per_step": 0}}))
        return
    torch.cuda.set_device(0)
    prec = {"fp32": M.PREC_FP32, "fp32_local": M.PREC_FP32_LOCAL, "fp64": M.PREC_FP64}[args.precision]
    handles = [M.Problem(p, precision=prec) for p in probs]
    for s in range(args.warmup):
        M.run_batched(handles, hist, 1 + s, batches=16)
    ms, segs = [], 0
    with Clocks(0) as clk:
        for s in range(args.steps):
            st, _ = M.run_batched(handles, hist, 100 + s, batches=16)
            ms.append(st["kernel_ms"])
            segs += st["segments"]
    total = sum(hist) * args.steps
    t = sum(ms) / 1e3
    line = {"metric": METRIC, "value": total / t, "unit": "histories/s", "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": {M.PREC_FP32: "f32+f64", M.PREC_FP32_LOCAL: "f32 (f64 faces and census edges)",
                      M.PREC_FP64: "f64"}[prec], "data": "synthetic",
            "config": {"workload": "c5_batched_256_problems", "problems": len(probs),
                       "histories_per_step": int(sum(hist)), "batches": 16,
                       "block": st["block_size"], "ctas_per_sm": st["ctas_per_sm"],
                       "l2": "inputs (tallies 2.2 GB) larger than L2"},
            "segments_per_sec": segs / t, "clocks": clk.summary(), "gpu_launches": 16 * 3 + 1}
    for h in handles:
        h.close()
    print(json.dumps(line), flush=True)


def variants(M, prob, n_hist, args, mean, rel, stream):
    """The headline workload in the other modes of the tracker: device-timed
    histories/s and the region scalar's figure of merit 1/(relerr^2 T) for
    the cell-local FP32 mode, the FP32 mode with FP64 position and time
    accumulated every flight, the FP64 mode (the oracle's arithmetic, event
    for event) and, in the headline precision, for the
    collision estimator, for the combined track-length/collision estimator
    (both tallies, their minimum-variance combination), for implicit capture
    (weight cutoff 0.25, survival weight 0.5) and for population control (32
    batches, each combed back to its own size at every interior time
    edge)."""
    prec = {"fp32": M.PREC_FP32, "fp32_local": M.PREC_FP32_LOCAL, "fp64": M.PREC_FP64}[args.precision]
    modes = {"track_analog": {"precision": prec},
             "fp32_local": {"precision": M.PREC_FP32_LOCAL},
             "fp32_every_flight": {"precision": M.PREC_FP32},
             "fp64": {"precision": M.PREC_FP64},
             "collision_estimator": {"precision": prec, "estimator": M.EST_COLLISION},
             "combined_estimator": {"precision": prec, "estimator": M.EST_COMBINED},
             "implicit_capture": {"precision": prec, "implicit": (0.25, 0.5)},
             "population_control": {"precision": prec, "pc_target": n_hist // 32}}
    out = {}
    for name, kw in modes.items():
        with M.Problem(prob, block_size=args.block, **kw) as Q:
            nb = 32 if "pc_target" in kw else args.batches
            def one(s):
                st, sc = Q.run_ex(n_hist, seed=1, offset=history_offset(0, s, n_hist),
                                  batches=nb, mean=mean, relerr=rel,
                                  stream=stream.cuda_stream, want_scalar=True, want_stats=True)
                return st, sc
            for s in range(args.warmup):
                one(700 + s)
            ms, rels = [], []
            for s in range(args.steps):
                st, sc = one(720 + s)
                ms.append(st["kernel_ms"])
                rels.append(sc[1])
            t = float(np.mean(ms)) / 1e3
            r = float(np.mean(rels))
            out[name] = {"histories_per_s": n_hist / t, "region_relerr": r,
                         "fom_region": 1.0 / (r * r * t) if r > 0 else None,
                         "segments_per_history": st["segments"] / n_hist}
    return out


# Weight-window settings of the learned windows: source window 0.25 (the
# library default is 0.5), upper / survival ratios 4 / 2 (default 5 / 2.5).
# Over five pilot seeds on both boxes their median learned FOM was 4.6e4 (deep)
# and 7.0e4 (shallow) against 2.4e4 and 5.6e4 with the defaults, and two
# refits are needed (one gave a deep median of 106).  The fits and the refit
# runs count in the learned arm's time: swept over three pilot seeds with
# pilot, fits and refits in T, 10 epochs of 32768-sample minibatches and
# refit runs of 5e4 histories gave medians of 1.2e4 (deep) and 1.4e4
# (shallow) against 1.05e4 and 6.7e3 for 20 epochs of 16384 and refits of
# 1e5; 6 epochs, 40 epochs of 65536, or 3e4-history refits alone were worse.
WW_SETTINGS = {"source_wl": 0.25, "upper_ratio": 4.0, "survival_ratio": 2.0}


def fom_rel_uncertainty(n_batches):
    """Relative standard uncertainty of a figure of merit 1/(relerr^2 T) whose
    relerr comes from n batch means: the sample standard deviation of n
    normal values has relative error about 1/sqrt(2 (n - 1)), and the FOM
    goes as its inverse square."""
    return math.sqrt(2.0 / max(1, n_batches - 1))


def _timed(fn):
    """(result, wall seconds) of fn() between two device synchronisations."""
    import torch
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    r = fn()
    torch.cuda.synchronize()
    return r, time.perf_counter() - t0


def fom_deep(M, prec, n_analog=100_000_000, n_ww=100_000, refits=2, prob=None, seed0=7,
             per_event=False, match_relerr=None, ww_batches=32, epochs=10, fit_batch=32768,
             n_refit=50_000):
    """Figure of merit 1 / (relerr^2 T) of the far-region flux on the
    deep-penetration box (30 mfp absorber between a corner source and the
    region x in [90, 100]), analog against the learned weight windows.  The
    analog run's tally is the pilot; the network is refit twice, each time on
    the tally of a weight-window run with the previous windows (each such
    tally is an unbiased flux estimate that reaches deeper).

    T of the learned arm is reported three ways: the final weight-window
    run alone (device time, fom_transport_only), with the three fits and the
    two refit runs (wall time, fom_incl_fit), and with the analog pilot too
    (fom_incl_pilot).  The analog arm's T is its run's device time.
    match_relerr: also run the analog arm to about that relative error
    (chunks of 1e9 histories) and the learned arm's final run at the
    history count that reaches the same error, and compare the two at equal
    variance with every cost of the learned pipeline in T.  seed0 seeds the
    pilot; the weight-window runs use seed0 + 4, + 5, ....  per_event: the
    last fit's network sets every window at the event instead of a baked
    table (the refits still bake)."""
    import torch
    prob = prob if prob is not None else W.c4_deep()
    out = {"workload": prob.name, "region_cells": [list(prob.region_lo), list(prob.region_hi)]}
    dev = torch.device("cuda")
    tm = M.TALLY_GLOBAL if per_event else M.TALLY_AUTO
    with M.Problem(prob, precision=prec, tally_mode=tm) as P:
        mean = torch.zeros(P.n_bins, dtype=torch.float64, device=dev)
        rel = torch.zeros_like(mean)
        P.run_ex(1_000_000, seed0, mean=mean, relerr=rel)        # warm-up
        # the learned pipeline warms up too: its kernels (training, bake,
        # weighted tracker; the distillation when per event) load on their
        # first use, a once-per-process cost like the analog kernel's above.
        # One short fit on the warm-up tally and a 1000-history run with its
        # windows; then the problem is analog again for the pilot
        P.train_importance(mean, rel, epochs=1, batch=fit_batch, min_ratio=1e-20,
                           per_event=int(per_event), distill_steps=16, **WW_SETTINGS)
        P.run_ex(1000, seed0 + 999, batches=ww_batches)
        P.set_weight_windows(None)
        (st, (m_a, r_a)), wall_a = _timed(lambda: P.run_ex(n_analog, seed0, mean=mean, relerr=rel))
        t_a = st["kernel_ms"] / 1e3
        nb_a = st["n_batches"]
        out["analog"] = {"histories": n_analog, "mean": m_a, "relerr": r_a if m_a > 0 else None,
                         "seconds": t_a, "histories_per_s": n_analog / t_a, "batches": nb_a,
                         "fom": (1.0 / (r_a ** 2 * t_a)) if m_a > 0 and r_a > 0 else None,
                         "fom_rel_uncertainty": fom_rel_uncertainty(nb_a) if m_a > 0 else None,
                         "fom_upper_bound": None if m_a > 0 else 1.0 / t_a,
                         "note": None if m_a > 0 else "no analog history scored in the region: "
                                 "relerr >= 1, so FOM <= 1/T"}
        fit_wall, fit_dev, ww_wall = 0.0, 0.0, 0.0
        seed = seed0 + 4
        for it in range(refits + 1):
            rep, w = _timed(lambda: P.train_importance(
                mean, rel, epochs=epochs, batch=fit_batch, min_ratio=1e-20,
                per_event=int(per_event and it == refits), **WW_SETTINGS))
            fit_wall += w
            fit_dev += (rep["train_ms"] + rep["bake_ms"]) / 1e3
            if it < refits:
                _, w = _timed(lambda: P.run_ex(n_refit or n_ww, seed, batches=ww_batches,
                                               mean=mean, relerr=rel))
                ww_wall += w
                seed += 1
        st, (m_w, r_w) = P.run_ex(n_ww, seed, batches=ww_batches)
        t_w = st["kernel_ms"] / 1e3
        t_incl_fit = fit_wall + ww_wall + t_w
        t_incl_pilot = t_incl_fit + wall_a
        fom_w = (1.0 / (r_w ** 2 * t_w)) if m_w > 0 and r_w > 0 else None
        out["learned"] = {"histories": n_ww, "mean": m_w, "relerr": r_w, "seconds": t_w,
                          "batches": ww_batches, "histories_per_s": n_ww / t_w,
                          "fom_transport_only": fom_w,
                          "fom": fom_w,
                          "fom_incl_fit": (1.0 / (r_w ** 2 * t_incl_fit)) if fom_w else None,
                          "fom_incl_pilot": (1.0 / (r_w ** 2 * t_incl_pilot)) if fom_w else None,
                          "fom_rel_uncertainty": fom_rel_uncertainty(ww_batches),
                          "seconds_incl_fit": t_incl_fit, "seconds_incl_pilot": t_incl_pilot,
                          "splits": st["splits"], "segments_per_history": st["segments"] / n_ww,
                          "fit_seconds_wall": fit_wall, "fit_seconds_device": fit_dev,
                          "refit_runs_seconds_wall": ww_wall, "pilot_seconds_wall": wall_a,
                          "fits": refits + 1, "refits": refits}
        if match_relerr and m_a > 0 and fom_w:
            out["equal_variance"] = equal_variance(M, P, prob, prec, seed0, match_relerr, r_w, n_ww,
                                                   seed + 1, ww_batches,
                                                   fit_wall + ww_wall + wall_a)
    a, l = out["analog"], out["learned"]
    if l["fom"] and a["fom"]:
        out["ratio"] = l["fom"] / a["fom"]
        out["ratio_incl_fit"] = l["fom_incl_fit"] / a["fom"]
        out["ratio_incl_pilot"] = l["fom_incl_pilot"] / a["fom"]
        out["ratio_rel_uncertainty"] = math.hypot(a["fom_rel_uncertainty"], l["fom_rel_uncertainty"])
    elif l["fom"] and a["fom_upper_bound"]:
        out["ratio_lower_bound"] = l["fom"] / a["fom_upper_bound"]
        out["ratio_incl_fit_lower_bound"] = l["fom_incl_fit"] / a["fom_upper_bound"]
        out["ratio_incl_pilot_lower_bound"] = l["fom_incl_pilot"] / a["fom_upper_bound"]
    return out


def equal_variance(M, P, prob, prec, seed0, target, r_w1, n_w1, seed_w, ww_batches, overhead_s,
                   chunk=1_000_000_000, max_seconds=12.0):
    """Analog and learned runs of the far-region flux taken to the same
    relative error.  Analog: chunks of `chunk` histories (independent seeds)
    until the combined relative error reaches `target` or max_seconds of
    device time are spent; the learned arm's final run is then repeated with
    the history count that reaches the analog's error (from its first run's
    error, relerr ~ 1/sqrt(N), corrected up to twice from the error the run
    reached), and its T includes every cost of the pipeline (pilot, fits,
    refit runs: overhead_s) and every try of the final run."""
    import torch
    means, vars_, secs, nb = [], [], 0.0, 0
    with M.Problem(prob, precision=prec) as A:
        k = 0
        while True:
            st, (m, r) = A.run_ex(chunk, seed0 + 1000 + k, batches=32)
            k += 1
            means.append(m)
            vars_.append((m * r) ** 2)
            secs += st["kernel_ms"] / 1e3
            nb += st["n_batches"]
            mc = float(np.mean(means))
            rc = math.sqrt(sum(vars_)) / len(means) / mc if mc > 0 else float("inf")
            if rc <= target or secs >= max_seconds:
                break
    # the learned run's history count for the analog's error, from relerr ~
    # 1/sqrt(N): three tries at most, each from the last run's own error
    n_w, r_w1n, t_w = n_w1, r_w1, 0.0
    for attempt in range(3):
        n_w = int(max(2000, math.ceil(n_w * (r_w1n / rc) ** 2)))
        (st, (m_w, r_w)), wall = _timed(lambda: P.run_ex(n_w, seed_w + attempt, batches=ww_batches))
        t_w += st["kernel_ms"] / 1e3
        r_w1n = r_w
        if abs(r_w / rc - 1.0) < 0.15:
            break
    t_tot = overhead_s + t_w
    fa, fw = 1.0 / (rc * rc * secs), 1.0 / (r_w * r_w * t_tot)
    ua, uw = fom_rel_uncertainty(nb), fom_rel_uncertainty(ww_batches)
    z = (m_w - mc) / math.hypot(m_w * r_w, mc * rc)
    return {"target_relerr": target,
            "analog": {"histories": chunk * len(means), "mean": mc, "relerr": rc, "seconds": secs,
                       "batches": nb, "fom": fa, "fom_rel_uncertainty": ua},
            "learned": {"histories": n_w, "mean": m_w, "relerr": r_w, "seconds_runs": t_w,
                        "tries": attempt + 1,
                        "seconds_incl_pilot_and_fit": t_tot, "fom_incl_pilot": fw,
                        "fom_rel_uncertainty": uw},
            "agreement_z": z,
            "ratio_incl_pilot": fw / fa, "ratio_rel_uncertainty": math.hypot(ua, uw),
            "time_ratio": secs / t_tot}


def profile_deep(mode):
    """The deep box's learned-window transport in a form small enough to
    capture: the pilot in FP64 (another kernel instantiation), windows trained
    from it on an FP32 cell-local problem (a baked table, or per event), then
    one run of 1e5 histories whose first tracker launch is the first FP32
    cell-local one; spill banks of 2^22 particles keep the device memory to a
    few GB.  Prints the run's counts and device time."""
    import torch
    from paper_2409_04668_b300 import mcdc as M
    prob = W.c4_deep()
    dev = torch.device("cuda")
    with M.Problem(prob, precision=M.PREC_FP64, tally_mode=M.TALLY_GLOBAL, block_size=512) as P0:
        mean = torch.zeros(P0.n_bins, dtype=torch.float64, device=dev)
        rel = torch.zeros_like(mean)
        P0.run_ex(10_000_000, 7, mean=mean, relerr=rel)
    with M.Problem(prob, precision=M.PREC_FP32_LOCAL, tally_mode=M.TALLY_GLOBAL, block_size=512,
                   spill_particles=1 << 22) as P:
        rep = P.train_importance(mean, rel, epochs=10, batch=32768, min_ratio=1e-20,
                                 per_event=int(mode == "per_event"), **WW_SETTINGS)
        st, (m, r) = P.run_ex(100_000, 20, batches=16)
    print(json.dumps({"profile": f"deep_box_{mode}", "workload": prob.name, "histories": 100_000,
                      "fit": {k: rep[k] for k in ("samples", "steps", "train_ms", "bake_ms",
                                                  "distill_steps")},
                      "kernel_ms": st["kernel_ms"], "segments": st["segments"],
                      "collisions": st["collisions"], "crossings": st["crossings"],
                      "splits": st["splits"], "splits_dropped": st["splits_dropped"]}),
          flush=True)


def fom_over_pilots(M, prec, prob, seeds=(7, 107, 207, 307, 407), per_event=False,
                    match_relerr=None):
    """fom_deep for the first pilot seed in full, plus the learned FOM (and the
    ratio to analog, or its lower bound) for every seed and their medians: the
    windows depend on the pilot sample, so one seed is one draw of the whole
    pipeline (each FOM carries the +-25 % of its 32 batches, and the pipeline
    scatters beyond that; the median of five is the figure reported)."""
    runs = [fom_deep(M, prec, prob=prob, seed0=s, per_event=per_event,
                     match_relerr=match_relerr if k == 0 else None)
            for k, s in enumerate(seeds)]
    out = runs[0]
    out["pilot_seeds"] = list(seeds)
    for f in ("fom", "fom_incl_fit", "fom_incl_pilot"):
        v = [r["learned"][f] or 0.0 for r in runs]
        out[f"learned_{f}_by_pilot_seed"] = v
        out[f"learned_{f}_median"] = float(np.median(v))
    lb = "" if "ratio" in out else "_lower_bound"
    for f in ("ratio", "ratio_incl_fit", "ratio_incl_pilot"):
        v = [r.get(f + lb) or 0.0 for r in runs]
        out[f"{f}{lb}_by_pilot_seed"] = v
        out[f"{f}{lb}_median"] = float(np.median(v))
    return out


# DRAM bytes (read + write) per tracker launch from one ncu capture of the
# bench's own workload, keyed by (workload, precision, tally mode), with the
# digest of the library sources the capture ran on: a figure is reported only
# while the sources are unchanged (null otherwise, until it is re-measured).
MEASURED_TRAFFIC = {
    # ncu dram__bytes_read.sum + dram__bytes_write.sum, mean of the timed
    # tracker launches of the bench's own configuration
    ("c2_slab_20cm_2region_td", "fp32_local", 1): (341333, "23d89968d84502dc"),
    ("c3_channel_60cube_7g_td", "fp32_local", 2): (364779861, "23d89968d84502dc"),
}


def source_digest():
    """First 16 hex digits of the SHA-256 of the library's CUDA sources."""
    d = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2409_04668_b300", "csrc")
    for f in sorted(os.listdir(csrc)):
        if f.endswith((".cu", ".cuh", ".h")):
            d.update(f.encode())
            d.update(open(os.path.join(csrc, f), "rb").read())
    return d.hexdigest()[:16]


def measured_traffic(name, prec_name, tally_mode):
    v = MEASURED_TRAFFIC.get((name, prec_name, tally_mode))
    if v is None or v[1] != source_digest():
        return None
    return v[0]


def roofline(prob, seg_rate, pk, tally_mode, prec_name, measured_fp64=None):
    """Roofline of the tracker for the binding unit of its precision mode.

    FP32 split: every flight accumulates x (and y, z in 3-D) and t in FP64 and
    takes the face and census distances from them -- 8 FP64-pipe operations
    per 1-D flight, 16 per 3-D flight (conversions and adds) -- and the FP64
    pipe binds; peak = the recipe's nominal B300 FP64 rate, 1.25 TFLOP/s = 0.625
    T FP64-pipe operations/s.  Cell-local mode: no FP64 in a flight; bound by
    issue slots, lane-operations per flight of the algorithm as run (optical
    depth carried, so no Philox block or logarithm in a flight: divide 1,
    optical-depth update 2, lookup 3, face 4, census 3, nearest event 4,
    tally 4, move 4, resolution 4, collisions 18 and births 5 amortised = 52)
    against 148 SMs x 128 lanes x max SM clock.  Global tally
    (large meshes): a read-modify-write of the scored bin per flight, 8 B of
    an FP32 batch slice (16 B of an FP64 bin in FP64 mode), against the
    measured copy bandwidth."""
    three_d = prob.n[1] > 1 or prob.n[2] > 1
    if tally_mode == 2 and (prec_name == "fp64" or three_d):
        # a read-modify-write of the scored bin: FP64 in FP64 mode, an FP32
        # batch slice in the FP32 modes
        bps = 16 if prec_name == "fp64" else 8
        ach = seg_rate * bps / 1e9
        return {"bound": "hbm", "achieved": ach, "peak": pk["hbm_gbs"], "unit": "GB/s",
                "frac": ach / pk["hbm_gbs"],
                "traffic": measured_traffic(prob.name, prec_name, tally_mode),
                "traffic_unit": "DRAM bytes per launch (ncu)", "bytes_per_segment": bps,
                "peak_kind": "measured copy (MEASURED_PEAKS.json hbm_gbs)"}
    if prec_name == "fp32":
        ops = 16.0 if three_d else 8.0
        peak = 0.625
        ach = seg_rate * ops / 1e12
        out = {"bound": "alu", "achieved": ach, "peak": peak, "unit": "T FP64-pipe ops/s",
               "frac": ach / peak,
               "traffic": measured_traffic(prob.name, prec_name, tally_mode),
               "traffic_unit": "DRAM bytes per launch (ncu)", "ops_per_segment": ops,
               "peak_kind": "nominal B300 FP64 1.25 TFLOP/s = 0.625 T pipe ops/s (recipe)"}
        if measured_fp64 is not None:
            # half of a flight's FP64-pipe operations are conversions, half adds
            add, cvt = measured_fp64
            mix = 2.0 / (1.0 / add + 1.0 / cvt) / 1e12 if add > 0 and cvt > 0 else None
            out["measured_pipe"] = {"add_T_per_s": add / 1e12, "cvt_T_per_s": cvt / 1e12,
                                    "flight_mix_T_per_s": mix,
                                    "frac_of_measured": ach / mix if mix else None,
                                    "how": "mcdc_measure_fp64_pipe on this GPU before the run"}
        return out
    ops_per_seg = 52.0
    peak = 148 * 128 * pk.get("sm_max_mhz", 2032.0) * 1e6 / 1e12
    ach = seg_rate * ops_per_seg / 1e12
    return {"bound": "alu", "achieved": ach, "peak": peak, "unit": "T lane-ops/s",
            "frac": ach / peak, "traffic": measured_traffic(prob.name, prec_name, tally_mode),
            "traffic_unit": "DRAM bytes per launch (ncu)", "ops_per_segment": ops_per_seg,
            "peak_kind": "issue slots: 148 SM x 128 lanes x max SM clock (recipe unit "
                         "counts and clock)"}


if __name__ == "__main__":
    main()
