#!/usr/bin/env python3
"""Benchmark of the ACA minimal-solver hot path on GB300.

Headline (one JSON line on rank 0): batched ACA minimal solve over 2^26
synthetic minimal sets (16 float32 in, 9 out per set), H/s, with inputs
resident in HBM; a step is one aca_solve over the whole batch.  The same line
carries the roofline of that kernel, the FP64 oracle timed on the host cores,
an end-to-end number through the C ABI with host buffers, the SM clocks seen
during the measurement, and the other rows of the hot path measured in the
same run: SKS on the same sets, fused RANSAC on one image pair (N = 2000,
4096 hypotheses), batched uneven RANSAC (512 pairs) against 512 separate
per-problem launches, and the differentiable rectangle ACA (forward +
backward, batch 65536) against the plain solve.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

N > 1 runs under torchrun, one rank per GPU, each rank solving its own 2^26
sets (weak scaling, no collective on the data path).  --impl reference times
the FP64 CPU oracle on the host cores instead (rank 0 only).
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

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import workloads  # noqa: E402

N_LOG2 = 26
BYTES_PER_SET = 64 + 36          # 16 float32 in, 9 float32 out
FLOPS_PER_TEST = 21              # one hypothesis x point test, FMA = 2
RANSAC_THR = 3.0
SEED = 0


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--n-log2", type=int, default=N_LOG2)
    ap.add_argument("--no-rows", action="store_true", help="headline only")
    ap.add_argument("--rows", default="config0,sks,affine,ransac1,ransac512,adaptive,refit,diff,latency",
                    help="comma list of extra rows: config0, sks, affine, ransac1, ransac512, adaptive, refit, diff, "
                         "latency")
    ap.add_argument("--cpu-seconds", type=float, default=10.0, help="oracle timing of the headline")
    ap.add_argument("--row-cpu-seconds", type=float, default=3.0, help="oracle timing of each extra row")
    ap.add_argument("--ransac-tuning", default="",
                    help="block_warps,hyps_per_thread,tile_points for the RANSAC rows (skips the autotuner)")
    ap.add_argument("--no-plain", action="store_true", help="skip the 512 per-problem RANSAC launches")
    return ap.parse_args()


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return dict(hbm_gbs=float(d["hbm_gbs"]), source="measured", sm_max_mhz=float(d.get("sm_max_mhz", 2070)))
    except Exception:
        return dict(hbm_gbs=6800.0, source="fallback", sm_max_mhz=2070.0)


class ClockSampler:
    """nvidia-smi clock / throttle sampling (200 ms) around a measured region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,utilization.gpu,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            time.sleep(0.3)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        rows = []
        try:
            for line in open(self.path):
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 10:
                    rows.append(parts)
        except Exception:
            pass
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}

        def num(x):
            try:
                return float(x)
            except ValueError:
                return None
        load = [r for r in rows if (num(r[4]) or 0) > 0] or rows
        sm = [num(r[1]) for r in load if num(r[1]) is not None]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in load for i in range(4) if r[6 + i].lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": num(load[0][2]),
                "reasons": reasons, "samples": len(rows), "samples_under_load": len(load),
                "power_w_max": max((num(r[3]) or 0) for r in rows)}


def solve_traffic_per_launch(n):
    """DRAM bytes per launch of the headline kernel from the committed ncu
    capture (profiles/aca_solve_traffic.json), scaled to n sets; None when
    the kernel's sources changed since the capture."""
    import hashlib
    try:
        rec = json.load(open(os.path.join(ROOT, "profiles", "aca_solve_traffic.json")))
        h = hashlib.sha256()
        for f in rec["source_files"]:
            h.update(open(os.path.join(ROOT, f), "rb").read())
        if h.hexdigest() != rec["source_sha256"]:
            return None
        return rec["dram_bytes_per_set"] * n
    except Exception:
        return None


def rank_seed(rank: int) -> int:
    """Each rank solves its own batch of the same size (weak scaling)."""
    return SEED + rank


def max_over_ranks(x: float, torch, device) -> float:
    """Slowest rank's time: the whole job finishes when the last rank does."""
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(sets_per_rank: int, world: int, max_ms: float) -> float:
    """Whole-job H/s: the sets of all ranks over the slowest rank's time."""
    return sets_per_rank * world / (max_ms * 1e-3)


def sync_all(torch, dist_on):
    if dist_on:
        import torch.distributed as dist
        dist.barrier()
    torch.cuda.synchronize()


def link_bandwidth(torch, dev, stream):
    """Plain cudaMemcpyAsync bandwidth between page-locked host memory and the
    device (GB/s): H2D alone, D2H alone, and both at once on two streams."""
    nb = 1 << 30
    h_in = torch.empty(nb, dtype=torch.uint8).pin_memory()
    h_out = torch.empty(nb, dtype=torch.uint8).pin_memory()
    d_in = torch.empty(nb, dtype=torch.uint8, device=dev)
    d_out = torch.empty(nb, dtype=torch.uint8, device=dev)
    s2 = torch.cuda.Stream(device=dev)
    h2d = lambda: d_in.copy_(h_in, non_blocking=True)
    d2h = lambda: h_out.copy_(d_out, non_blocking=True)

    def both():
        s2.wait_stream(stream)
        with torch.cuda.stream(s2):
            d2h()
        h2d()
        stream.wait_stream(s2)
    for f in (h2d, d2h, both):
        f()
    torch.cuda.synchronize()
    t_in = time_region(torch, h2d, 5, stream)
    t_out = time_region(torch, d2h, 5, stream)
    t_both = time_region(torch, both, 5, stream)
    del h_in, h_out, d_in, d_out
    return {"h2d_gbs": nb / (t_in * 1e-3) / 1e9, "d2h_gbs": nb / (t_out * 1e-3) / 1e9,
            "h2d_gbs_duplex": nb / (t_both * 1e-3) / 1e9, "d2h_gbs_duplex": nb / (t_both * 1e-3) / 1e9}


def time_region(torch, fn, steps, stream):
    """Average ms per call of fn over `steps` calls, CUDA events on `stream`."""
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        fn()
    e1.record(stream)
    e1.synchronize()
    return e0.elapsed_time(e1) / steps


def cpu_baseline_aca(pts16, seconds):
    """The FP64 oracle's ACA over chunks of the same sets on the host cores."""
    import oracle
    n = pts16.shape[1]
    chunk = min(n, 1 << 21)
    done, t0, k = 0, time.perf_counter(), 0
    aos = oracle.sets_aos(pts16[:, :chunk])
    while True:
        t = time.perf_counter()
        oracle.lib().oracle_aca(aos.ctypes.data_as(oracle._d), np.empty((chunk, 9)).ctypes.data_as(oracle._d), chunk)
        done += chunk
        k += 1
        if time.perf_counter() - t0 >= seconds:
            break
    el = time.perf_counter() - t0
    return {"value": done / el, "unit": "H/s", "cores": oracle.num_threads(), "kind": "oracle",
            "sample": f"{k} passes of the FP64 C oracle (OpenMP) over the first {chunk} of the 2^{int(np.log2(n))} "
                      f"sets ({el:.1f} s)"}


def error_stats(H_planes_np, flags_np, pts16, n, rng):
    import oracle
    idx = np.sort(rng.choice(n, size=min(n, 1 << 16), replace=False))
    ref = oracle.aca(pts16[:, idx])
    a = H_planes_np[:, idx].T.astype(np.float64)
    a /= np.linalg.norm(a, axis=1, keepdims=True)
    b = ref / np.linalg.norm(ref, axis=1, keepdims=True)
    a *= np.sign(np.sum(a * b, axis=1, keepdims=True))
    e = np.abs(a - b).max(axis=1)
    flagged = (flags_np[idx] & 7) > 0
    ok = ~flagged
    beta = oracle.aca_fp32_bound(pts16[:, idx])
    within = ok & (beta <= 1e-4)
    bound = np.maximum(1e-4, beta + beta * beta)
    return {"sample_sets": int(idx.size), "max_err": float(e[ok].max()), "median_err": float(np.median(e[ok])),
            "frac_above_1e-4": float(np.mean(e[ok] > 1e-4)), "flagged_sets": int(flagged.sum()),
            "flagged_max_err": float(e[flagged].max()) if flagged.any() else None,
            "sets_with_bound_below_1e-4": int(within.sum()), "their_max_err": float(e[within].max()),
            "max_err_over_bound": float(np.max(e[ok] / bound[ok])),
            "max_err_over_fp32_bound": float(np.max(e[ok] / beta[ok])),
            "metric": "max |H_gpu - H_fp64| with both at unit Frobenius norm, sign aligned; flagged = a triple "
                      "within 1 px of collinear (excluded); fp32 bound = the oracle's first-order bound on the "
                      "rounding error of the library's FP32 evaluation order; bound = max(1e-4, fp32 bound)"}


def run_reference(args, rank):
    """The FP64 CPU oracle on the host cores, same metric and workload."""
    if rank != 0:
        return
    import oracle
    oracle.build()
    n = 1 << args.n_log2
    sample = 1 << 20
    ms = workloads.minimal_sets(sample, seed=SEED, degenerate_frac=0.01, keep_truth=False, workers=os.cpu_count())
    aos = oracle.sets_aos(ms.pts)
    out = np.empty((sample, 9))
    run = lambda: oracle.lib().oracle_aca(aos.ctypes.data_as(oracle._d), out.ctypes.data_as(oracle._d), sample)
    for _ in range(args.warmup):
        run()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        run()
    el = time.perf_counter() - t0
    v = sample * args.steps / el
    line = {"metric": "ACA minimal solves per second (config 1: 2^26 sets, FP32 SoA 16 in / 9 out)", "value": v,
            "unit": "H/s", "impl": "reference", "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": el / args.steps * 1e3, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"aca_solve, 2^{args.n_log2} minimal sets (a {sample}-set sample per step)",
                       "sets": n, "sample_sets_per_step": sample},
            "cpu_baseline": {"value": v, "unit": "H/s", "cores": oracle.num_threads(), "kind": "oracle",
                             "sample": f"the first {sample} sets of the workload per step"},
            "e2e": {"value": v, "unit": "H/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank)
        return
    n = 1 << args.n_log2
    # host-side generation first (process pool before any CUDA call)
    ms = workloads.minimal_sets(n, seed=rank_seed(rank), degenerate_frac=0.01, keep_truth=False,
                                workers=max(1, os.cpu_count() or 1))
    rows_on = not args.no_rows and world == 1
    args.row_set = set(r for r in args.rows.split(",") if r) if rows_on else set()
    rp = workloads.ransac_problem(2000, 0.6, 1.0, seed=SEED) if "ransac1" in args.row_set else None
    rb = workloads.ransac_batch(512, seed=SEED) if args.row_set & {"ransac512", "adaptive", "refit"} else None
    rect = workloads.rect_batch(65536, seed=SEED) if "diff" in args.row_set else None

    import torch
    dist_on = world > 1
    if dist_on:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    from paper_2402_18008_gb300 import _lib, api
    _lib.load()
    peaks = measured_peaks()
    sms = torch.cuda.get_device_properties(dev).multi_processor_count

    pts = torch.from_numpy(ms.pts).to(dev)
    H = torch.empty((9, n), dtype=torch.float32, device=dev)
    flags = torch.empty(n, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream()
    solve = lambda: _lib.aca_solve(pts, H, None, n=n)
    res = {}
    with ClockSampler(local) as clocks:
        for _ in range(args.warmup):
            solve()
        sync_all(torch, dist_on)
        ms_step = time_region(torch, solve, args.steps, stream)
        sync_all(torch, dist_on)
        ms_step = max_over_ranks(ms_step, torch, dev)
        # errors vs the FP64 oracle on a sample (flags from a flags-on solve)
        _lib.aca_solve(pts, H, flags, n=n)
        torch.cuda.synchronize()
        if rank == 0:
            res["err"] = error_stats(H.cpu().numpy(), flags.cpu().numpy(), ms.pts, n, np.random.default_rng(1))
        if rows_on:
            ctx = {"peaks": peaks, "sms": sms, "pts_np": ms.pts, "cpu_s": args.row_cpu_seconds}
            if args.row_set & {"ransac1", "ransac512", "adaptive"}:
                ctx["fma"] = measure_fma(torch, _lib, sms, stream, dev)
            res.update(run_rows(torch, _lib, api, pts, H, flags, n, rp, rb, rect, args, stream, dev, ctx))
    clk = clocks.summary()
    if rank != 0:
        if dist_on:
            dist.destroy_process_group()
        return

    # end to end through the C ABI with host buffers: the sets start in
    # pinned host memory and the homographies end there, every step.  The
    # call is aca_solve on the host buffers themselves: the kernel reads the
    # sets over the host link and writes H back over it (zero-copy).  For
    # comparison, the staged form: H2D copy, solve in HBM, D2H copy.
    e2e_steps = max(3, min(args.steps, 10))
    pts_h = torch.from_numpy(ms.pts).pin_memory()
    H_h = torch.empty((9, n), dtype=torch.float32).pin_memory()

    def e2e_step():
        _lib.aca_solve(pts_h, H_h, None, n=n)

    def staged_step():
        pts.copy_(pts_h, non_blocking=True)
        _lib.aca_solve(pts, H, None, n=n)
        H_h.copy_(H, non_blocking=True)
    pinned = api.PinnedSolver(dev)
    pipelined_step = lambda: pinned(pts_h, H_h, n)
    for f in (e2e_step, staged_step, pipelined_step):
        f()
    torch.cuda.synchronize()
    zero_copy_ms = time_region(torch, e2e_step, e2e_steps, stream)
    staged_ms = time_region(torch, staged_step, e2e_steps, stream)
    pipelined_ms = time_region(torch, pipelined_step, e2e_steps, stream)
    e2e_ms = min(zero_copy_ms, pipelined_ms)
    e2e_path = ("aca_solve on pinned host buffers (zero-copy over the host link)" if zero_copy_ms <= pipelined_ms
                else "api.PinnedSolver: chunked H2D -> solve -> D2H on 3 streams")
    link = link_bandwidth(torch, dev, stream)
    in_b, out_b = 64 * n, 36 * n
    link_ms = max(in_b / link["h2d_gbs"], out_b / link["d2h_gbs"]) / 1e6

    cpu = cpu_baseline_aca(ms.pts, args.cpu_seconds)
    value = job_throughput(n, world, ms_step)
    achieved = BYTES_PER_SET * n / (ms_step * 1e-3) / 1e9
    line = {
        "metric": "ACA minimal solves per second (config 1: 2^26 sets, FP32 SoA 16 in / 9 out)",
        "value": value, "unit": "H/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32", "data": "synthetic",
        "config": {"workload": f"aca_solve over 2^{args.n_log2} minimal sets per GPU (1% near-degenerate)",
                   "sets_per_gpu": n, "bytes_per_set": BYTES_PER_SET, "norm": "none",
                   "l2": "inputs (4 GiB) larger than L2, no flush"},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                     "frac": achieved / peaks["hbm_gbs"], "traffic": solve_traffic_per_launch(n),
                     "peak_source": peaks["source"], "kernel": "solve_ring_kernel<ACA, NONE, no flags>",
                     "algorithmic_bytes_per_launch": BYTES_PER_SET * n},
        "cpu_baseline": cpu,
        "e2e": {"value": n / (e2e_ms * 1e-3), "unit": "H/s", "h2d_bytes_per_step": in_b,
                "d2h_bytes_per_step": out_b, "ms_per_step": e2e_ms, "path": e2e_path,
                "zero_copy_ms_per_step": zero_copy_ms, "pipelined_3_streams_ms_per_step": pipelined_ms,
                "serial_staged_copies_ms_per_step": staged_ms,
                "roofline": {"bound": "host link", "link": link, "link_bound_ms": link_ms,
                             "frac": link_ms / e2e_ms,
                             "note": "bound = max(in bytes / H2D rate, out bytes / D2H rate), each rate measured "
                                     "alone with plain cudaMemcpyAsync copies of 1 GiB pinned buffers (the link is "
                                     "full duplex; the copy engines run both directions at once at the _duplex "
                                     "rates, below what the zero-copy kernel reaches)"}},
        "gpu_launches": args.steps,
        "clocks": clk,
        "max_err_vs_fp64": res.get("err"),
        "sms": sms,
    }
    if rows_on:
        line["rows"] = {k: v for k, v in res.items() if k != "err"}
    print(json.dumps(line), flush=True)
    if dist_on:
        dist.destroy_process_group()


def fp32_peak_tflops(sms, mhz):
    return sms * 128 * 2 * mhz * 1e6 / 1e12


def measure_fma(torch, _lib, sms, stream, dev):
    """The FP32 rate measured by the library's FMA probe (aca_fma_probe: 8
    independent FMA chains per thread, 4 blocks of 256 threads per SM), as
    scalar FMAs and as packed f32x2 FMAs (the form the RANSAC scoring
    issues), TFLOP/s from CUDA events over 10 launches."""
    blocks, threads, steps = sms * 4, 256, 4096
    sink = torch.empty(blocks * threads, dtype=torch.float32, device=dev)
    out = {"blocks": blocks, "threads": threads, "steps": steps}
    for name, packed in (("scalar_tflops", False), ("packed_f32x2_tflops", True)):
        f = lambda: _lib.fma_probe(sink, packed, blocks, threads, steps)
        flops = f()
        for _ in range(3):
            f()
        out[name] = flops / (time_region(torch, f, 10, stream) * 1e-3) / 1e12
    return out


def row_counter(row):
    """The ncu counter behind a row's roofline, from the committed capture
    (profiles/row_counters.json); marked stale when the kernel's sources
    changed since the capture."""
    import hashlib
    try:
        rec = json.load(open(os.path.join(ROOT, "profiles", "row_counters.json")))[row]
        h = hashlib.sha256()
        for f in rec["source_files"]:
            h.update(open(os.path.join(ROOT, f), "rb").read())
        out = {k: v for k, v in rec.items() if k not in ("source_files", "source_sha256")}
        if h.hexdigest() != rec["source_sha256"]:
            out["stale"] = True
        return out
    except Exception:
        return None


def roofline_hbm(row, bytes_per_launch, ms, ctx, kernel, note=None):
    achieved = bytes_per_launch / (ms * 1e-3) / 1e9
    peak = ctx["peaks"]["hbm_gbs"]
    r = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
         "peak_source": ctx["peaks"]["source"], "kernel": kernel, "algorithmic_bytes_per_launch": bytes_per_launch,
         "counter": row_counter(row)}
    if note:
        r["note"] = note
    return r


def roofline_alu(row, flops, ms, ctx, kernel, note=None):
    """FP32-pipe bound: peak = SMs x 128 FP32 lanes x 2 (FMA) x max SM clock,
    with the FMA probe's measured rates beside it."""
    peak = fp32_peak_tflops(ctx["sms"], ctx["peaks"]["sm_max_mhz"])
    achieved = flops / (ms * 1e-3) / 1e12
    r = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
         "peak_source": f"derived: {ctx['sms']} SMs x 128 FP32 lanes x 2 x {ctx['peaks']['sm_max_mhz']:.0f} MHz",
         "kernel": kernel, "algorithmic_flops_per_launch": flops, "flops_per_test": FLOPS_PER_TEST,
         "counter": row_counter(row)}
    fma = ctx.get("fma")
    if fma:
        best = max(fma["scalar_tflops"], fma["packed_f32x2_tflops"])
        r["peak_measured"] = {"fma_probe": fma, "tflops": best, "frac_of_measured": achieved / best}
    if note:
        r["note"] = note
    return r


def cpu_rate(run_once, units_per_call, seconds, unit, sample):
    """The oracle as it stands, timed on the host cores: units per second over
    repeated calls totalling about `seconds`."""
    import oracle
    run_once()                     # warm (page-in, thread pool)
    done, k, t0 = 0.0, 0, time.perf_counter()
    while True:
        run_once()
        done += units_per_call
        k += 1
        if time.perf_counter() - t0 >= seconds:
            break
    el = time.perf_counter() - t0
    return {"value": done / el, "unit": unit, "cores": oracle.num_threads(), "kind": "oracle",
            "sample": f"{sample}; {k} calls in {el:.1f} s"}


def run_rows(torch, _lib, api, pts, H, flags, n, rp, rb, rect, args, stream, dev, ctx):
    out = {}
    reps = max(20, args.steps // 4)
    if "config0" in args.row_set:
        out.update(row_config0(torch, _lib, stream, dev, ctx))
    if "sks" in args.row_set:
        out.update(row_sks(torch, _lib, pts, H, flags, n, reps, stream, ctx))
    fixed = None
    if args.ransac_tuning:
        w, h, t = (int(x) for x in args.ransac_tuning.split(","))
        fixed = dict(block_warps=w, hyps_per_thread=h, tile_points=t)
    if "affine" in args.row_set:
        out.update(row_affine(torch, _lib, pts, n, reps, stream, ctx))
    if rp is not None:
        out.update(row_ransac1(torch, api, rp, stream, dev, ctx, fixed))
    if rb is not None and "ransac512" in args.row_set:
        out.update(row_ransac512(torch, api, rb, stream, dev, ctx, fixed, not args.no_plain))
    if rb is not None and "adaptive" in args.row_set:
        out.update(row_adaptive(torch, api, rb, stream, dev, ctx, fixed))
    if rb is not None and "refit" in args.row_set:
        out.update(row_refit(torch, _lib, api, rb, stream, dev, ctx, fixed))
    if rect is not None:
        out.update(row_diff(torch, _lib, rect, stream, dev, ctx))
    if "latency" in args.row_set:
        out.update(row_latency(torch, _lib, pts, H, n, stream, ctx))
    return out


# The paper's GPU sample numbers (Sec. 6.4, Table 8) and its ACA times on an
# RTX 3090 in FP64, microseconds; context only (other hardware and precision).
PAPER_TABLE8_ACA_US = {1: 3.11, 10: 3.16, 100: 3.19, 1000: 3.20, 10000: 5.26, 100000: 29.3, 1000000: 245.0}


def row_latency(torch, _lib, pts, H, n_total, stream, ctx):
    """aca_solve on the first m sets of the resident batch for the paper's
    sample numbers.  Device time per call: 100 calls captured in one CUDA
    graph, the graph replayed, CUDA events around the replays (host launch
    cost excluded, as in a kernel-time measurement); plus the host-side cost
    of one eager call through the Python binding.  Per size, the fraction of
    HBM bandwidth the call's 100 B per set reach (small calls are bound by
    launch latency, not bandwidth); the row's roofline is that of the
    largest size; the oracle's time per call on the host cores is timed at
    every size up to 1e5 sets."""
    import oracle
    res = {"sizes": {}}
    peak = ctx["peaks"]["hbm_gbs"]
    # Table 8's sample numbers plus the 1K-20K range of the paper's Fig. 8
    # (where its per-H time levels off, near its GPU's core count), extended
    # to 40K for GB300's 19456 FP32 lanes
    sizes = sorted(set(PAPER_TABLE8_ACA_US) | {2000, 5000, 15000, 20000, 30000, 40000})
    for m in sizes:
        if m > n_total:
            break
        f = lambda: _lib.aca_solve(pts, H, None, n=m)
        for _ in range(5):
            f()
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        s = torch.cuda.Stream()
        with torch.cuda.stream(s):
            with torch.cuda.graph(g, stream=s):
                for _ in range(100):
                    _lib.aca_solve(pts, H, None, n=m, stream=s)
        torch.cuda.synchronize()
        g.replay()
        torch.cuda.synchronize()
        t = time_region(torch, g.replay, 10, stream) / 100
        eager = time_region(torch, f, 200, stream)
        prepared = _lib.prepare_aca_solve(pts, H, None, n=m)
        prep = time_region(torch, prepared, 200, stream)
        res["sizes"][str(m)] = {"us": t * 1e3, "ns_per_set": t * 1e6 / m, "eager_call_us": eager * 1e3,
                                "prepared_call_us": prep * 1e3,
                                "hbm_frac": BYTES_PER_SET * m / (t * 1e-3) / 1e9 / peak,
                                "paper_rtx3090_fp64_us": PAPER_TABLE8_ACA_US.get(m)}
        last = (m, t)
    m, t = last
    res["unit"] = "us per call"
    res["value"] = t * 1e3
    res["value_at_sets"] = m
    kernel = "solve_scalar_kernel<ACA>" if m < (1 << 18) else "solve_ring_kernel<ACA, NONE, no flags>"
    res["roofline"] = roofline_hbm("aca_latency_sweep", BYTES_PER_SET * m, t, ctx, kernel,
                                   note=f"the largest size of the sweep ({m} sets); below 2^18 sets the library "
                                        "runs solve_scalar_kernel and a call is bound by launch latency "
                                        "(hbm_frac per size shows it); the counter is that kernel's capture")
    # the oracle's time per call, per size: about cpu_s in all
    cpu_sizes = [s for s in res["sizes"] if int(s) <= 100000]
    mmax = max(int(s) for s in cpu_sizes)
    aos = oracle.sets_aos(ctx["pts_np"][:, :mmax])
    buf = np.empty((mmax, 9))
    per_size = {}
    for s in cpu_sizes:
        k = int(s)
        r = cpu_rate(lambda: oracle.lib().oracle_aca(aos.ctypes.data_as(oracle._d), buf.ctypes.data_as(oracle._d), k),
                     1, ctx["cpu_s"] / len(cpu_sizes), "calls/s", f"FP64 ACA oracle over {k} sets")
        per_size[s] = 1e6 / r["value"]
    top = str(max(int(s) for s in cpu_sizes))
    res["cpu_baseline"] = {"value": per_size[top], "unit": "us per call", "at_sets": int(top),
                           "us_per_call_by_size": per_size, "cores": oracle.num_threads(), "kind": "oracle",
                           "sample": f"FP64 ACA oracle (Eq. 20-29) on the first m sets, m in the sweep up to "
                                     f"{top}; about {ctx['cpu_s'] / len(cpu_sizes):.2f} s per size"}
    return {"aca_latency_sweep": res}


def row_sks(torch, _lib, pts, H, flags, n, reps, stream, ctx):
    import oracle
    out = {}
    chunk = min(n, 1 << 20)
    aos = oracle.sets_aos(ctx["pts_np"][:, :chunk])
    buf = np.empty((chunk, 9))
    # SKS on the same sets
    sks = lambda: _lib.sks_solve(pts, H, None, n=n)
    for _ in range(3):
        sks()
    t = time_region(torch, sks, reps, stream)
    out["sks_solve"] = {"value": n / (t * 1e-3), "unit": "H/s", "ms": t,
                        "roofline": roofline_hbm("sks_solve", BYTES_PER_SET * n, t, ctx, "solve_ring_kernel<SKS>"),
                        "cpu_baseline": cpu_rate(lambda: oracle.lib().oracle_sks(aos.ctypes.data_as(oracle._d),
                                                                                   buf.ctypes.data_as(oracle._d), chunk),
                                                 chunk, ctx["cpu_s"], "H/s",
                                                 f"FP64 SKS oracle (Eq. 4-14) over the first {chunk} of the sets")}
    fl = lambda: _lib.aca_solve(pts, H, flags, n=n)
    for _ in range(3):
        fl()
    t = time_region(torch, fl, reps, stream)
    out["aca_solve_with_flags"] = {
        "value": n / (t * 1e-3), "unit": "H/s", "ms": t,
        "roofline": roofline_hbm("aca_solve_with_flags", (BYTES_PER_SET + 1) * n, t, ctx,
                                 "solve_ring_kernel<ACA, NONE, flags>"),
        "cpu_baseline": cpu_rate(lambda: oracle.lib().oracle_aca(aos.ctypes.data_as(oracle._d),
                                                                buf.ctypes.data_as(oracle._d), chunk),
                                 chunk, ctx["cpu_s"], "H/s",
                                 f"FP64 ACA oracle (the oracle has no flag computation) over the first {chunk} sets")}
    return out


def row_affine(torch, _lib, pts, n, reps, stream, ctx):
    """Three-point affine solve (Eq. 38) on the M, N, P points of the same
    sets: 12 float planes in, 9 out (84 B per set)."""
    import oracle
    p12 = torch.cat([pts[0:6], pts[8:14]], dim=0).contiguous()
    A = torch.empty((9, n), dtype=torch.float32, device=pts.device)
    f = lambda: _lib.aca_affine_solve(p12, A, n=n)
    for _ in range(3):
        f()
    t = time_region(torch, f, reps, stream)
    chunk = min(n, 1 << 20)
    p12h = np.concatenate([ctx["pts_np"][0:6, :chunk], ctx["pts_np"][8:14, :chunk]], axis=0)
    aos = np.ascontiguousarray(p12h.T.astype(np.float64))
    buf = np.empty((chunk, 9))
    out = {"aca_affine_solve": {
        "value": n / (t * 1e-3), "unit": "H/s", "ms": t, "bytes_per_set": 84,
        "roofline": roofline_hbm("aca_affine_solve", 84 * n, t, ctx, "affine_ring_kernel"),
        "cpu_baseline": cpu_rate(lambda: oracle.lib().oracle_aca_affine(aos.ctypes.data_as(oracle._d),
                                                                       buf.ctypes.data_as(oracle._d), chunk),
                                 chunk, ctx["cpu_s"], "H/s", f"FP64 affine oracle (Eq. 38) over the first {chunk} sets")}}
    del p12, A
    return out


def row_config0(torch, _lib, stream, dev, ctx):
    """Config 0: 4096 minimal sets, the parity configuration.  Device time per
    aca_solve from graph replays, the largest error against the FP64 oracle,
    and the oracle's ACA (O1) and independent DLT (O2) on one host thread and
    on all host cores."""
    import oracle
    ms0 = workloads.minimal_sets(4096, seed=0)
    pts0 = torch.from_numpy(ms0.pts).to(dev)
    H0 = torch.empty((9, 4096), dtype=torch.float32, device=dev)
    f = lambda: _lib.aca_solve(pts0, H0, None, n=4096)
    for _ in range(5):
        f()
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        with torch.cuda.graph(g, stream=s):
            for _ in range(100):
                _lib.aca_solve(pts0, H0, None, n=4096, stream=s)
    g.replay()
    torch.cuda.synchronize()
    t = time_region(torch, g.replay, 10, stream) / 100
    a = H0.cpu().numpy().T.astype(np.float64)
    ref = oracle.aca(ms0.pts)
    a /= np.linalg.norm(a, axis=1, keepdims=True)
    b = ref / np.linalg.norm(ref, axis=1, keepdims=True)
    a *= np.sign(np.sum(a * b, axis=1, keepdims=True))
    err = np.abs(a - b).max(axis=1)
    aos = oracle.sets_aos(ms0.pts)
    buf = np.empty((4096, 9))
    cores = oracle.num_threads()
    cpu = {}
    for name, fn in (("aca_O1", "oracle_aca"), ("dlt_O2", "oracle_dlt")):
        for thr in (1, cores):
            oracle.set_num_threads(thr)
            run = lambda: getattr(oracle.lib(), fn)(aos.ctypes.data_as(oracle._d), buf.ctypes.data_as(oracle._d), 4096)
            cpu[f"{name}_{thr}_threads"] = cpu_rate(run, 4096, min(2.0, ctx["cpu_s"]), "H/s",
                                                    f"FP64 {fn} over the 4096 config-0 sets, {thr} thread(s)")
            cpu[f"{name}_{thr}_threads"]["cores"] = thr
    oracle.set_num_threads(cores)
    return {"aca_config0_4096": {
        "value": 4096 / (t * 1e-3), "unit": "H/s", "us_per_call_device": t * 1e3,
        "max_err_vs_fp64": float(err.max()), "median_err_vs_fp64": float(np.median(err)),
        "roofline": roofline_hbm("aca_config0_4096", BYTES_PER_SET * 4096, t, ctx, "solve_scalar_kernel<ACA>",
                                 note="410 KB per call: launch/latency-bound, not HBM-bound"),
        "cpu_baseline": cpu[f"aca_O1_{cores}_threads"], "cpu_oracles": cpu}}


def row_ransac1(torch, api, rp, stream, dev, ctx, fixed=None):
    out = {}
    # fused RANSAC, one pair (config 2), graph-replayed
    from paper_2402_18008_gb300 import autotune
    corr = torch.from_numpy(rp.corr).to(dev)
    off2 = torch.tensor([0, 2000], dtype=torch.int64, device=dev)
    k2 = torch.tensor([4096], dtype=torch.int32, device=dev)
    make2 = lambda **kw: api.RansacPlan(corr, off2, k2, RANSAC_THR, SEED, 4096, **kw)
    best2 = fixed or autotune.tune(make2, 1, 2000, 4096, device=dev)[0]
    plan2 = make2(**best2).capture()
    for _ in range(5):
        plan2.replay()
    t = time_region(torch, plan2.replay, 200, stream)
    # eight such RANSACs back to back in one graph, each with its own buffers:
    # the cost of one more RANSAC once the graph launch is shared
    plans8 = [make2(**best2) for _ in range(8)]
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        for p in plans8:
            p.run()
    torch.cuda.current_stream().wait_stream(side)
    g8 = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g8):
        for p in plans8:
            p.run()
    for _ in range(3):
        g8.replay()
    t8 = time_region(torch, g8.replay, 100, stream)
    tests = 4096 * 2000
    import oracle
    cnt = np.empty(4096, np.int32)
    c = np.ascontiguousarray(rp.corr, np.float32)
    run = lambda: oracle.lib().oracle_score_problem(c.ctypes.data_as(oracle._f), 2000, 4096, RANSAC_THR, SEED, 0,
                                                    cnt.ctypes.data_as(oracle._i32), None, None, 0.0)
    out["ransac_fused_one_pair"] = {
        "value": tests / (t * 1e-3), "unit": "hyp*pts/s", "ms_per_ransac": t,
        "ms_per_ransac_8_in_one_graph": t8 / 8, "ms_per_added_ransac": (t8 - t) / 7,
        "tflops_fp32": tests * FLOPS_PER_TEST / (t * 1e-3) / 1e12, "tuning": best2,
        "roofline": roofline_alu("ransac_fused_one_pair", tests * FLOPS_PER_TEST, t, ctx, "ransac_fused_kernel",
                                 note="whole RANSAC per graph replay (one launch): sampling, solve, scoring, argmax, "
                                      "re-solve, outputs"),
        "cpu_baseline": cpu_rate(run, tests, ctx["cpu_s"], "hyp*pts/s",
                                 "brute-force FP64 scoring oracle (O5) on the same pair, 4096 hypotheses"),
        "config": "N=2000, 60% inliers, 4096 hypotheses, thr 3 px, graph replay"}
    return out


def row_ransac512(torch, api, rb, stream, dev, ctx, fixed=None, plain=True):
    out = {}
    # batched uneven RANSAC (config 3) vs 512 separate per-problem launches
    tot = int(rb.n_hyp.sum())
    Ns = rb.offsets[1:] - rb.offsets[:-1]
    tests3 = float(np.sum(rb.n_hyp.astype(np.float64) * Ns))
    corr3 = torch.from_numpy(rb.corr).to(dev)
    off3 = torch.from_numpy(rb.offsets).to(dev)
    k3 = torch.from_numpy(rb.n_hyp).to(dev)
    from paper_2402_18008_gb300 import autotune
    make3 = lambda **kw: api.RansacPlan(corr3, off3, k3, RANSAC_THR, SEED, tot, **kw)
    best3 = fixed or autotune.tune(make3, len(rb.n_hyp), int(rb.offsets[-1]), tot, device=dev)[0]
    plan3 = make3(**best3).capture()
    for _ in range(3):
        plan3.replay()
    t3 = time_region(torch, plan3.replay, 20, stream)
    res = {"value": tests3 / (t3 * 1e-3), "unit": "hyp*pts/s", "ms_batched": t3,
           "tflops_fp32": tests3 * FLOPS_PER_TEST / (t3 * 1e-3) / 1e12, "tests": tests3, "hypotheses": tot,
           "points": int(rb.offsets[-1]), "tuning": best3,
           "config": "512 pairs, N log-uniform [200,8000], eps U[0.1,0.9], adaptive hypotheses (99%, cap 16384), "
                     "one graph replay",
           "roofline": roofline_alu("ransac_batched_512", tests3 * FLOPS_PER_TEST, t3, ctx, "ransac_score_kernel"),
           "cpu_baseline": cpu_ransac_pairs(rb, ctx["cpu_s"])}
    if not plain:
        out["ransac_batched_512"] = res
        return out
    plains = []
    for p in range(len(rb.n_hyp)):
        a, b = int(rb.offsets[p]), int(rb.offsets[p + 1])
        plains.append(api.RansacPlan(corr3[a:b], torch.tensor([0, b - a], dtype=torch.int64, device=dev),
                                     k3[p:p + 1], RANSAC_THR, SEED, int(rb.n_hyp[p]), problem_base=p))

    def run_plain():
        for pl in plains:
            pl.run()
    run_plain()
    tp = time_region(torch, run_plain, 3, stream)
    # check: batched == plain (best hypothesis per problem)
    same = all(int(pl.best_hyp.item()) == int(plan3.best_hyp[p].item()) for p, pl in enumerate(plains))
    res.update(ms_512_plain_launches=tp, speedup_vs_plain=tp / t3, batched_equals_plain=same)
    out["ransac_batched_512"] = res
    return out


ADAPTIVE_CAP = 16384


def cpu_ransac_pairs(rb, seconds, cap=None):
    """The brute-force FP64 RANSAC oracle (O5) over the batch's pairs in
    order, as many as fit in about `seconds`: hypothesis x point tests per
    second (with `cap`, the adaptive oracle, which scores every one of the
    cap hypotheses and then finds the sequential stop)."""
    import oracle
    done, k, t0 = 0.0, 0, time.perf_counter()
    P = len(rb.n_hyp)
    while k < P:
        a, b = int(rb.offsets[k]), int(rb.offsets[k + 1])
        if cap is None:
            oracle.ransac(rb.corr[a:b], [0, b - a], rb.n_hyp[k:k + 1], RANSAC_THR, SEED, problem_base=k,
                          want_counts=False)
            done += float(rb.n_hyp[k]) * (b - a)
        else:
            oracle.ransac_adaptive(rb.corr[a:b], [0, b - a], [cap], RANSAC_THR, SEED, 0.99, problem_base=k,
                                   want_band=False)
            done += float(cap) * (b - a)
        k += 1
        if time.perf_counter() - t0 >= seconds:
            break
    el = time.perf_counter() - t0
    what = "adaptive FP64 RANSAC oracle (scores all cap hypotheses, then the sequential stop)" if cap else \
        "brute-force FP64 RANSAC oracle (O5)"
    return {"value": done / el, "unit": "hyp*pts/s", "cores": oracle.num_threads(), "kind": "oracle",
            "sample": f"{what} over the first {k} of the {P} pairs ({el:.1f} s)"}


def row_adaptive(torch, api, rb, stream, dev, ctx, fixed=None):
    """Batched RANSAC with the online adaptive stop (99% confidence) over the
    512 pairs with the same cap for every pair (no knowledge of the inlier
    ratio), against fixed counts: the cap for every pair, and counts computed
    from the generated inlier ratios (the batched row's workload)."""
    P = len(rb.n_hyp)
    Ns = (rb.offsets[1:] - rb.offsets[:-1]).astype(np.float64)
    corr = torch.from_numpy(rb.corr).to(dev)
    off = torch.from_numpy(rb.offsets).to(dev)
    caps_np = np.full(P, ADAPTIVE_CAP, np.int32)
    caps = torch.from_numpy(caps_np).to(dev)
    tot = int(caps_np.sum())
    from paper_2402_18008_gb300 import autotune
    k = torch.from_numpy(rb.n_hyp).to(dev)
    make = lambda **kw: api.RansacPlan(corr, off, k, RANSAC_THR, SEED, int(rb.n_hyp.sum()), **kw)
    best = fixed or autotune.tune(make, P, int(rb.offsets[-1]), int(rb.n_hyp.sum()), device=dev)[0]
    make_a = lambda **kw: api.RansacPlan(corr, off, caps, RANSAC_THR, SEED, tot, confidence=0.99, **kw)
    best_a = fixed or autotune.tune(make_a, P, int(rb.offsets[-1]), tot, device=dev, tag="adaptive")[0]
    res = {"unit": "ms per batch", "pairs": P, "cap": ADAPTIVE_CAP, "confidence": 0.99, "tuning": best_a,
           "tuning_fixed_count": best,
           "config": "512 pairs, N log-uniform [200,8000], eps U[0.1,0.9]; one graph replay each"}
    plans = {"adaptive": make_a(**best_a),
             "fixed_cap": api.RansacPlan(corr, off, caps, RANSAC_THR, SEED, tot, **best),
             "fixed_from_true_ratio": make(**best)}
    for name, plan in plans.items():
        plan.capture()
        for _ in range(3):
            plan.replay()
        res[f"ms_{name}"] = time_region(torch, plan.replay, 10 if name == "fixed_cap" else 20, stream)
    ne = plans["adaptive"].n_evaluated.cpu().numpy().astype(np.float64)
    res.update(hypotheses_evaluated=int(ne.sum()), tests_evaluated=float(np.sum(ne * Ns)),
               median_evaluated=float(np.median(ne)), max_evaluated=int(ne.max()),
               hypotheses_fixed_from_true_ratio=int(rb.n_hyp.sum()),
               value=res["ms_adaptive"], speedup_vs_fixed_cap=res["ms_fixed_cap"] / res["ms_adaptive"])
    res["roofline"] = roofline_alu("ransac_adaptive_512", res["tests_evaluated"] * FLOPS_PER_TEST, res["ms_adaptive"],
                                   ctx, "ransac_score_kernel<adaptive>",
                                   note="useful work: the tests of the hypotheses the sequential loop evaluates")
    res["cpu_baseline"] = cpu_ransac_pairs(rb, ctx["cpu_s"], cap=ADAPTIVE_CAP)
    return {"ransac_adaptive_512": res}


def row_refit(torch, _lib, api, rb, stream, dev, ctx, fixed=None):
    """Refit on all inliers (aca_refit) over the 512 pairs of the batched
    RANSAC workload: with the generated inlier masks alone (DLT only and DLT
    + 10 LM steps), and appended to the batched RANSAC in one CUDA graph."""
    P = len(rb.n_hyp)
    corr = torch.from_numpy(rb.corr).to(dev)
    off = torch.from_numpy(rb.offsets).to(dev)
    mask = torch.from_numpy(rb.is_inlier.astype(np.uint8)).to(dev)
    H = torch.empty((P, 9), dtype=torch.float32, device=dev)
    used = int(rb.is_inlier.sum())
    res = {"unit": "used points/s", "pairs": P, "used_points": used,
           "config": "512 pairs, N log-uniform [200,8000], eps U[0.1,0.9]; masks = generated inliers"}
    for iters in (0, 10):
        f = lambda: _lib.aca_refit(corr, off, H, mask=mask, lm_iters=iters)
        for _ in range(3):
            f()
        t = time_region(torch, f, 20, stream)
        res[f"ms_lm{iters}"] = t
        if iters == 10:
            res["value"] = used / (t * 1e-3)
    tot = int(rb.n_hyp.sum())
    k = torch.from_numpy(rb.n_hyp).to(dev)
    from paper_2402_18008_gb300 import autotune
    make = lambda **kw: api.RansacPlan(corr, off, k, RANSAC_THR, SEED, tot, **kw)
    best = fixed or autotune.tune(make, P, int(rb.offsets[-1]), tot, device=dev)[0]
    times = {}
    for name, kw in (("ransac_only", {"want_mask": True}), ("ransac_plus_refit", {"refit_iters": 10})):
        plan = make(**best, **kw).capture()
        for _ in range(3):
            plan.replay()
        times[name] = time_region(torch, plan.replay, 20, stream)
    # the paper's stages 3-5 without knowing the inlier ratios: the online
    # adaptive stop (99 %, cap 16384 per pair) and the refit, one graph
    # (with the adaptive plan's own launch shape: the tuner's entry for it,
    # cached by the adaptive row when that ran first)
    caps = torch.full((P,), ADAPTIVE_CAP, dtype=torch.int32, device=dev)
    make_a = lambda **kw: api.RansacPlan(corr, off, caps, RANSAC_THR, SEED, ADAPTIVE_CAP * P, confidence=0.99, **kw)
    best_a = fixed or autotune.tune(make_a, P, int(rb.offsets[-1]), ADAPTIVE_CAP * P, device=dev, tag="adaptive")[0]
    plan = api.RansacPlan(corr, off, caps, RANSAC_THR, SEED, ADAPTIVE_CAP * P, confidence=0.99, refit_iters=10,
                          **best_a).capture()
    for _ in range(3):
        plan.replay()
    times["adaptive_plus_refit"] = time_region(torch, plan.replay, 20, stream)
    res.update(ms_ransac_with_mask=times["ransac_only"], ms_ransac_plus_refit=times["ransac_plus_refit"],
               refit_share_of_pipeline=1.0 - times["ransac_only"] / times["ransac_plus_refit"],
               ms_adaptive_ransac_plus_refit=times["adaptive_plus_refit"], tuning_adaptive=best_a,
               us_per_pair_adaptive_ransac_plus_refit=times["adaptive_plus_refit"] * 1e3 / P)
    # compulsory traffic: every correspondence (16 B) and mask byte read once,
    # 9 floats + 2 ints written per pair
    npts = int(rb.offsets[-1])
    res["roofline"] = roofline_hbm("refit_512", 17 * npts + 44 * P, res["ms_lm10"], ctx, "refit_kernel",
                                   note="latency-bound: per-problem passes and serial solves, not HBM traffic")
    import oracle
    done, k, t0 = 0.0, 0, time.perf_counter()
    while k < P:
        a, b = int(rb.offsets[k]), int(rb.offsets[k + 1])
        oracle.refit(rb.corr[a:b], [0, b - a], rb.is_inlier[a:b], 10)
        done += float(rb.is_inlier[a:b].sum())
        k += 1
        if time.perf_counter() - t0 >= ctx["cpu_s"]:
            break
    el = time.perf_counter() - t0
    res["cpu_baseline"] = {"value": done / el, "unit": "used points/s", "cores": 1, "kind": "oracle",
                           "sample": f"float64 refit oracle (normalised DLT + 10 LM steps, numpy, one thread) over "
                                     f"the first {k} of the {P} pairs ({el:.1f} s)"}
    return {"refit_512": res}


def row_diff(torch, _lib, rect, stream, dev, ctx):
    out = {}
    # differentiable rectangle ACA (config 4): forward + backward vs plain solve
    B = rect.tgt.shape[1]
    tgt = torch.from_numpy(rect.tgt).to(dev)
    Hr = torch.empty((9, B), dtype=torch.float32, device=dev)
    gH = torch.randn((9, B), dtype=torch.float32, device=dev)
    gT = torch.empty((8, B), dtype=torch.float32, device=dev)

    def fwd_bwd():
        _lib.aca_rect_solve(tgt, rect.rect, Hr)
        _lib.aca_rect_backward(tgt, rect.rect, gH, gT)
    src = np.repeat(rect.src_corners.reshape(8, 1), B, axis=1).astype(np.float32)
    pts4 = torch.from_numpy(np.concatenate([src, rect.tgt], axis=0)).to(dev)
    Hg = torch.empty((9, B), dtype=torch.float32, device=dev)
    plain = lambda: _lib.aca_solve(pts4, Hg, None, n=B)
    # comparison: the same Eq. 42 as plain torch tensor operations with torch
    # autograd for the backward (one kernel per operation)
    tgt_t = tgt.clone().requires_grad_(True)

    def torch_fwd_bwd():
        x0, y0, w, r = (float(v) for v in rect.rect)
        Mx, My, Nx, Ny, Px, Py, Qx, Qy = tgt_t
        MPx, MPy, MQx, MQy = Px - Mx, Py - My, Qx - Mx, Qy - My
        q4x = MQx * MPy - MQy * MPx
        q4y = (Nx - Mx) * MQy - (Ny - My) * MQx
        t2 = (Px - Nx) * (Qy - Ny) - (Py - Ny) * (Qx - Nx)
        b13, b23, b33 = -q4x * x0, -r * q4y * y0, -t2 * (x0 + r * y0 + w)
        Ht = torch.stack([Nx * q4x + Mx * t2, Px * r * q4y + Mx * r * t2, Nx * b13 + Px * b23 + Mx * b33,
                          Ny * q4x + My * t2, Py * r * q4y + My * r * t2, Ny * b13 + Py * b23 + My * b33,
                          q4x + t2, r * q4y + r * t2, b13 + b23 + b33])
        tgt_t.grad = None
        (Ht * gH).sum().backward()
    for f in (fwd_bwd, plain, torch_fwd_bwd):
        for _ in range(5):
            f()
    fwd_p = _lib.prepare_aca_rect_solve(tgt, rect.rect, Hr)
    bwd_p = _lib.prepare_aca_rect_backward(tgt, rect.rect, gH, gT)

    def fwd_bwd_prepared():
        fwd_p()
        bwd_p()
    fwd_bwd_prepared()
    tfb = time_region(torch, fwd_bwd, 200, stream)
    tfp = time_region(torch, fwd_bwd_prepared, 200, stream)
    tpl = time_region(torch, plain, 200, stream)
    ttt = time_region(torch, torch_fwd_bwd, 50, stream)
    # device time: 50 forward + backward pairs captured in one CUDA graph
    g = torch.cuda.CUDAGraph()
    s = torch.cuda.Stream()
    torch.cuda.synchronize()
    with torch.cuda.stream(s):
        with torch.cuda.graph(g, stream=s):
            for _ in range(50):
                _lib.aca_rect_solve(tgt, rect.rect, Hr, stream=s)
                _lib.aca_rect_backward(tgt, rect.rect, gH, gT, stream=s)
    g.replay()
    torch.cuda.synchronize()
    tdev = time_region(torch, g.replay, 10, stream) / 50
    # the same pair at 2^24 sets (the vectorised kernels, 2.8 GB per pair,
    # larger than L2): whether the kernels reach the HBM roofline once the
    # batch is no longer launch-bound
    BL = 1 << 24
    tgtL = torch.from_numpy(np.ascontiguousarray(np.tile(rect.tgt, (1, BL // B)))).to(dev)
    HrL = torch.empty((9, BL), dtype=torch.float32, device=dev)
    gHL = torch.randn((9, BL), dtype=torch.float32, device=dev)
    gTL = torch.empty((8, BL), dtype=torch.float32, device=dev)
    gL = torch.cuda.CUDAGraph()
    torch.cuda.synchronize()
    with torch.cuda.stream(s):
        with torch.cuda.graph(gL, stream=s):
            for _ in range(5):
                _lib.aca_rect_solve(tgtL, rect.rect, HrL, stream=s)
                _lib.aca_rect_backward(tgtL, rect.rect, gHL, gTL, stream=s)
    gL.replay()
    torch.cuda.synchronize()
    tdevL = time_region(torch, gL.replay, 4, stream) / 5
    del tgtL, HrL, gHL, gTL, gL
    import oracle
    tg = np.ascontiguousarray(rect.tgt.T.astype(np.float64))
    x0, y0, w, r = (float(v) for v in rect.rect)
    Hbuf = np.empty((B, 9))
    Jbuf = np.empty((B, 9, 8))
    gHh = gH.cpu().numpy().T.astype(np.float64)

    def cpu_fwd_bwd():
        oracle.lib().oracle_aca_rect(tg.ctypes.data_as(oracle._d), x0, y0, w, r, Hbuf.ctypes.data_as(oracle._d), B)
        oracle.lib().oracle_aca_rect_jacobian(tg.ctypes.data_as(oracle._d), x0, y0, w, r,
                                              Jbuf.ctypes.data_as(oracle._d), B)
        np.einsum("nik,ni->nk", Jbuf, gHh)
    out["diff_aca_rect_65536"] = {
        "value": B / (tfb * 1e-3), "unit": "sets/s (fwd+bwd, eager calls)",
        "ms_fwd_bwd": tfb, "ms_fwd_bwd_prepared_calls": tfp, "ms_fwd_bwd_device": tdev,
        "sets_per_s_device": B / (tdev * 1e-3),
        "ms_plain_aca_solve": tpl, "ratio_vs_plain": tfb / tpl,
        "ms_torch_ops_autograd_fwd_bwd": ttt, "speedup_vs_torch_ops": ttt / tfb,
        # forward 32 B in + 36 out, backward 32 + 36 in + 32 out, per set
        "roofline": roofline_hbm("diff_aca_rect_65536", 168 * B, tdev, ctx,
                                 "rect_scalar_kernel + rect_backward_scalar_kernel",
                                 note="11 MB per forward + backward: latency-bound at this batch (below 2^18 "
                                      "sets the library runs one set per thread)"),
        "large_batch": {"sets": BL, "ms_fwd_bwd_device": tdevL, "sets_per_s_device": BL / (tdevL * 1e-3),
                        "roofline": roofline_hbm("diff_aca_rect_large", 168 * BL, tdevL, ctx,
                                                 "rect_vec4_kernel + rect_backward_vec4_kernel",
                                                 note="the same forward + backward pair at 2^24 sets, one graph "
                                                      "of 5 pairs; inputs larger than L2")},
        "cpu_baseline": cpu_rate(cpu_fwd_bwd, B, ctx["cpu_s"], "sets/s",
                                 "FP64 Eq. 42 forward + analytic Jacobian oracle and its product with dL/dH, "
                                 f"{B} sets")}
    return out


if __name__ == "__main__":
    main()
