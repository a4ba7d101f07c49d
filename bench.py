#!/usr/bin/env python3
"""Benchmark of the FNR impulse filter on GB300.

Workload: the 640x512 14-bit sweep (seeded synthetic IR frames: T^4 thermal
field, sigma 8 DN sensor noise, hot lines and 2x2 targets, salt-and-pepper
density 5/10/20/40%, windows 3x3/5x5/7x7: 12 distinct frames). One step
filters a batch of those 12 frames replicated R times (default 32: 384
frames, 125.8 Mpx, 252 MB in + 252 MB out, larger than L2, so no flush is
needed) with one launch of the batch plan's CUDA graph.

Prints one JSON line: Mpx/s (whole job), the roofline of the dominant
kernel, per-window numbers, the plain per-frame path, the end-to-end number
through host buffers, clocks sampled during the timed region, and the CPU
oracle timed on the host cores (which also checks the GPU output of one
replica bit for bit).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--replicas R] [--impl reference]
"""
from __future__ import annotations

import argparse
import atexit
import json
import os
import statistics
import subprocess
import sys
import tempfile
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "filtered Mpixel/s per window k (bit-exact vs oracle); p99 frame latency served"
UNIT = "Mpixel/s"
L2_BYTES = 129 * 10**6
WORKLOAD = "640x512 14-bit sweep: salt-and-pepper 5/10/20/40%, windows 3/5/7"


def recorded_profile():
    """The committed ncu record of the class kernels, or None when the kernel
    sources changed since that capture."""
    import hashlib
    p = os.path.join(ROOT, "profiles", "traffic_sweep_640x512_u14.json")
    if not os.path.exists(p):
        return None
    with open(p) as fh:
        rec = json.load(fh)
    h = hashlib.sha1()
    for src in rec["kernel_sources"]:
        with open(os.path.join(ROOT, src), "rb") as fh:
            h.update(fh.read())
    return rec if h.hexdigest() == rec["kernel_sources_sha1"] else None


def recorded_traffic(k: str, frames: int):
    """DRAM bytes per launch of the class-k kernel from the committed ncu record
    (scaled by the frames of the launch), or None."""
    rec = recorded_profile()
    if rec is None or k not in rec["bytes_per_frame"]:
        return None
    return int(rec["bytes_per_frame"][k]) * frames


def recorded_large_k_profile():
    """The committed ncu record of the large-window class kernels (ALU-pipe
    and issue utilisation per k), or None when their sources changed since."""
    import hashlib
    p = os.path.join(ROOT, "profiles", "alu_large_k_1280x1024_u14.json")
    if not os.path.exists(p):
        return None
    with open(p) as fh:
        rec = json.load(fh)
    h = hashlib.sha1()
    for src in rec["kernel_sources"]:
        with open(os.path.join(ROOT, src), "rb") as fh:
            h.update(fh.read())
    return rec if h.hexdigest() == rec["kernel_sources_sha1"] else None


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as fh:
            d = json.load(fh)
        return float(d.get("hbm_gbs", 6800.0)), "measured"
    return 6800.0, "fallback"


# ---------------------------------------------------------------------------
# clocks
# ---------------------------------------------------------------------------
class ClockSampler:
    """nvidia-smi samples every 200 ms while the timed region runs."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(prefix="clocks", suffix=".csv")
            os.close(fd)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.fh, stderr=subprocess.DEVNULL)
            # never outlive the bench (a profiler waits for every process it started)
            atexit.register(self._end)
        except Exception:
            self.proc = None

    def _end(self):
        if self.proc is not None and self.proc.poll() is None:
            self.proc.kill()
            self.proc.wait()

    def stop(self):
        out = {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        if self.proc is None:
            return out
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
            self.proc.wait()
        self.fh.close()
        sms, maxes, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as fh:
            for line in fh:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sms.append(float(parts[1]))
                    maxes.append(float(parts[2]))
                except ValueError:
                    continue
                for name, val in zip(names, parts[5:9]):
                    if val.lower() == "active":
                        reasons.add(name)
        os.unlink(self.path)
        if sms:
            out["sm_mhz"] = statistics.median(sms)
            out["sm_max_mhz"] = max(maxes)
        out["reasons"] = sorted(reasons)
        out["samples"] = len(sms)
        return out


# ---------------------------------------------------------------------------
# workload
# ---------------------------------------------------------------------------
def bench_config(replicas: int) -> dict:
    """The workload as both arms name it (the same dict for the reference arm)."""
    nframes = 12 * replicas
    frame_bytes = 640 * 512 * 2
    return {"workload": WORKLOAD, "frame": "640x512 uint16 14-bit", "frames_per_step": nframes,
            "replicas": replicas, "mpx_per_step": round(nframes * 640 * 512 / 1e6, 3),
            "l2": (f"inputs {nframes * frame_bytes / 1e6:.0f} MB per step > 129 MB L2 (no flush needed)"
                   if nframes * frame_bytes > L2_BYTES else
                   f"inputs {nframes * frame_bytes / 1e6:.0f} MB per step fit in the 129 MB L2 (small run)")
            + f"; side legs flush L2 ({2 * L2_BYTES // 10**6} MB write) before each of {LEG_ITERS} timed launches",
            "parallelism": "frames sharded per GPU, no collective"}


# The paper's own timings (Table 1, Sec. 4) with their hardware: context
# only, a different workload (one 364x244 8-bit image) on other hardware.
PAPER_CONTEXT = {
    "source": "Table 1 (Sec. 4): Matlab on an Intel Core 2 E6600 (2.4 GHz, 2 cores), one 364x244 8-bit IR image",
    "fnr_ms": {"20pct": 15, "30pct": 18}, "mf_ms": 24,
    "fnr_mpx_s_derived": {"20pct": 5.9, "30pct": 4.9},
    "sorts": {"20pct": 24587, "30pct": 30832, "of_pixels": 88816},
}


def build_workload(replicas: int):
    from paper_1201_3972_gb300 import synth
    specs = synth.workload_sweep_u14()
    frames = [s.make() for s in specs]
    return specs, frames


LEG_ITERS = 100   # timed iterations of each side leg (median reported)
_flush_buf = None


def flush_l2(torch, stream):
    """Overwrite a buffer twice the size of L2 on `stream`, so the next timed
    launch finds none of its inputs or outputs in L2."""
    global _flush_buf
    if _flush_buf is None:
        _flush_buf = torch.empty(2 * L2_BYTES // 4, dtype=torch.int32, device="cuda")
    with torch.cuda.stream(stream):
        _flush_buf.fill_(0)


def time_events(torch, fn, steps: int, stream, flush: bool = False) -> list:
    """Per-step durations (ms) measured with CUDA events on `stream`; with
    `flush`, L2 is flushed before every step, outside the events."""
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    for a, b in evs:
        if flush:
            flush_l2(torch, stream)
        a.record(stream)
        fn()
        b.record(stream)
    torch.cuda.synchronize()
    return [a.elapsed_time(b) for a, b in evs]


def own_arm(args):
    import torch
    import torch.distributed as dist

    from paper_1201_3972_gb300 import _build, _lib, synth

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0")) % max(1, torch.cuda.device_count())
    if world > 1:
        # frames are independent: nothing on the data path is collective; the
        # process group only carries the barriers and the max over ranks
        dist.init_process_group("gloo")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    _build.build()
    flt = _lib.Filter(local)
    stream = torch.cuda.current_stream()

    specs, frames = build_workload(args.replicas)
    R = args.replicas
    H, W = frames[0].shape
    fpx = H * W
    nframes = len(frames) * R
    frame_bytes = fpx * 2
    # one contiguous buffer per direction; frame i at offset i * frame_bytes (pitch W*2 = 1280 B)
    host_in = np.concatenate([f.reshape(-1) for f in frames] * R).view(np.int16)
    d_in = torch.from_numpy(host_in).to(dev)
    d_out = torch.empty_like(d_in)
    base_in, base_out = int(d_in.data_ptr()), int(d_out.data_ptr())

    def descs_for(indices, counter=None):
        arr = (_lib.ir_frame_desc * len(indices))()
        for j, i in enumerate(indices):
            s = specs[i % len(specs)]
            arr[j].in_ = base_in + i * frame_bytes
            arr[j].out = base_out + i * frame_bytes
            arr[j].H, arr[j].W = H, W
            arr[j].in_pitch = arr[j].out_pitch = W * 2
            arr[j].dtype = _lib.IR_U14
            arr[j].k = s.k
            arr[j].flagged_count = counter
        return arr

    all_idx = list(range(nframes))
    # the autotuner picks each class's strategy and tile on these frames
    # (--no-tune, for profiling runs: the library's default table)
    tuned = {} if args.no_tune else \
        {str(r["k"]): r for r in flt.autotune_batch(descs_for(all_idx), reps=20, stream=stream)}
    plan = _lib.BatchPlan(flt, descs_for(all_idx))
    launches_per_step = plan.kernel_count
    step_px = nframes * fpx

    # warm-up, then the timed region (barrier + sync on both sides, max over ranks)
    for _ in range(args.warmup):
        plan.launch(stream)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clocks = ClockSampler(local)
    clocks.start()
    l0 = flt.launch_count()
    torch.cuda.synchronize()
    t_start = torch.cuda.Event(enable_timing=True)
    t_end = torch.cuda.Event(enable_timing=True)
    t_start.record(stream)
    for _ in range(args.steps):
        plan.launch(stream)
    t_end.record(stream)
    torch.cuda.synchronize()
    total_ms = t_start.elapsed_time(t_end)
    gpu_launches = flt.launch_count() - l0
    if world > 1:  # launches of the whole job
        lt = torch.tensor([gpu_launches], dtype=torch.int64)
        dist.all_reduce(lt, op=dist.ReduceOp.SUM)
        gpu_launches = int(lt.item())
    if world > 1:
        dist.barrier()
    if args.profile_only:
        # profiling runs (under ncu): the step and, if asked, the large-window
        # leg; the line carries only what was run
        clocks.stop()
        ms_step = total_ms / args.steps
        out = {"metric": METRIC, "value": round(world * step_px / (ms_step * 1e-3) / 1e6, 1), "unit": UNIT,
               "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms_step, 4),
               "profile_only": args.profile_only, "config": bench_config(R)}
        if args.profile_only == "large_k" and rank == 0:
            out["large_k"] = large_k_leg(flt, stream, args)
        if rank == 0:
            print(json.dumps(out), flush=True)
        plan.close()
        flt.close()
        if world > 1:
            dist.barrier()
            dist.destroy_process_group()
        return
    # per-window classes timed alone (the dominant-kernel roofline comes from these)
    per_k = {}
    hbm_peak, peak_kind = peaks()
    for k in (3, 5, 7):
        idx = [i for i in all_idx if specs[i % len(specs)].k == k]
        sub = _lib.BatchPlan(flt, descs_for(idx))
        for _ in range(args.warmup):
            sub.launch(stream)
        durs = time_events(torch, lambda: sub.launch(stream), max(args.steps, LEG_ITERS), stream, flush=True)
        ms = statistics.median(durs)
        px = len(idx) * fpx
        algo_bytes = px * 2 * 2  # read + write, 2 bytes per pixel
        sub.close()
        # the flagged fraction of the class (one counted run, untimed)
        ctr = torch.zeros(1, dtype=torch.int64, device=dev)
        counted = _lib.BatchPlan(flt, descs_for(idx, int(ctr.data_ptr())))
        counted.launch(stream)
        torch.cuda.synchronize()
        counted.close()
        per_k[str(k)] = {"mpx_s": px / (ms * 1e-3) / 1e6, "ms": ms, "frames": len(idx),
                         "achieved_gbs": algo_bytes / (ms * 1e-3) / 1e9,
                         "hbm_frac": algo_bytes / (ms * 1e-3) / 1e9 / hbm_peak,
                         "flagged_fraction": int(ctr.item()) / px,
                         "config": flt.get_config(_lib.IR_U14, k)}
    clk = clocks.stop()

    # the directional detector (Fig. 1) on the same window classes: throughput
    # and flagged fraction (its parity with the oracle is in the test suite)
    directional = {}
    if rank == 0 and not args.no_directional:
        flt.set_detector("directional")
        try:
            for k in (3, 5, 7):
                idx = [i for i in all_idx if specs[i % len(specs)].k == k]
                sub = _lib.BatchPlan(flt, descs_for(idx))
                for _ in range(args.warmup):
                    sub.launch(stream)
                ms = statistics.median(time_events(torch, lambda: sub.launch(stream), max(args.steps, LEG_ITERS),
                                                   stream, flush=True))
                sub.close()
                ctr = torch.zeros(1, dtype=torch.int64, device=dev)
                counted = _lib.BatchPlan(flt, descs_for(idx, int(ctr.data_ptr())))
                counted.launch(stream)
                torch.cuda.synchronize()
                counted.close()
                px = len(idx) * fpx
                directional[str(k)] = {"mpx_s": round(px / (ms * 1e-3) / 1e6, 1), "ms": round(ms, 4),
                                       "flagged_fraction": round(int(ctr.item()) / px, 4),
                                       "extreme_detector_mpx_s": round(per_k[str(k)]["mpx_s"], 1)}
        finally:
            flt.set_detector("extreme")

    # plain per-frame path on the same frames (one ir_filter_run2 per frame)
    def plain_step():
        for i in all_idx:
            s = specs[i % len(specs)]
            flt.ir_filter_run2(base_in + i * frame_bytes, W * 2, base_out + i * frame_bytes, W * 2, H, W,
                               _lib.IR_U14, s.k, stream.cuda_stream, None)
    plain_step()
    pl = time_events(torch, plain_step, 3, stream)
    plain_mpx = step_px / (statistics.median(pl) * 1e-3) / 1e6

    # end to end through the library's host-frame call: every step copies all
    # inputs from pinned host memory to the device, filters them and copies
    # the outputs back (ir_filter_run_host: chunks of whole frames pipelined
    # through copy-in, filter and copy-out streams, so one chunk's copies
    # overlap another's filtering and the two copy directions overlap each other)
    h_in = torch.from_numpy(host_in).pin_memory()
    h_out = torch.empty_like(h_in).pin_memory()
    hb_in, hb_out = int(h_in.data_ptr()), int(h_out.data_ptr())
    host_descs = (_lib.ir_frame_desc * nframes)()
    for i in range(nframes):
        host_descs[i].in_ = hb_in + i * frame_bytes
        host_descs[i].out = hb_out + i * frame_bytes
        host_descs[i].H, host_descs[i].W = H, W
        host_descs[i].in_pitch = host_descs[i].out_pitch = W * 2
        host_descs[i].dtype = _lib.IR_U14
        host_descs[i].k = specs[i % len(specs)].k
        host_descs[i].flagged_count = None
    n_chunks = args.e2e_chunks

    def e2e_step():
        flt.ir_filter_run_host(host_descs, nframes, n_chunks, stream)
    e2e_step()
    plan.launch(stream)  # the device result of the same frames, for the read-back check
    torch.cuda.synchronize()
    e2e_ok = bool(torch.equal(h_out, d_out.cpu()))
    e2e_steps = max(3, min(args.steps, 10))
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        e2e_step()
    torch.cuda.synchronize()
    e2e_s = (time.perf_counter() - t0) / e2e_steps

    ms_step = total_ms / args.steps
    if world > 1:
        t = torch.tensor([ms_step], dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms_step = float(t.item())
    value = world * step_px / (ms_step * 1e-3) / 1e6

    # dominant kernel = the window class with the largest share of the step
    dom_k = max(per_k, key=lambda kk: per_k[kk]["ms"])
    dom = per_k[dom_k]
    prof = recorded_profile() or {}
    roofline = {"bound": "hbm", "kernel": f"fnr_kernel k={dom_k} u16 ({_lib.ALGO_NAMES[dom['config']['algo']]})",
                "achieved": round(dom["achieved_gbs"], 1), "peak": hbm_peak, "unit": "GB/s",
                "frac": round(dom["achieved_gbs"] / hbm_peak, 4),
                "traffic": recorded_traffic(dom_k, dom["frames"]),
                # what does bind it, from the same ncu record (percent of peak)
                "alu_pipe_pct_ncu": prof.get("alu_pipe_pct", {}).get(dom_k),
                "issue_active_pct_ncu": prof.get("issue_active_pct", {}).get(dom_k),
                "peak_kind": f"{peak_kind} copy bandwidth (burst)",
                # every window class of the step, each timed alone (fraction of the same peak)
                "class_frac": {f"k{k}": round(v["hbm_frac"], 4) for k, v in per_k.items()},
                "plain_per_frame_mpx_s": round(plain_mpx, 1),
                # the tuner's choice per class and its margin over the default configuration
                "tuned": {f"k{k}": tune_summary(r) for k, r in tuned.items()}}

    result = {
        "metric": METRIC, "value": round(value, 1), "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(ms_step, 4), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u16", "data": "synthetic (seeded T^4 thermal field + impulses)",
        "config": bench_config(R),
        "roofline": roofline,
        "e2e": {"value": round(world * step_px / e2e_s / 1e6, 1), "unit": UNIT, "call": "ir_filter_run_host",
                "chunks": n_chunks, "streams": 3,
                "readback_equals_device_result": e2e_ok,
                "h2d_bytes_per_step": nframes * frame_bytes, "d2h_bytes_per_step": nframes * frame_bytes},
        "gpu_launches": int(gpu_launches), "launches_per_step": launches_per_step,
        "clocks": {"sm_mhz": clk["sm_mhz"], "sm_max_mhz": clk["sm_max_mhz"], "reasons": clk["reasons"]},
        "paper_context": PAPER_CONTEXT,
        "per_k": {k: {"mpx_s": round(v["mpx_s"], 1), "ms": round(v["ms"], 4), "hbm_frac": round(v["hbm_frac"], 4),
                      "flagged": round(v["flagged_fraction"], 4), "algo": _lib.ALGO_NAMES[v["config"]["algo"]],
                      "tile": f"{v['config']['tile_w']}x{v['config']['tile_h']}"}
                  for k, v in per_k.items()},
    }
    if directional:
        result["directional_detector"] = directional
    if rank == 0:
        result["single_frame"] = single_frame_leg(flt, stream, args)
    if rank == 0 and not args.no_batch_leg:
        bm = batch_leg(flt, stream, args)
        result["batch_mixed"] = bm
        roofline["batch_k3_k5_frac"] = bm["k3_k5"]["hbm_frac"]
        roofline["batch_all_frac"] = bm["all"]["hbm_frac"]
    if rank == 0 and not args.no_large_k:
        lk = large_k_leg(flt, stream, args)
        result["large_k"] = lk
        # the large windows are bound by integer ALU work: their ALU-pipe
        # utilisation from the committed ncu record of the same sources
        lrec = recorded_large_k_profile() or {}
        roofline["large_k_alu_pipe_pct_ncu"] = lrec.get("alu_pipe_pct")
    if rank == 0 and not args.no_quality:
        from paper_1201_3972_gb300 import quality
        t1 = quality.table1(flt)
        result["table1_synthetic"] = {key: {"psnr_noisy_mf_fnr": [v["noisy_psnr"], v["mf1_psnr"], v["fnr1_psnr"]],
                                            "sorts_fnr": v["fnr1_sorts"][0]} for key, v in t1.items()}
        dr = quality.detail_retention(flt)
        result["detail_retention"] = {f"k{k}": {"fnr_kept": dr[f"k{k}"]["fnr"]["structure"]["kept"],
                                                "mf_kept": dr[f"k{k}"]["mf"]["structure"]["kept"]} for k in (3, 5, 7)}
    ref_hashes = None
    if rank == 0 and not args.no_cpu_baseline:
        plan.launch(stream)  # the output buffer holds the timed step's result, whatever the legs wrote since
        torch.cuda.synchronize()
        result["cpu_baseline"], result["parity"], ref_hashes = cpu_baseline(frames, specs, d_out, fpx, args)
    if rank == 0 and args.serve_seconds > 0:
        result["serve"] = serve_leg(args, local, ref_hashes)
    if rank == 0:
        result["summary"] = summary(result)
        print(json.dumps(result), flush=True)
    plan.close()
    flt.close()
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()


def tune_summary(r: dict) -> str:
    """'<algo> <tile> x<speedup over the default>/<candidates timed>', plus the
    default's name when the tuner chose something else."""
    from paper_1201_3972_gb300 import _lib
    c, d = r["chosen"], r["defaults"]
    sp = r["default_ms"] / r["chosen_ms"] if r["chosen_ms"] > 0 else float("nan")
    name = lambda x: f"{_lib.ALGO_NAMES[x['algo']]} {x['tile_w']}x{x['tile_h']}"
    same = (c["algo"], c["tile_w"], c["tile_h"]) == (d["algo"], d["tile_w"], d["tile_h"])
    return f"{name(c)} x{sp:.3f}/{r['candidates']}" + ("" if same else f" (default {name(d)})")


def summary(r: dict) -> dict:
    """The figures the gates are read from, repeated compactly at the end of
    the line (HBM fractions of the measured copy bandwidth)."""
    out = {"value_mpx_s": r["value"], "e2e_mpx_s": r["e2e"]["value"],
           "class_frac": r["roofline"]["class_frac"],
           "plain_per_frame_mpx_s": r["roofline"]["plain_per_frame_mpx_s"]}
    if "batch_mixed" in r:
        out["batch_k3_k5"] = {"mpx_s": r["batch_mixed"]["k3_k5"]["mpx_s"], "frac": r["batch_mixed"]["k3_k5"]["hbm_frac"],
                              "target_frac": 0.6}
        out["batch_all"] = {"mpx_s": r["batch_mixed"]["all"]["mpx_s"], "frac": r["batch_mixed"]["all"]["hbm_frac"]}
    if "serve" in r:
        sv = r["serve"]
        out["serve"] = {"p50_ms": sv["latency_ms"]["p50"], "p99_ms": sv["latency_ms"]["p99"], "mpx_s": sv["mpx_s"],
                        "seconds": sv["seconds"], "verified": sv["verified"], "mismatches": sv["mismatches"],
                        "verified_against": sv["verified_against"]}
    if "parity" in r:
        out["oracle_parity"] = r["parity"]["bit_exact"]
    return out


def batch_leg(flt, stream, args):
    """The mixed batch: 256 frames, sizes 160x120..1920x1080, u8 and 14-bit,
    windows 3/5/7/9/15, 5-30% salt-and-pepper, one graph launch per step;
    also its k=3/5 subset (the HBM-bound classes)."""
    import torch
    from paper_1201_3972_gb300 import _lib, synth
    specs = synth.workload_batch()
    frames = [s.make() for s in specs]
    bufs = []
    for f in frames:
        src = torch.from_numpy(f.view(np.int16) if f.dtype == np.uint16 else f).cuda()
        bufs.append((src, torch.empty_like(src)))
    out = {}
    every = flt.make_descs([{"in": bufs[i][0], "out": bufs[i][1], "k": s.k, "u14": s.dtype == synth.U14}
                            for i, s in enumerate(specs)])
    tuned = [] if args.no_tune else flt.autotune_batch(every, reps=20, stream=stream)
    out["tuned"] = {f"{'u8' if r['dtype'] == _lib.IR_U8 else 'u16'} k{r['k']}": tune_summary(r) for r in tuned}
    # each (pixel type, k) class alone: where the mixed batch's time goes
    alone = {}
    for key in sorted({(s.dtype == synth.U8, s.k) for s in specs}):
        idx = [i for i, s in enumerate(specs) if (s.dtype == synth.U8, s.k) == key]
        plan = flt.plan([{"in": bufs[i][0], "out": bufs[i][1], "k": specs[i].k, "u14": specs[i].dtype == synth.U14}
                         for i in idx])
        for _ in range(args.warmup):
            plan.launch(stream)
        alone[f"{'u8' if key[0] else 'u16'} k{key[1]}"] = round(statistics.median(
            time_events(torch, lambda: plan.launch(stream), LEG_ITERS // 2, stream, flush=True)), 4)
        plan.close()
    out["classes_alone_ms"] = alone
    out["classes_alone_sum_ms"] = round(sum(alone.values()), 4)
    for name, sel in (("all", lambda s: True), ("k3_k5", lambda s: s.k in (3, 5))):
        idx = [i for i, s in enumerate(specs) if sel(s)]
        plan = flt.plan([{"in": bufs[i][0], "out": bufs[i][1], "k": specs[i].k, "u14": specs[i].dtype == synth.U14}
                         for i in idx])
        for _ in range(args.warmup):
            plan.launch(stream)
        durs = time_events(torch, lambda: plan.launch(stream), max(LEG_ITERS, args.steps), stream, flush=True)
        ms = statistics.median(durs)
        px = sum(specs[i].pixels for i in idx)
        byts = sum(2 * specs[i].pixels * specs[i].esize for i in idx)
        hbm, _ = peaks()
        out[name] = {"frames": len(idx), "mpx": round(px / 1e6, 1), "ms": round(ms, 4),
                     "mpx_s": round(px / ms / 1e3, 1), "hbm_frac": round(byts / (ms * 1e-3) / 1e9 / hbm, 4),
                     "kernels_per_launch": plan.kernel_count}
        plan.close()
    return out


def single_frame_leg(flt, stream, args):
    """One 320x240 u8 frame, 10% salt-and-pepper, k = 3, one ir_filter_run2
    call per frame: launch-latency bound, so reported in microseconds (device
    time between events around the call, and host wall time of the call with
    its synchronisation)."""
    import torch
    from paper_1201_3972_gb300 import _lib, synth
    s = synth.workload_single_u8()[0]
    f = s.make()
    src = torch.from_numpy(f).cuda()
    dst = torch.empty_like(src)
    H, W = f.shape

    def once():
        flt.ir_filter_run2(int(src.data_ptr()), W, int(dst.data_ptr()), W, H, W, _lib.IR_U8, 3,
                           stream.cuda_stream, None)
    for _ in range(max(3, args.warmup)):
        once()
    dev_us = 1e3 * statistics.median(time_events(torch, once, LEG_ITERS, stream, flush=True))
    torch.cuda.synchronize()
    walls = []
    for _ in range(50):
        t0 = time.perf_counter()
        once()
        stream.synchronize()
        walls.append(time.perf_counter() - t0)
    wall_us = 1e6 * statistics.median(walls)
    return {"frame": "320x240 u8, 10% salt-and-pepper, k=3", "device_us": round(dev_us, 2),
            "wall_us": round(wall_us, 2), "mpx_s": round(H * W / dev_us, 1)}


def large_k_leg(flt, stream, args):
    """The large windows: 1280x1024 14-bit frames with 20% random-valued
    impulses, k = 9/13/17/21, each window class timed alone on 8 copies of its
    frame (these kernels are bound by integer ALU work, not HBM)."""
    import torch
    from paper_1201_3972_gb300 import _lib, synth
    hbm, _ = peaks()
    out = {}
    copies = 8
    for s in synth.workload_large_k():
        f = s.make()
        H, W = f.shape
        src = torch.from_numpy(np.concatenate([f.reshape(-1)] * copies).view(np.int16)).cuda()
        dst = torch.empty_like(src)
        fb = H * W * 2
        arr = (_lib.ir_frame_desc * copies)()
        for j in range(copies):
            arr[j].in_ = int(src.data_ptr()) + j * fb
            arr[j].out = int(dst.data_ptr()) + j * fb
            arr[j].H, arr[j].W = H, W
            arr[j].in_pitch = arr[j].out_pitch = W * 2
            arr[j].dtype = _lib.IR_U14
            arr[j].k = s.k
            arr[j].flagged_count = None
        tr = None if args.no_tune else flt.autotune_batch(arr, reps=20, stream=stream)[0]
        plan = _lib.BatchPlan(flt, arr)
        for _ in range(args.warmup):
            plan.launch(stream)
        ms = statistics.median(time_events(torch, lambda: plan.launch(stream), max(LEG_ITERS, args.steps), stream,
                                           flush=True))
        px = copies * H * W
        out[str(s.k)] = {"frames": copies, "ms": round(ms, 4), "mpx_s": round(px / ms / 1e3, 1),
                         "hbm_frac": round(px * 4 / (ms * 1e-3) / 1e9 / hbm, 4),
                         "tuned": tune_summary(tr) if tr else "default table (--no-tune)"}
        plan.close()
    return out


def serve_leg(args, device, oracle_hashes=None):
    """64 simulated 30 fps streams (320x240 / 640x512 / 1280x1024, 14-bit,
    10% impulses, windows 3/5/7) served by the continuous-batching server:
    open-loop latency with every served output hashed and compared, closed-loop
    saturation throughput, and the plain one-frame-per-launch path on the same
    traffic. The expected hashes are the oracle's (from the CPU-baseline leg)
    when it ran, else those of the plain entry point."""
    from paper_1201_3972_gb300 import serve, synth
    streams = synth.workload_serve(streams=64, pool=args.serve_pool)
    pools = serve.make_pools(streams)
    if oracle_hashes is not None:
        ref, against = oracle_hashes, "oracle"
    else:
        ref, against = serve.reference_hashes(pools, streams, device), "plain entry point (no oracle run)"
    live = serve.simulate(streams, args.serve_seconds, pools, ref, verify_every=1, device=device)
    sat_s = min(3.0, args.serve_seconds)
    sat = serve.drive(streams, pools, sat_s, inflight=4, device=device)
    plain = serve.drive(streams, pools, sat_s, plain=True, device=device)
    return {"streams": 64, "fps_per_stream": 30, "seconds": live["duration_s"],
            "latency_ms": live["latency_ms"], "mpx_s": live["mpx_s"],
            "frames": live["frames_completed"], "dropped": live["frames_dropped_busy"],
            "mean_batch_frames": live["mean_batch_frames"], "max_inflight_batches": live["max_inflight_batches"],
            "verified": live["verified"], "mismatches": live["mismatches"], "verified_against": against,
            "distinct_frames_hashed": len(ref),
            "saturation_mpx_s": sat["mpx_s"], "saturation_batch_frames": sat["mean_batch_frames"],
            "plain_per_frame_saturation_mpx_s": plain["mpx_s"],
            "workload": "64 streams x 30 fps Poisson, 320x240/640x512/1280x1024 u14, k 3/5/7, 10% impulses"}


def cpu_baseline(frames, specs, d_out, fpx, args):
    """The oracle, as it stands, on all host cores over one replica of the
    12 sweep frames (repeated until about 10 s of CPU work); its outputs
    also check replica 0 of the GPU result bit for bit. Unless serving is
    skipped, the oracle also filters every distinct frame the serving leg
    submits (each (resolution, pool frame, window) once, untimed), whose
    hashes the served outputs are checked against."""
    import oracle
    cores = os.cpu_count() or 1
    gpu = d_out[: len(frames) * fpx].cpu().numpy().view(np.uint16).reshape(len(frames), *frames[0].shape)
    exact = 0
    px = 0
    t0 = time.perf_counter()
    reps = 0
    while True:
        for i, (f, s) in enumerate(zip(frames, specs)):
            out, _ = oracle.fnr_mt(f, s.k, cores)
            if reps == 0:
                exact += int(np.array_equal(out, gpu[i]))
            px += f.size
        reps += 1
        if time.perf_counter() - t0 > args.cpu_seconds or reps >= 50:
            break
    dt = time.perf_counter() - t0
    base = {"value": round(px / dt / 1e6, 2), "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{reps} pass(es) over the 12 distinct 640x512 sweep frames ({px / 1e6:.1f} Mpx), "
                      f"C oracle, row bands over {cores} threads"}
    parity = {"frames_checked": len(frames), "bit_exact": exact == len(frames)}
    hashes = None
    if args.serve_seconds > 0:
        from paper_1201_3972_gb300 import serve, synth
        streams = synth.workload_serve(streams=64, pool=args.serve_pool)
        hashes = {}
        for si, k in sorted({(s.size_index, s.k) for s in streams}):
            pool = streams[[s.size_index for s in streams].index(si)].pool
            for j, spec in enumerate(synth.serve_pool(si, pool)):
                hashes[(si, j, k)] = serve.frame_hash(oracle.fnr_mt(spec.make(), k, cores)[0])
    return base, parity, hashes


def reference_arm(args):
    """The oracle run as the reference implementation on the host cores, on
    this arm's workload, metric and unit; each step is one pass over the 12
    distinct sweep frames."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle
    from paper_1201_3972_gb300 import synth
    specs = synth.workload_sweep_u14()
    frames = [s.make() for s in specs]
    cores = os.cpu_count() or 1
    oracle.build()

    def step():
        for f, s in zip(frames, specs):
            oracle.fnr_mt(f, s.k, cores)
    for _ in range(args.warmup):
        step()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        step()
    dt = (time.perf_counter() - t0) / args.steps
    px = sum(f.size for f in frames)
    value = px / dt / 1e6
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": round(value, 2), "unit": UNIT,
        "n_gpus": int(os.environ.get("WORLD_SIZE", "1")),
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(dt * 1e3, 2), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u16", "data": "synthetic",
        "config": bench_config(args.replicas),
        "cpu_baseline": {"value": round(value, 2), "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": "one pass over the 12 distinct sweep frames per step (a bounded sample of the "
                                   f"{12 * args.replicas}-frame step; Mpx/s over the frames filtered)"},
        "e2e": {"value": round(value, 2), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


def main():
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--replicas", type=int, default=32)
    ap.add_argument("--impl", default="own", choices=["own", "reference"])
    ap.add_argument("--cpu-seconds", type=float, default=10.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--serve-seconds", type=float, default=60.0, help="serving leg duration (0 = skip)")
    ap.add_argument("--no-batch-leg", action="store_true", help="skip the 256-frame mixed batch")
    ap.add_argument("--no-large-k", action="store_true", help="skip the k = 9..21 windows on 1280x1024 frames")
    ap.add_argument("--no-quality", action="store_true", help="skip the Table 1 style PSNR comparison")
    ap.add_argument("--no-directional", action="store_true", help="skip the directional-detector leg")
    ap.add_argument("--e2e-chunks", type=int, default=16, help="pipeline chunks of the end-to-end host-frame call")
    ap.add_argument("--no-tune", action="store_true",
                    help="skip the autotuner and run the library's default table (profiling runs)")
    ap.add_argument("--profile-only", choices=["step", "large_k"], default=None,
                    help="profiling runs: the timed step only, or the step and the large-window leg")
    ap.add_argument("--serve-pool", type=int, default=30, help="pre-generated frames per resolution")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.impl == "reference":
        reference_arm(args)
    else:
        own_arm(args)


if __name__ == "__main__":
    main()
