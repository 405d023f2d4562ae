#!/usr/bin/env python
"""Mojette encode/decode benchmark on GB300 (one JSON line on rank 0).

Workload (default "plain_at_scale"): 262144 stripes of 8 KB (Q = 4 lines of
P = 256 uint64 pixels, uniform random from a seed), n = 6 projections with
p in {-3,-2,-1,1,2,3}. One step = encode every stripe, then decode every
stripe under each of the 15 two-erasure patterns (16 kernel launches).
Metric: user-data GB/s = stripes * 8192 B * 16 / step time.

Timing: W warm-up steps, then K steps between a barrier + synchronize on
both sides, CUDA events on the launching stream around every launch, max
over ranks. Inputs (2.1 GB image, 3.3 GB projections) exceed the 129 MB L2,
so no flush is needed between steps.

The same line carries, unless switched off:
  wide     the (12,8) geometry the paper's Sec. 3.1 also measures: 262144
           stripes at 8 KB (Q=8, P=128) and at 4 KB (Q=8, P=64), encode and
           15 sampled four-erasure decodes, each kernel's ms and fraction of
           the HBM roofline;
  alternatives  the opt-in decode kernels on the same workloads: decode_ilv
           (the path with stripes across lanes) and decode_vander (Eq. 1 as
           a Vandermonde system: not the paper's inverse, reported apart);
  e2e      the step through the C ABI from pinned host buffers, copies timed
           (decode inputs: only the surviving projections' slices);
  batched  500000 mixed stripes (4 KB / 8 KB x (3,2), (6,4), (12,8), 0..n-k
           erasures each) as two CUDA-graph launches per step, against the
           same work as plain per-(geometry, mask) launches;
  served   the request server under closed-loop and Poisson load (p50/p99),
           against the same requests served one at a time;
  systematic  (with --systematic) the systematic form (data lines stored
           as they are, parity projections): parity encode and in-place
           decode per number of lost data lines, 8 KB stripes of (6,4) and
           (12,8);
  cpu_baseline  the oracle on the host cores, on a bounded sample, one
           thread and all cores.

Decode bytes (the HBM roofline): every bin of the Q projections the path
uses (sum of their B_i) read, plus the Q * P pixels written; encode bytes:
the Q * P pixels read plus every bin written.

--impl reference times the CPU oracle (the slow plain implementation the
tests compare against) on the host cores, on bounded samples of the same
workload: it is the reported baseline arm, not a target.
"""
from __future__ import annotations

import argparse
import hashlib
import itertools
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_1504_07038_gb300 import inputs  # noqa: E402

SIX = [-3, -2, -1, 1, 2, 3]
TWELVE = [v for v in range(-6, 7) if v]
WORKLOADS = {
    "plain_at_scale": dict(P=256, Q=4, p=SIX, S=262144, erasures=2,
                           desc="262144 stripes x 8 KB (Q=4, P=256 uint64), (6,4) p=+-1..3; "
                                "encode + decode under all 15 two-erasure masks"),
    "profile_8k": dict(P=256, Q=4, p=SIX, S=32768, erasures=2, mask_sample=1,
                       desc="32768 stripes x 8 KB (Q=4, P=256), (6,4); encode + 1 two-erasure decode "
                            "(small case for ncu captures; 268 MB image > L2)"),
    "profile_wide8k": dict(P=128, Q=8, p=TWELVE, S=32768, erasures=4, mask_sample=1,
                           desc="32768 stripes x 8 KB (Q=8, P=128), (12,8); encode + 1 four-erasure decode "
                                "(small case for ncu captures; 268 MB image > L2)"),
    "profile_wide4k": dict(P=64, Q=8, p=TWELVE, S=65536, erasures=4, mask_sample=1,
                           desc="65536 stripes x 4 KB (Q=8, P=64), (12,8); encode + 1 four-erasure decode "
                                "(small case for ncu captures; 268 MB image > L2)"),
    "plain": dict(P=128, Q=4, p=SIX, S=1024, erasures=2,
                  desc="1024 stripes x 4 KB (Q=4, P=128), (6,4); encode + 15 two-erasure decodes"),
    "wide_4k": dict(P=64, Q=8, p=TWELVE, S=262144, erasures=4, mask_sample=15,
                    desc="262144 stripes x 4 KB (Q=8, P=64), (12,8); encode + 15 four-erasure decodes"),
    "wide_8k": dict(P=128, Q=8, p=TWELVE, S=262144, erasures=4, mask_sample=15,
                    desc="262144 stripes x 8 KB (Q=8, P=128), (12,8); encode + 15 four-erasure decodes"),
}
# Mixed batch: 4 KB and 8 KB stripes of the (3,2), (6,4) and (12,8) codes.
BATCH_GEOMS = [(256, 2, [-1, 1, 2]), (512, 2, [-1, 1, 2]), (128, 4, SIX), (256, 4, SIX),
               (64, 8, TWELVE), (128, 8, TWELVE)]
BATCHED = dict(S=500000,
                            desc="500000 stripes, seeded mix of 4 KB / 8 KB x (3,2) p={-1,1,2}, (6,4) "
                                 "p=+-1..3, (12,8) p=+-1..6, 0..n-k seeded erasures each, random order; "
                                 "one step = encode every stripe, then decode every stripe")
METRIC = "Mojette encode/decode user-data GB/s & % HBM roofline; batched vs plain, 1 GB300"
KERNEL_SOURCES = ["encode_kernels.cuh", "decode_kernels.cuh", "encode.cu", "decode.cu", "ptx.cuh",
                  "mojette_internal.h"]


def decode_kernel_name(plan, mask, S) -> str:
    """The decode kernel the library launches for this plan, mask and size."""
    from paper_1504_07038_gb300 import binding as mj
    return mj.mojette_decode_kernel(plan, mask, S)


def workload_masks(w):
    n = len(w["p"])
    ms = inputs.all_masks(n, w["erasures"])
    k = w.get("mask_sample")
    if k and len(ms) > k:
        ms = ms[:: len(ms) // k][:k]
    return ms


def kernel_hash() -> str:
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        with open(os.path.join(ROOT, "paper_1504_07038_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def ncu_traffic(kernel: str, workload: str):
    """Per-launch DRAM bytes from the committed ncu summary, if it was taken
    on the current kernel sources; else None."""
    path = os.path.join(ROOT, "profiles", "dram_traffic.json")
    try:
        with open(path) as f:
            d = json.load(f)
        e = d[workload][kernel]
        if e.get("kernel_hash") != kernel_hash():
            return None
        return float(e["bytes_per_launch"])
    except Exception:
        return None


class ClockSampler:
    """nvidia-smi clocks and throttle reasons during the timed region."""
    Q = ("index,uuid,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, uuid: str | None):
        self.uuid = uuid
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                                          "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL,
                                         text=True)
        except Exception:
            self.proc = None
            return
        self.t = threading.Thread(target=self._read, daemon=True)
        self.t.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.t.join(timeout=5)
        rows = []
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 10:
                continue
            if self.uuid and parts[1] != self.uuid and len({r.split(",")[1] for r in self.lines if "," in r}) > 1:
                continue
            rows.append(parts)
        if not rows:
            return None
        sm = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        smax = [float(r[3]) for r in rows if r[3].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[6 + k].lower() == "active"})
        loaded = [v for v in sm if smax and v > 0.5 * max(smax)] or sm
        return {"sm_mhz": statistics.median(loaded) if loaded else None,
                "sm_max_mhz": max(smax) if smax else None, "reasons": reasons, "samples": len(rows)}


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def replica_first_stripe(rank: int, S: int) -> int:
    """Replicas: rank r encodes and decodes stripes r*S .. r*S + S - 1 of the
    seeded stream (weak scaling: the same work per GPU, disjoint data, no
    exchange between ranks)."""
    return rank * S


def max_over_ranks(x: float, dist=None) -> float:
    """The slowest rank's time (every rank gets it); x itself on one GPU."""
    if dist is None:
        return x
    import torch
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ------------------------------------------------------------------ GPU arm --

def workload_config(args, w, world):
    """The `config` of the JSON line (both arms): the workload, not the
    implementation."""
    return {"workload": args.workload, "description": w["desc"], "stripes": w["S"],
            "block_bytes": w["Q"] * w["P"] * 8, "Q": w["Q"], "P": w["P"], "n": len(w["p"]), "p": w["p"],
            "decode_masks": len(workload_masks(w)), "launches_per_step": 1 + len(workload_masks(w)),
            "l2": "inputs larger than L2 (no flush)", "parallelism": f"replicas x{world}"}


def decode_bytes(plan, masks, S):
    """Algorithmic HBM bytes of one decode launch per mask: every bin of the
    Q projections the path uses (the sum of their B_i) read, and the Q * P
    pixels written."""
    from paper_1504_07038_gb300 import binding as mj
    out = []
    for m in masks:
        sc = mj.mojette_schedule(plan, m)
        used = set(sc["left"]) | set(sc["right"])
        out.append(S * 8 * (sum(int(plan.bins[i]) for i in used) + plan.Q * plan.P))
    return out


def time_launches(fn, reps, stream):
    """Median CUDA-event time (ms) of fn() on `stream` over reps launches
    (after one untimed launch)."""
    import torch
    fn()
    ts = []
    for _ in range(reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        fn()
        e1.record(stream)
        ts.append((e0, e1))
    torch.cuda.synchronize()
    return statistics.median(a.elapsed_time(b) for a, b in ts)


def with_kernel(name):
    """Context manager: MOJETTE_DECODE_KERNEL set to name (read at every
    plain launch) for the duration."""
    class _K:
        def __enter__(self):
            self.old = os.environ.get("MOJETTE_DECODE_KERNEL")
            os.environ["MOJETTE_DECODE_KERNEL"] = name

        def __exit__(self, *exc):
            if self.old is None:
                os.environ.pop("MOJETTE_DECODE_KERNEL", None)
            else:
                os.environ["MOJETTE_DECODE_KERNEL"] = self.old
    return _K()


def kernel_stats(ms, bytes_, user, peak, traffic=None):
    gbs = bytes_ / (ms * 1e-3) / 1e9
    return {"ms": round(ms, 4), "hbm_gbs": round(gbs, 1), "frac": round(gbs / peak, 4),
            "user_gbs": round(user / (ms * 1e-3) / 1e9, 1), "algorithmic_bytes_per_launch": int(bytes_),
            "traffic": traffic}


def alt_decodes(plan, d_img, d_proj, d_out, masks, S, dbytes, user, peak, stream, reps=3):
    """The opt-in decode kernels on a workload: ms (mean over masks of the
    median over reps) and fraction of the roofline, each checked exact."""
    import torch
    from paper_1504_07038_gb300 import binding as mj
    out = {}
    for name, what in (("ilv", "the Sec. 2.2 path, stripes across lanes (one lane per stripe, front and "
                                "half of the lines)"),
                       ("vander", "Eq. 1 solved as a Vandermonde system: exact, not the paper's inverse")):
        with with_kernel(name):
            kname = mj.mojette_decode_kernel(plan, masks[0], S)
            if kname != "decode_" + name:
                continue
            d_out.zero_()
            ms = [time_launches(lambda m=m: mj.mojette_decode(plan, d_proj, m, d_out, S, stream), reps, stream)
                  for m in masks]
        out[kname] = kernel_stats(statistics.mean(ms), statistics.mean(dbytes), user, peak)
        out[kname]["exact"] = bool(torch.equal(d_out, d_img))
        out[kname]["what"] = what
    return out


def run_workload(args, w, name, peak, stream, rank, timed_steps, clocks=None, keep=False):
    """Encode every stripe, then decode every stripe under each of the
    workload's masks, timed per launch with CUDA events on `stream`.
    Returns (result dict, buffers or None)."""
    import torch
    from paper_1504_07038_gb300 import binding as mj

    P, Q, p, S = w["P"], w["Q"], w["p"], w["S"]
    masks = workload_masks(w)
    plan = mj.mojette_plan(P, Q, p)
    img_np = inputs.stripes(S, Q, P, seed=args.seed, first=replica_first_stripe(rank, S))
    h_img = torch.from_numpy(img_np.view(np.int64)).pin_memory()
    del img_np
    d_img = h_img.cuda()
    d_proj = torch.empty((S, plan.total), dtype=torch.int64, device="cuda")
    d_out = torch.empty((S, Q, P), dtype=torch.int64, device="cuda")
    launches = 1 + len(masks)

    def mk():
        return torch.cuda.Event(enable_timing=True)

    def step(ev=None):
        if ev:
            ev[0][0].record(stream)
        mj.mojette_encode(plan, d_img, d_proj, S, stream)
        if ev:
            ev[0][1].record(stream)
        for k, m in enumerate(masks):
            if ev:
                ev[1 + k][0].record(stream)
            mj.mojette_decode(plan, d_proj, m, d_out, S, stream)
            if ev:
                ev[1 + k][1].record(stream)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    mj.mojette_device_status()        # raises if any bounded wait expired
    exact = bool(torch.equal(d_out, d_img))
    events = [[(mk(), mk()) for _ in range(launches)] for _ in range(timed_steps)]
    if clocks:
        clocks.start()
        time.sleep(0.4)
    t0, t1 = mk(), mk()
    t0.record(stream)
    for k in range(timed_steps):
        step(events[k])
    t1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop() if clocks else None
    mj.mojette_device_status()
    enc_ms = statistics.mean(e[0][0].elapsed_time(e[0][1]) for e in events)
    by_mask = [statistics.median(e[1 + k][0].elapsed_time(e[1 + k][1]) for e in events)
               for k in range(len(masks))]
    dec_ms = statistics.mean(by_mask)
    user = S * Q * P * 8
    dbytes = decode_bytes(plan, masks, S)
    enc_bytes = S * (Q * P + plan.total) * 8
    dec_name = decode_kernel_name(plan, masks[0], S)
    traffic_key = name if not args.stripes else None
    kern = {"encode_tiles": kernel_stats(enc_ms, enc_bytes, user, peak, ncu_traffic("encode_tiles", traffic_key)),
            dec_name: kernel_stats(dec_ms, statistics.mean(dbytes), user, peak, ncu_traffic(dec_name, traffic_key))}
    kern[dec_name]["path_bytes_per_launch"] = S * 2 * Q * P * 8
    kern[dec_name]["ms_by_mask"] = {"min": round(min(by_mask), 4), "max": round(max(by_mask), 4),
                                    "max_over_min": round(max(by_mask) / min(by_mask), 4), "masks": len(masks)}
    res = {"total_ms": t0.elapsed_time(t1), "steps": timed_steps, "launches_per_step": launches,
           "user_bytes": user, "kernels": kern, "decode_kernel": dec_name, "exact": exact,
           "clocks": clk, "masks": masks, "dec_bytes": dbytes, "plan": plan,
           "desc": w["desc"], "stripes": S}
    if not args.no_alternatives:
        res["alternatives"] = alt_decodes(plan, d_img, d_proj, d_out, masks, S, dbytes, user, peak, stream)
    bufs = (plan, h_img, d_img, d_proj, d_out, masks) if keep else None
    if not keep:
        del d_img, d_proj, d_out, h_img
        torch.cuda.empty_cache()
    return res, bufs


def run_gpu(args, w):
    import torch
    from paper_1504_07038_gb300 import binding as mj

    world, rank, local = dist_setup()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    stream = torch.cuda.current_stream()
    peak, peak_kind = measured_peaks()

    def barrier():
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        torch.cuda.synchronize()

    uuid = None
    try:
        uuid = str(torch.cuda.get_device_properties(local).uuid)
        uuid = uuid if uuid.startswith("GPU-") else "GPU-" + uuid
    except Exception:
        pass
    barrier()
    main, bufs = run_workload(args, w, args.workload, peak, stream, rank, args.steps, ClockSampler(uuid), keep=True)
    barrier()
    total_ms = max_over_ranks(main["total_ms"], dist)

    # end to end through the C ABI with host buffers (pinned), copies timed
    plan, h_img, d_img, d_proj, d_out, masks = bufs
    e2e = None if args.no_e2e else run_e2e(args, w, plan, h_img, d_img, d_proj, d_out, masks, stream)
    del bufs, h_img, d_img, d_proj, d_out
    torch.cuda.empty_cache()

    if rank != 0:
        if dist:
            dist.barrier()
            dist.destroy_process_group()
        return None

    S, Q, P, p = w["S"], w["Q"], w["P"], w["p"]
    ms_step = total_ms / args.steps
    launches = main["launches_per_step"]
    value = world * main["user_bytes"] * launches / (ms_step * 1e-3) / 1e9
    dec_name = main["decode_kernel"]
    dk = main["kernels"][dec_name]
    line = {
        "metric": METRIC,
        "value": round(value, 3),
        "unit": "GB/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": round(ms_step, 4),
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "u64",
        "data": "synthetic (seeded SplitMix64 uniform uint64 pixels)",
        "config": workload_config(args, w, world),
        "roofline": {"bound": "hbm", "kernel": dec_name, "achieved": dk["hbm_gbs"],
                     "peak": peak, "unit": "GB/s", "frac": dk["frac"],
                     "peak_kind": f"{peak_kind} (copy bandwidth, burst)",
                     "traffic": dk["traffic"],
                     "algorithmic_bytes_per_launch": dk["algorithmic_bytes_per_launch"],
                     "bytes": "sum of B_i over the Q projections the path uses, read, + Q*P pixels written"},
        "kernels": main["kernels"],
        "exact": main["exact"],
        "gpu_launches": args.steps * launches,
        "clocks": main["clocks"],
        "e2e": e2e,
    }
    if "alternatives" in main:
        line["alternatives"] = main["alternatives"]
    if not args.no_wide and args.workload == "plain_at_scale":
        line["wide"] = {}
        for wl in ("wide_8k", "wide_4k"):
            ww = dict(WORKLOADS[wl])
            r, _ = run_workload(args, ww, wl, peak, stream, rank, max(3, min(args.steps, 10)))
            line["wide"][wl] = {"description": ww["desc"], "decode_kernel": r["decode_kernel"],
                                "kernels": r["kernels"], "exact": r["exact"],
                                "step_user_gbs": round(r["user_bytes"] * r["launches_per_step"] /
                                                       (r["total_ms"] / r["steps"] * 1e-3) / 1e9, 1)}
            if "alternatives" in r:
                line["wide"][wl]["alternatives"] = r["alternatives"]
    if not args.no_batched:
        line["batched"] = run_batched(args, rank)
    if not args.no_served:
        line["served"] = run_served(args, rank)
    if args.systematic:
        line["systematic"] = run_systematic(args, rank)
    if world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(w, main["masks"], budget_s=args.cpu_seconds)
    if dist:
        dist.barrier()
        dist.destroy_process_group()
    return line


def run_e2e(args, w, plan, h_img, d_img, d_proj, d_out, masks, stream):
    """Same metric through the C ABI with host buffers: every step copies the
    image in and the projections out (encode), then for each mask the
    projections the decode reads in (mojette_stage_survivors: the Q
    surviving projections' slices, what a storage read fetches) and the
    image out, from/to pinned host memory. Three streams -- host-to-device
    copies, kernels, device-to-host copies -- ordered by events, so that
    both copy directions run back to back while the kernels run; the stripes
    are cut into `chunks` slices, and the decode's input and output buffers
    are doubled (mask k uses buffer k mod 2), so the copies of one mask
    overlap the decode of the next. Decode reads a separate device buffer,
    filled with junk before the timed region, so the round-trip check shows
    the copied data is what is used."""
    import torch
    from paper_1504_07038_gb300 import binding as mj

    S, Q, P = w["S"], w["Q"], w["P"]
    h_proj = torch.empty((S, plan.total), dtype=torch.int64).pin_memory()
    h_out = torch.empty((S, Q, P), dtype=torch.int64).pin_memory()
    d_in = [torch.full((S, plan.total), 0x0BAD0BAD0BAD0BAD, dtype=torch.int64, device="cuda")
            for _ in range(2)]
    d_o = [d_out, torch.empty_like(d_out)]
    chunks = args.e2e_chunks
    s_in, s_k, s_out = torch.cuda.Stream(), torch.cuda.Stream(), torch.cuda.Stream()
    bounds = [(S * c // chunks, S * (c + 1) // chunks) for c in range(chunks)]
    staged = [0]
    ev = lambda: torch.cuda.Event()   # noqa: E731
    # per slice, the last event that used each buffer (carried across steps)
    last = {key: [None] * chunks for key in ("enc", "proj", "stage_done", "dec0", "dec1", "out0", "out1")}

    def after(st, e):
        if e is not None:
            st.wait_event(e)

    def step():
        staged[0] = 0
        e_proj = [None] * chunks
        for c, (a, b) in enumerate(bounds):
            after(s_in, last["enc"][c])                 # d_img slice free
            with torch.cuda.stream(s_in):
                d_img[a:b].copy_(h_img[a:b], non_blocking=True)
                e_img = ev(); e_img.record(s_in)
            s_k.wait_event(e_img)
            after(s_k, last["proj"][c])                 # d_proj slice copied out
            with torch.cuda.stream(s_k):
                mj.mojette_encode(plan, d_img[a:b], d_proj[a:b], b - a, s_k)
                e_enc = ev(); e_enc.record(s_k)
            last["enc"][c] = e_enc
            s_out.wait_event(e_enc)
            after(s_out, last["stage_done"][c])         # h_proj slice no longer read
            with torch.cuda.stream(s_out):
                h_proj[a:b].copy_(d_proj[a:b], non_blocking=True)
                e = ev(); e.record(s_out)
            e_proj[c] = e
            last["proj"][c] = e
        for k, m in enumerate(masks):
            j = k % 2
            for c, (a, b) in enumerate(bounds):
                s_in.wait_event(e_proj[c])
                after(s_in, last[f"dec{j}"][c])         # d_in[j] slice read by its last decode
                with torch.cuda.stream(s_in):
                    staged[0] += mj.mojette_stage_survivors(plan, h_proj[a:b], m, d_in[j][a:b], b - a, s_in)
                    e_st = ev(); e_st.record(s_in)
                last["stage_done"][c] = e_st
                s_k.wait_event(e_st)
                after(s_k, last[f"out{j}"][c])          # d_o[j] slice copied out
                with torch.cuda.stream(s_k):
                    mj.mojette_decode(plan, d_in[j][a:b], m, d_o[j][a:b], b - a, s_k)
                    e_d = ev(); e_d.record(s_k)
                last[f"dec{j}"][c] = e_d
                s_out.wait_event(e_d)
                with torch.cuda.stream(s_out):
                    h_out[a:b].copy_(d_o[j][a:b], non_blocking=True)
                    e_o = ev(); e_o.record(s_out)
                last[f"out{j}"][c] = e_o

    def fork():
        for st in (s_in, s_k, s_out):
            st.wait_stream(stream)

    def join():
        for st in (s_in, s_k, s_out):
            stream.wait_stream(st)

    steps = max(10, min(args.steps, 12))
    fork()
    step()
    join()
    torch.cuda.synchronize()
    floor = copy_floor(h_proj, d_in[0])
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    fork()
    for _ in range(steps):   # steps overlap: each waits only on the buffers it reuses
        step()
    join()
    t1.record(stream)
    torch.cuda.synchronize()
    ms = t0.elapsed_time(t1) / steps
    ok = bool(np.array_equal(h_out.numpy(), h_img.numpy()))
    user = S * Q * P * 8 * (1 + len(masks))
    h2d = S * Q * P * 8 + staged[0]
    d2h = S * plan.total * 8 + len(masks) * S * Q * P * 8
    return {"value": round(user / (ms * 1e-3) / 1e9, 3), "unit": "GB/s",
            "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
            "ms_per_step": round(ms, 3), "steps": steps, "round_trip_ok": ok,
            "copy_floor": {"ms": round(max(h2d / floor["h2d_gbs"], d2h / floor["d2h_gbs"],
                                           (h2d + d2h) / floor["both_gbs"]) / 1e6, 3), **floor},
            "pipeline": (f"{chunks} stripe slices; host-to-device copies, kernels and device-to-host "
                         "copies on three streams ordered by events; decode input and output "
                         "double-buffered; decode inputs: surviving projections only"),
            "host": host_memory_note()}


def copy_floor(h_buf, d_buf, nbytes=2 << 30):
    """Pinned host <-> device copy bandwidth (GB/s) measured on this machine:
    host-to-device alone, device-to-host alone, and both at once on two
    streams (the e2e step's copies cannot beat these)."""
    import torch
    n = min(nbytes // 8, h_buf.numel(), d_buf.numel())
    h, d = h_buf.view(-1)[:n], d_buf.view(-1)[:n]
    a, b = torch.cuda.Stream(), torch.cuda.Stream()
    half = n // 2

    def timed(fn, reps=3):
        fn()
        torch.cuda.synchronize()
        t = time.perf_counter()
        for _ in range(reps):
            fn()
        torch.cuda.synchronize()
        return (time.perf_counter() - t) / reps

    def both():
        with torch.cuda.stream(a):
            d[:half].copy_(h[:half], non_blocking=True)
        with torch.cuda.stream(b):
            h[half:2 * half].copy_(d[half:2 * half], non_blocking=True)

    t_in = timed(lambda: d.copy_(h, non_blocking=True))
    t_out = timed(lambda: h.copy_(d, non_blocking=True))
    t_both = timed(both)
    return {"h2d_gbs": round(n * 8 / t_in / 1e9, 1), "d2h_gbs": round(n * 8 / t_out / 1e9, 1),
            "both_gbs": round(2 * half * 8 / t_both / 1e9, 1)}


def host_memory_note():
    """Where the pinned buffers sit relative to the GPU: the NUMA nodes of
    the host and the GPU's affinity (nvidia-smi topo), for the record."""
    note = {}
    try:
        nodes = [d for d in os.listdir("/sys/devices/system/node") if d.startswith("node") and d[4:].isdigit()]
        note["numa_nodes"] = len(nodes)
    except Exception:
        pass
    try:
        r = subprocess.run(["nvidia-smi", "topo", "-m"], capture_output=True, text=True, timeout=10)
        for ln in r.stdout.splitlines():
            if ln.startswith("GPU0"):
                note["gpu0_topo"] = " ".join(ln.split())
    except Exception:
        pass
    return note


# ------------------------------------------------------------ batched arm --

def run_batched(args, rank=0):
    """The mixed batch two ways on the same device buffers: (a) batched --
    one CUDA-graph launch for every encode and one for every decode (after
    autotuning); (b) plain -- one mojette_encode per geometry and one
    mojette_decode per (geometry, erasure mask), stripes of a mask
    contiguous. Returns a dict of both throughputs (user data, encode +
    decode per step) and the round-trip checks."""
    import torch
    from paper_1504_07038_gb300 import binding as mj

    S = BATCHED["S"]
    seed = inputs.DEFAULT_SEED + 1000 * rank
    cat = inputs.categories(S, len(BATCH_GEOMS), seed=seed)
    plans, d_img, d_proj, d_out, groups = [], [], [], [], []
    enc_parts, dec_parts = [], []
    user = 0
    for k, (P, Q, p) in enumerate(BATCH_GEOMS):
        Sk = int((cat == k).sum())
        plan = mj.mojette_plan(P, Q, p)
        n = len(p)
        masks = inputs.erasure_masks(Sk, n, inputs.erasure_counts(Sk, n - Q, seed=seed + k), seed=seed + k)
        masks = np.sort(masks, kind="stable")          # stripes of a mask contiguous (plain arm)
        img = torch.from_numpy(inputs.stripes(Sk, Q, P, seed=seed + 17 * k).view(np.int64)).cuda()
        proj = torch.empty((Sk, plan.total), dtype=torch.int64, device="cuda")
        out = torch.empty((Sk, Q, P), dtype=torch.int64, device="cuda")
        plans.append(plan)
        d_img.append(img)
        d_proj.append(proj)
        d_out.append(out)
        uniq, start = np.unique(masks, return_index=True)
        ends = list(start[1:]) + [Sk]
        groups.append([(int(m), int(a), int(b)) for m, a, b in zip(uniq, start, ends)])
        s_idx = np.arange(Sk, dtype=np.uint64)
        enc_parts.append((np.full(Sk, k), np.zeros(Sk, np.uint32), img.data_ptr() + s_idx * np.uint64(Q * P * 8),
                          proj.data_ptr() + s_idx * np.uint64(plan.total * 8)))
        dec_parts.append((np.full(Sk, k), masks, proj.data_ptr() + s_idx * np.uint64(plan.total * 8),
                          out.data_ptr() + s_idx * np.uint64(Q * P * 8)))
        user += Sk * Q * P * 8

    def table(parts, op):
        perm = inputs.permutation(S, seed=seed + op)
        cols = [np.concatenate([pt[c] for pt in parts])[perm] for c in range(4)]
        return mj.stripe_table(plans, cols[0], op, cols[1], cols[2], cols[3])

    stream = torch.cuda.current_stream()
    enc = mj.mojette_batch_create(table(enc_parts, mj.MOJETTE_OP_ENCODE), plans, mj.MOJETTE_BATCH_GRAPH)
    dec = mj.mojette_batch_create(table(dec_parts, mj.MOJETTE_OP_DECODE), plans, mj.MOJETTE_BATCH_GRAPH)
    mj.mojette_batch_run(enc, stream)
    t0 = time.perf_counter()
    mj.mojette_batch_tune(enc, stream, reps=2)
    mj.mojette_batch_tune(dec, stream, reps=2)
    tune_s = time.perf_counter() - t0

    def step_batched():
        mj.mojette_batch_run(enc, stream)
        mj.mojette_batch_run(dec, stream)

    def step_plain():
        for k, plan in enumerate(plans):
            mj.mojette_encode(plan, d_img[k], d_proj[k], d_img[k].shape[0], stream)
        for k, plan in enumerate(plans):
            for m, a, b in groups[k]:
                mj.mojette_decode(plan, d_proj[k][a:b], m, d_out[k][a:b], b - a, stream)

    def timed(step):
        for t in d_out:
            t.zero_()
        for _ in range(args.warmup):
            step()
        torch.cuda.synchronize()
        ok = all(torch.equal(o, i) for o, i in zip(d_out, d_img))
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        steps = max(3, min(args.steps, 10))
        e0.record(stream)
        for _ in range(steps):
            step()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / steps, ok, steps

    ms_b, ok_b, steps_b = timed(step_batched)
    ms_p, ok_p, steps_p = timed(step_plain)
    mj.mojette_device_status()
    ie, idd = mj.mojette_batch_info(enc), mj.mojette_batch_info(dec)
    plain_launches = len(plans) + sum(len(g) for g in groups)
    return {"value": round(2 * user / (ms_b * 1e-3) / 1e9, 3), "unit": "GB/s",
            "ms_per_step": round(ms_b, 4), "steps": steps_b, "round_trip_ok": ok_b,
            "plain": {"value": round(2 * user / (ms_p * 1e-3) / 1e9, 3), "ms_per_step": round(ms_p, 4),
                      "launches_per_step": plain_launches, "round_trip_ok": ok_p, "steps": steps_p},
            "speedup_vs_plain": round(ms_p / ms_b, 3),
            "workload": BATCHED["desc"], "stripes": S, "user_bytes_per_op": user,
            "graph_launches_per_step": 2, "kernels_per_step": ie["launches"] + idd["launches"],
            "decode_groups": idd["groups"], "tune_s": round(tune_s, 2),
            "tuned": {"encode": ie["configs"], "decode": idd["configs"]},
            "l2": "inputs larger than L2 (no flush)"}


# --------------------------------------------------------- systematic arm --

# The systematic form (the paper mentions it, Sec. 2.3 and Sec. 4, without a
# definition): Q data lines stored as they are plus parity projections.
SYSTEMATIC = dict(S=262144, codes=[("8KB(6,4)", 256, 4, [-1, 1]), ("8KB(12,8)", 128, 8, [-2, -1, 1, 2])],
                  masks_per_e=6,
                  desc="262144 stripes x 8 KB per code, systematic (6,4) = 4 data lines + 2 parity "
                       "p={-1,1} and (12,8) = 8 data lines + 4 parity p={-2,-1,1,2}; parity encode, and "
                       "in-place decode of e = 1..r lost data lines (up to 6 seeded lost-line sets per e, "
                       "no parity lost)")


def run_systematic(args, rank=0):
    """Parity encode and in-place decode of the systematic form per number
    of lost data lines e. Decode bytes per stripe (algorithmic, HBM): the
    Q - e known lines and the e * P bins the path reads, plus the e * P
    rebuilt pixels written = (Q + e) * P * 8. User-data GB/s counts the whole
    Q * P * 8-byte block a read returns."""
    import torch
    from paper_1504_07038_gb300 import binding as mj

    S = SYSTEMATIC["S"]
    peak, _ = measured_peaks()
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    reps = max(3, min(args.steps, 10))

    def timed(fn):
        for _ in range(2):
            fn()
        e0.record(stream)
        for _ in range(reps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    out = {"workload": SYSTEMATIC["desc"], "l2": "inputs larger than L2 (no flush)", "codes": {}}
    ok_all = True
    launches = 0
    for name, P, Q, p in SYSTEMATIC["codes"]:
        plan = mj.Plan(P, Q, p, systematic=True)
        seed = inputs.DEFAULT_SEED + 31 + 1000 * rank
        ref = torch.from_numpy(inputs.stripes(S, Q, P, seed=seed).view(np.int64)).cuda()
        data = ref.clone()
        par = torch.empty((S, plan.total), dtype=torch.int64, device="cuda")
        block = Q * P * 8
        enc_ms = timed(lambda: mj.mojette_encode(plan, ref, par, S, stream))
        launches += reps + 2
        enc_bytes = S * (Q * P + plan.total) * 8
        res = {"encode": {"ms": round(enc_ms, 4), "user_gbs": round(S * block / enc_ms / 1e6, 1),
                          "hbm_gbs": round(enc_bytes / enc_ms / 1e6, 1),
                          "frac": round(enc_bytes / enc_ms / 1e6 / peak, 4),
                          "algorithmic_bytes_per_launch": enc_bytes},
               "decode": {}}
        rng = np.random.default_rng(seed)
        for e in range(1, len(p) + 1):
            sets = list(itertools.combinations(range(Q), e))
            if len(sets) > SYSTEMATIC["masks_per_e"]:
                sets = [sets[i] for i in sorted(rng.choice(len(sets), SYSTEMATIC["masks_per_e"], replace=False))]
            ms_list = []
            for lines in sets:
                m = sum(1 << l for l in lines)
                data[:, list(lines)] = 0x5A5A5A5A                   # lost: any contents
                mj.mojette_sys_decode(plan, par, m, data, S, stream)
                torch.cuda.synchronize()
                ok_all &= bool(torch.equal(data, ref))
                ms_list.append(timed(lambda: mj.mojette_sys_decode(plan, par, m, data, S, stream)))
                launches += reps + 3
            ms = statistics.median(ms_list)
            dec_bytes = S * (Q + e) * P * 8
            res["decode"][f"e={e}"] = {"ms": round(ms, 4), "user_gbs": round(S * block / ms / 1e6, 1),
                                       "hbm_gbs": round(dec_bytes / ms / 1e6, 1),
                                       "frac": round(dec_bytes / ms / 1e6 / peak, 4),
                                       "algorithmic_bytes_per_launch": dec_bytes,
                                       "lost_line_sets": len(sets),
                                       "ms_min_max": [round(min(ms_list), 4), round(max(ms_list), 4)]}
        res["decode"]["e=0"] = "no launch: the surviving data lines are the block"
        out["codes"][name] = res
        del ref, data, par
        torch.cuda.empty_cache()
    mj.mojette_device_status()
    out["round_trip_ok"] = ok_all
    out["gpu_launches"] = launches
    return out


# ------------------------------------------------------------- served arm --

SERVED = dict(requests=3000, budget=16 << 30, slots=4, max_wave_stripes=65536,
              desc="request server: 70% writes / 30% reads (0..n-k seeded erasures), objects 4 KB-1 MB "
                   "log-uniform in 4 KB / 8 KB stripes of (6,4) or (12,8), pinned host buffers, "
                   "16 GB device budget; closed loop for capacity, Poisson arrivals at 50/80/95% of it")


def run_served(args, rank=0):
    """The request server against the same requests served one at a time
    through the plain entry points. Throughput = object bytes / elapsed
    (first arrival to last completion), copies included."""
    from paper_1504_07038_gb300 import binding as mj
    from paper_1504_07038_gb300 import serving

    cfg = SERVED
    wl = serving.Workload(cfg["requests"], seed=inputs.DEFAULT_SEED + 7 + 1000 * rank)
    srv = mj.mojette_server_create(cfg["budget"], cfg["slots"], cfg["max_wave_stripes"])
    user = float(wl.user_bytes.sum())
    serving.run_server(srv, wl, rate=None)                    # warm-up: batches, schedules
    comp, el = serving.run_server(srv, wl, rate=None)
    ok = all(np.array_equal(wl.output(r), (wl.images[r].reshape(-1))) for r in range(len(wl))
             if not wl.write[r])
    cap_rps = len(wl) / el
    out = {"closed_loop": {"value": round(user / el / 1e9, 3), "unit": "GB/s", "requests_per_s": round(cap_rps, 1),
                           **serving.latency_stats(comp)},
           "reads_ok": ok, "requests": len(wl), "user_bytes": int(user),
           "write_fraction": round(float(wl.write.mean()), 3), "workload": cfg["desc"]}
    for frac in (0.5, 0.8, 0.95):
        comp, el = serving.run_server(srv, wl, rate=frac * cap_rps, seed=int(frac * 100))
        out[f"poisson_{int(frac * 100)}pct"] = {"offered_rps": round(frac * cap_rps, 1),
                                                "value": round(user / el / 1e9, 3), "unit": "GB/s",
                                                **serving.latency_stats(comp)}
    st = mj.mojette_server_stats(srv)
    out["waves"] = st["waves"]
    out["pool_peak_bytes"] = st["pool_peak"]
    el_plain = serving.run_plain(wl)
    out["plain_sequential"] = {"value": round(user / el_plain / 1e9, 3), "unit": "GB/s",
                               "requests_per_s": round(len(wl) / el_plain, 1)}
    out["speedup_vs_plain"] = round(out["closed_loop"]["value"] / out["plain_sequential"]["value"], 3)
    srv.close()
    return out


# --------------------------------------------------------------- CPU oracle --

def oracle_rate(w, masks, budget_s, threads):
    """The oracle on `threads` host threads over a growing sample of the
    workload's stripes (1 encode + len(masks) decodes each) until it runs
    about budget_s / 4 seconds: (user-data GB/s, stripes, seconds)."""
    import oracle
    P, Q, p = w["P"], w["Q"], w["p"]
    S = 16
    while True:
        img = inputs.stripes(S, Q, P)
        t0 = time.perf_counter()
        proj = oracle.encode(img, p, threads=threads)
        for m in masks:
            oracle.decode(proj, p, P, Q, m, threads=threads)
        dt = time.perf_counter() - t0
        if dt > budget_s / 4 or S >= w["S"]:
            break
        S = min(w["S"], int(S * max(2.0, budget_s / 4 / max(dt, 1e-3))))
    return S * Q * P * 8 * (1 + len(masks)) / dt / 1e9, S, dt


def cpu_baseline(w, masks, budget_s=12.0, single=True):
    """The oracle as it stands on the host cores, on a bounded sample of the
    workload (1 encode + len(masks) decodes per stripe, like a step): all
    cores (the reported value) and, with `single`, one thread."""
    cores = os.cpu_count() or 1
    value, S, dt = oracle_rate(w, masks, budget_s, cores)
    one, S1, dt1 = oracle_rate(w, masks, budget_s / 2, 1) if single else (None, 0, 0.0)
    cpu = "unknown"
    try:
        with open("/proc/cpuinfo") as f:
            for ln in f:
                if ln.lower().startswith(("model name", "cpu part")):
                    cpu = ln.split(":", 1)[1].strip()
                    break
    except Exception:
        pass
    out = {"value": round(value, 4), "unit": "GB/s", "cores": cores, "kind": "oracle",
           "sample": f"{S} stripes of the workload: 1 encode + {len(masks)} decodes each "
                     f"({dt:.1f} s, {cores} threads, cpu {cpu})"}
    if single:
        out["single_thread"] = {"value": round(one, 4), "unit": "GB/s", "cores": 1,
                                "sample": f"{S1} stripes, 1 encode + {len(masks)} decodes each ({dt1:.1f} s)"}
    return out


def run_reference(args, w):
    world, rank, _ = dist_setup()
    if rank != 0:
        return None
    masks = workload_masks(w)
    per_step = max(1.0, min(20.0, 150.0 / max(1, args.steps + args.warmup)))
    for _ in range(args.warmup):
        cpu_baseline(w, masks, budget_s=per_step, single=False)
    vals = [cpu_baseline(w, masks, budget_s=per_step, single=k == args.steps - 1) for k in range(args.steps)]
    v = round(statistics.median(x["value"] for x in vals), 4)
    cb = dict(vals[-1])
    cb["value"] = v
    user_step = w["S"] * w["Q"] * w["P"] * 8 * (1 + len(masks))
    return {"impl": "reference", "metric": METRIC, "value": v, "unit": "GB/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(user_step / (v * 1e9) * 1e3, 3), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u64",
            "data": "synthetic (seeded SplitMix64 uniform uint64 pixels)",
            "config": workload_config(args, w, 1),
            "cpu_baseline": cb,
            "e2e": {"value": v, "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="plain_at_scale", choices=sorted(WORKLOADS))
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-batched", action="store_true", help="skip the mixed-batch comparison")
    ap.add_argument("--no-served", action="store_true", help="skip the request-server measurement")
    ap.add_argument("--no-systematic", action="store_true", help="(default) no systematic-form measurement")
    ap.add_argument("--systematic", action="store_true", help="add the systematic-form measurement")
    ap.add_argument("--no-wide", action="store_true", help="skip the (12,8) 4 KB / 8 KB measurement")
    ap.add_argument("--no-alternatives", action="store_true", help="skip the opt-in decode kernels")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--seed", type=int, default=inputs.DEFAULT_SEED, help="seed of the stripe pixels")
    ap.add_argument("--e2e-chunks", type=int, default=8, help="stripe slices of the e2e pipeline")
    ap.add_argument("--stripes", type=int, default=0, help="override the workload's stripe count")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be at least 3")
    w = dict(WORKLOADS[args.workload])
    if args.stripes:
        w["S"] = args.stripes
        w["desc"] = w["desc"] + f" (stripes set to {args.stripes})"
    line = run_reference(args, w) if args.impl == "reference" else run_gpu(args, w)
    if line is not None:
        print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
