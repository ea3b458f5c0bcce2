#!/usr/bin/env python
"""Benchmark of the micro-batch stream engine's hot path on B300.

Workload (one step = one micro-batch through the whole hot path: fused
filter/window/pre-aggregate pass, sort + reduce into window state, window
assembly and row emission, carry of open panes):
  large float stream: 2^26-event micro-batches (1 GiB of columns, larger than
  L2), ts monotone with U{0..5} ms gaps, key Zipf(1.1) over 1M keys, value
  float32 lognormal(0,1); query: value > 0.5, sliding window 60 s / slide 5 s,
  count/sum/min/max/avg with FP64 sums.  Synthetic data generated on the device.

Output: one JSON line (rank 0).  `value` = events/s with the input resident in
HBM; `e2e` = the same through the C ABI from pinned host buffers, host->device
copy of the batch and device->host copy of every result row inside the timed
region.  `roofline` covers the kernel with the largest share of the step,
`agg_pass` the fused aggregation pass, `cpu_baseline` the CPU oracle on a
bounded sample.  `--impl reference` times the CPU oracle instead.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WINDOW_SIZE_MS, WINDOW_SLIDE_MS, FILTER_GT = 60_000, 5_000, 0.5
ROW_BYTES = 48           # lms_result_row
GROUP_BYTES = 32         # one (pane, key) group: gkey 8 + count 8 + sum 8 + min 4 + max 4
EVENT_BYTES = 16         # ts 8 + key 4 + value 4
WORKLOAD = ("large float stream: micro-batches of 2^{lg} events, key Zipf(1.1) over 1M keys, "
            "value float32 lognormal(0,1), ts +U{{0..5}} ms; query value>0.5, sliding 60 s / "
            "5 s, count/sum/min/max/avg (FP64 sums)")


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6400.0, "fallback"


def _ncu_traffic():
    """DRAM bytes per launch from the committed ncu summary (kernel -> (events, bytes))."""
    p = os.path.join(ROOT, "profiles", "ncu_traffic.txt")
    out = {}
    if os.path.exists(p):
        for line in open(p):
            parts = line.split()
            if len(parts) == 3 and not line.startswith("#"):
                out[parts[0]] = (int(parts[1]), float(parts[2]))
    return out


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.dev = device_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200", "-i", str(self.dev)],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.lines:
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax = float(f[2])
            except ValueError:
                continue
            for name, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


def cpu_baseline(lg: int, seed: int):
    """The CPU oracle, as it stands, on a bounded sample of the same workload (1 core)."""
    from oracle import window_agg as wa
    from paper_2111_04289_b300 import synth

    gen = synth.LargeFloatStream(seed=seed)
    b = gen.next_batch(1 << lg)
    o = wa.WindowAggOracle(True, 0)
    o.add_query(wa.COL_VALUE, wa.OP_GT, 0, FILTER_GT, WINDOW_SIZE_MS, WINDOW_SLIDE_MS)
    t0 = time.perf_counter()
    o.push(b.ts, b.key, b.value, None)
    dt = time.perf_counter() - t0
    return {"value": (1 << lg) / dt, "unit": "events/s", "cores": 1, "kind": "oracle",
            "sample": f"one micro-batch of 2^{lg} events of the same workload "
                      f"({dt:.1f} s single-threaded)"}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    from oracle import window_agg as wa
    from paper_2111_04289_b300 import synth

    lg = args.ref_log2
    gen = synth.LargeFloatStream(seed=synth.BASE_SEED + 2)
    o = wa.WindowAggOracle(True, 0)
    qid = o.add_query(wa.COL_VALUE, wa.OP_GT, 0, FILTER_GT, WINDOW_SIZE_MS, WINDOW_SLIDE_MS)
    times = []
    for step in range(args.warmup + args.steps):
        b = gen.next_batch(1 << lg)
        t0 = time.perf_counter()
        o.push(b.ts, b.key, b.value, None)
        o.take_rows(qid)
        dt = time.perf_counter() - t0
        if step >= args.warmup:
            times.append(dt)
    total = sum(times)
    v = args.steps * (1 << lg) / total
    line = {"impl": "reference", "metric": "events/s", "value": v, "unit": "events/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * total / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD.format(lg=lg) + " (bounded CPU sample per step)",
                       "batch_events": 1 << lg},
            "cpu_baseline": {"value": v, "unit": "events/s", "cores": 1, "kind": "oracle",
                             "sample": f"{args.steps} micro-batches of 2^{lg} events"},
            "e2e": {"value": v, "unit": "events/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def run_ours(args):
    import torch

    from paper_2111_04289_b300 import lmstream as lm
    from paper_2111_04289_b300 import synth

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    lg = args.log2n
    n = 1 << lg
    nb = args.warmup + args.steps
    batches = synth.device_large_float_batches(torch, nb, n, synth.BASE_SEED + 100 + rank, dev)
    torch.cuda.synchronize()
    cur = torch.cuda.current_stream()
    s = lm.Stream("float32", device=local, cuda_stream=cur.cuda_stream, enable_timing=True,
                  k1_variant=args.k1_variant)
    qid = s.register_query(WINDOW_SIZE_MS, WINDOW_SLIDE_MS, "value", "gt", FILTER_GT)
    for i in range(args.warmup):
        b = batches[i]
        s.push(b["ts"], b["key"], b["value"])
        s.discard(qid)
    torch.cuda.synchronize()
    st0 = s.stats()
    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.3)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    w0 = time.perf_counter()
    e0.record(cur)
    for i in range(args.warmup, nb):
        b = batches[i]
        s.push(b["ts"], b["key"], b["value"])
        s.discard(qid)
    e1.record(cur)
    torch.cuda.synchronize()
    wall = time.perf_counter() - w0
    if dist:
        dist.barrier()
    clocks = sampler.stop()
    st1 = s.stats()
    ms = e0.elapsed_time(e1)
    t = torch.tensor([ms], device=dev, dtype=torch.float64)
    if dist:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    ms_max = float(t.item())
    K = args.steps
    value = K * n * world / (ms_max / 1e3)
    d = {k: st1[k] - st0[k] for k in ("k1_ms", "sort_ms", "emit_ms", "e1_ms", "e2_ms",
                                      "k1_launches", "kernel_launches", "partials",
                                      "groups_built", "rows_emitted", "events")}
    peak, peak_kind = _peaks()
    traffic = _ncu_traffic()

    def roof(name, bytes_per_launch, ms_per_launch):
        gbs = bytes_per_launch / (ms_per_launch / 1e3) / 1e9
        tr = traffic.get(name)
        tv = None if tr is None else tr[1] * (n / tr[0])
        return {"kernel": name, "bound": "hbm", "achieved": gbs, "peak": peak, "unit": "GB/s",
                "frac": gbs / peak, "peak_kind": peak_kind, "traffic": tv,
                "algorithmic_bytes": bytes_per_launch, "ms_per_launch": ms_per_launch}

    k1_bytes = EVENT_BYTES * n + GROUP_BYTES * d["partials"] / K
    k1 = roof("k1_fused", k1_bytes, d["k1_ms"] / max(1, d["k1_launches"]))
    e2_bytes = ROW_BYTES * d["rows_emitted"] / K + GROUP_BYTES * d["groups_built"] / K
    e2 = roof("k_emit_write", e2_bytes, d["e2_ms"] / K)
    share = {"k1_fused_ms": d["k1_ms"] / K, "sort_reduce_ms": d["sort_ms"] / K,
             "emit_ms": d["emit_ms"] / K, "emit_count_ms": d["e1_ms"] / K,
             "emit_write_ms": d["e2_ms"] / K}
    dominant = e2 if d["e2_ms"] >= d["k1_ms"] else k1

    line = {"metric": "events/s", "value": value, "unit": "events/s", "n_gpus": world,
            "steps": K, "warmup": args.warmup, "ms_per_step": ms_max / K,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (generated on device, seeded)",
            "config": {"workload": WORKLOAD.format(lg=lg), "batch_events": n, "queries": 1,
                       "parallelism": f"replicas x{world} (no data-path collective)",
                       "l2": "inputs larger than L2 (1 GiB of columns per micro-batch)"},
            "roofline": dominant, "agg_pass": k1, "phase_ms_per_step": share,
            "rows_per_step": d["rows_emitted"] / K, "gpu_launches": d["kernel_launches"],
            "wall_s": wall, "clocks": clocks}
    s.close()
    del batches
    torch.cuda.synchronize()
    if not args.no_e2e:
        line["e2e"] = run_e2e(args, torch, lm, synth, dev, local, rank, world, dist)
    if rank == 0 and not args.no_cpu:
        line["cpu_baseline"] = cpu_baseline(args.cpu_log2, synth.BASE_SEED + 2)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.barrier()
        dist.destroy_process_group()
    return 0


def run_e2e(args, torch, lm, synth, dev, local, rank, world, dist):
    """Same metric through the C ABI with host buffers: H2D of the batch and D2H
    of every result row inside the timed region, one micro-batch per step."""
    lg = args.log2n
    n = 1 << lg
    steps = args.e2e_steps
    batches = synth.device_large_float_batches(torch, 1 + steps, n,
                                               synth.BASE_SEED + 200 + rank, dev)
    h_ts = torch.empty(n, dtype=torch.int64, pin_memory=True)
    h_key = torch.empty(n, dtype=torch.int32, pin_memory=True)
    h_val = torch.empty(n, dtype=torch.float32, pin_memory=True)
    out_rows = 1 << 22
    h_out = torch.empty(out_rows * ROW_BYTES, dtype=torch.uint8, pin_memory=True)
    s = lm.Stream("float32", device=local)
    qid = s.register_query(WINDOW_SIZE_MS, WINDOW_SLIDE_MS, "value", "gt", FILTER_GT)
    times, rows_total = [], 0
    for i in range(1 + steps):
        b = batches[i]
        h_ts.copy_(b["ts"])
        h_key.copy_(b["key"])
        h_val.copy_(b["value"])
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        s.push(h_ts, h_key, h_val)
        got = 0
        while True:
            m = s.poll_into(qid, h_out.data_ptr(), out_rows)
            if m == 0:
                break
            got += m
        dt = time.perf_counter() - t0
        if i >= 1:
            times.append(dt)
            rows_total += got
    s.close()
    tt = torch.tensor([sum(times)], dtype=torch.float64, device=dev)
    if dist:
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
    return {"value": steps * n * world / float(tt.item()), "unit": "events/s",
            "h2d_bytes_per_step": EVENT_BYTES * n, "d2h_bytes_per_step": ROW_BYTES * rows_total // steps,
            "steps": steps, "warmup": 1}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--log2n", type=int, default=26)
    ap.add_argument("--e2e-steps", type=int, default=2)
    ap.add_argument("--cpu-log2", type=int, default=22)
    ap.add_argument("--ref-log2", type=int, default=20)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--k1-variant", type=int, default=0)
    args = ap.parse_args()
    if args.warmup < 3 and args.impl == "ours":
        print("note: warmup < 3 is below the timing rules", file=sys.stderr)
    sys.exit(run_reference(args) if args.impl == "reference" else run_ours(args))


if __name__ == "__main__":
    main()
