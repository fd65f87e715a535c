#!/usr/bin/env python
"""Benchmark of the product-to-sum element-matrix fill (one JSON line on stdout).

python bench.py [--gpus N] [--steps K] [--warmup W] [--workload c2] [--impl ours|reference]

A step is one pass of the whole fill over the workload's batch of synthetic elements:
coupling factor + moments (one kernel) and the product-to-sum contraction (one kernel)
writing every FP64 entry of every element matrix.  `value` is matrix entries per second
over all ranks, inputs resident in HBM; `e2e` is the same metric through the library's
public API with pinned host inputs copied in and every output entry copied back to host
inside the timed region.  Under torchrun each rank fills its own batch (weak scaling, no
collective on the data path; one all-reduce of the elapsed time).
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

from paper_1703_09619_gb300 import workloads as W  # noqa: E402

METRIC = "matrix entries/s: learned+mixed-prec vs plain FP64 fill, one GB300, rel err ≤1e-8"
PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
# FP64 FMA rate of the part: 152 SMs x 2 DFMA/clk/SM (measured by a throughput probe:
# 0.598 TFMA/s at the running clock) -> at the 2070 MHz maximum SM clock:
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.070e9 / 1e12


def log(*a):
    print(*a, file=sys.stderr, flush=True)


def load_peaks():
    try:
        with open(PEAKS_FILE) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


# ----------------------------------------------------------------------------- counting
def _runs():
    """nnz of every Eq. (3) coefficient run, from the library's tables."""
    from paper_1703_09619_gb300 import p2s
    n = p2s.MAX_ORDER
    cnt = np.zeros((4, n, n), dtype=np.int64)
    for t in range(4):
        for a in range(n):
            for b in range(n):
                cnt[t, a, b] = np.count_nonzero(p2s.linearisation(t, a, b, 2 * n))
    return cnt


def contract_fma_count(orders, types_mask):
    """Algorithmic FMAs of the sparse three-stage contraction (Eq. (4)) for a batch."""
    cnt = _runs()
    total = 0
    uniq, counts = np.unique(orders.reshape(orders.shape[0], -1), axis=0, return_counts=True)
    nc = orders.shape[1]
    for row, mult in zip(uniq, counts):
        o = row.reshape(nc, 3)
        s = 0
        for gi in range(nc):
            for gj in range(nc):
                Ni, Nj = o[gi], o[gj]
                K = Ni + Nj - 1
                for t in range(4):
                    if not types_mask & (1 << t):
                        continue
                    cu = cnt[t, :Ni[0], :Nj[0]].sum()
                    cv = cnt[t, :Ni[1], :Nj[1]].sum()
                    cw = cnt[t, :Ni[2], :Nj[2]].sum()
                    s += cu * K[1] * K[2]                        # stage 1
                    s += Ni[0] * Nj[0] * cv * K[2]               # stage 2
                    s += Ni[0] * Ni[1] * Nj[0] * Nj[1] * cw      # stage 3
        total += int(s) * int(mult)
    return total


def moment_mac_count(orders, npts):
    """Algorithmic MACs of the sum-factorised moment contraction (Eq. (4) moments)."""
    total = 0
    nc = orders.shape[1]
    npairs = 1 if nc == 1 else 6
    for e in range(orders.shape[0]):
        K = [int(k) for k in 2 * orders[e].max(axis=0) - 1]
        G = int(npts[e])
        total += npairs * (K[0] * G ** 3 + K[0] * K[1] * G ** 2 + K[0] * K[1] * K[2] * G)
    return int(total)


# ----------------------------------------------------------------------------- clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index):
        self.dev = device_index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.dev), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
        return False

    def summary(self):
        rows = []
        try:
            for line in open(self.path):
                p = [x.strip() for x in line.split(",")]
                if len(p) >= 9:
                    rows.append(p)
        except Exception:
            pass
        finally:
            try:
                os.unlink(self.path)
            except Exception:
                pass
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}

        def num(x):
            try:
                return float(x)
            except ValueError:
                return float("nan")
        sm = [num(r[1]) for r in rows]
        smax = max(num(r[2]) for r in rows)
        power = [num(r[3]) for r in rows]
        pmax = max(power) if power else 0
        load = [s for s, p in zip(sm, power) if p >= 0.5 * pmax] or sm
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            for i, n in enumerate(names):
                if r[5 + i].lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": statistics.median(load), "sm_max_mhz": smax, "reasons": sorted(reasons),
                "samples": len(rows), "power_w_max": pmax}


# ----------------------------------------------------------------------------- oracle legs
def oracle_sample(wl, n_elem, seed=5):
    """Time the CPU oracle on a seeded element sample; returns (entries/s, seconds, desc, threads)."""
    import oracle
    rng = np.random.default_rng(seed)
    idx = np.sort(rng.choice(wl.n_elem, size=min(n_elem, wl.n_elem), replace=False))
    sub = wl.subset(idx)
    threads = oracle.default_threads()
    t0 = time.perf_counter()
    oracle.fill(sub.orders, sub.kind, sub.params, sub.nodes, sub.bulge, sub.npts, sub.types_mask, threads)
    dt = time.perf_counter() - t0
    return sub.entries() / dt, dt, "%d of %d elements (seed %d), every entry, all types" % (
        idx.size, wl.n_elem, seed), threads


def cpu_sample_size(name):
    # about 5-20 s of oracle work on a 16-core host
    return {"c1": 1, "c2": 3, "c3": 2, "c4": 12, "c5": 1}[name]


def run_reference(args, wl):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    n = max(1, cpu_sample_size(args.workload) // 2)
    for _ in range(args.warmup):
        oracle_sample(wl, 1, seed=99)
    vals, secs = [], []
    desc = threads = None
    for k in range(args.steps):
        v, dt, desc, threads = oracle_sample(wl, n, seed=100 + k)
        vals.append(v)
        secs.append(dt)
    value = float(np.mean(vals))
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "entries/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * float(np.mean(secs)),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": workload_config(args, wl),
        "cpu_baseline": {"value": value, "unit": "entries/s", "cores": threads, "kind": "oracle",
                         "sample": "per step: " + desc},
        "e2e": {"value": value, "unit": "entries/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def workload_config(args, wl):
    o = wl.orders
    return {"workload": "%s: %s" % (args.workload, wl.description), "elements": wl.n_elem,
            "n_comp": wl.n_comp, "orders": "uniform %d" % o[0, 0, 0] if (o == o[0, 0, 0]).all() else "mixed",
            "npts": int(wl.npts[0]) if (wl.npts == wl.npts[0]).all() else "per-element",
            "precision": args.precision, "entries_per_step": wl.entries(),
            "l2": "outputs (%.1f GB) exceed L2; L2 also flushed (256 MB write) between steps" % (8e-9 * wl.entries())}


# ----------------------------------------------------------------------------- GPU leg
def run_ours(args, wl):
    import torch
    import torch.distributed as dist

    from paper_1703_09619_gb300 import p2s

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    ctx = p2s.Context(local)
    prec = p2s.MIXED if args.precision == "mixed" else p2s.FP64
    npts = int(wl.npts[0]) if (wl.npts == wl.npts[0]).all() else wl.npts
    plan = p2s.Plan(ctx, wl.orders, npts, prec, wl.types_mask)
    params, nodes, bulge = p2s.device_inputs(wl, dev)
    out = torch.empty(plan.output_entries, dtype=torch.float64, device=dev)
    mom = torch.empty(max(plan.moment_entries, 1), dtype=torch.float64, device=dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)

    def step(evs=None):
        if evs:
            evs[0].record(stream)
        plan.moments(wl.kind, params, nodes, bulge, mom, stream=stream)
        if evs:
            evs[1].record(stream)
        plan.contract(mom, out, stream=stream)
        if evs:
            evs[2].record(stream)

    for _ in range(args.warmup):
        step()
        flush.zero_()
    torch.cuda.synchronize()
    rc = ctx.sync_status(stream)
    if rc != 0:
        raise RuntimeError("device status %d after warm-up" % rc)

    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(args.steps)]
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        for k in range(args.steps):
            step(evs[k])
            flush.zero_()
        torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    mom_ms = [a.elapsed_time(b) for a, b, _ in evs]
    con_ms = [b.elapsed_time(c) for _, b, c in evs]
    step_ms = [a.elapsed_time(c) for a, _, c in evs]
    total_ms = float(sum(step_ms))
    if world > 1:
        t = torch.tensor([total_ms], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())
    clocks = clk.summary()

    entries = wl.entries()
    value = world * entries * args.steps / (total_ms * 1e-3)
    peaks, src = load_peaks()
    con_avg = float(np.mean(con_ms))
    mom_avg = float(np.mean(mom_ms))
    fmas = contract_fma_count(wl.orders, wl.types_mask)
    bytes_written = 8 * entries
    macs = moment_mac_count(wl.orders, wl.npts)
    achieved_flops = 2 * fmas / (con_avg * 1e-3) / 1e12
    achieved_gbs = bytes_written / (con_avg * 1e-3) / 1e9
    if prec == p2s.FP64:
        roof = {"bound": "alu", "kernel": "k_contract<ArithF64>", "achieved": achieved_flops,
                "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s", "frac": achieved_flops / FP64_PEAK_TFLOPS,
                "traffic": None,
                "peak_source": "FP64 FMA: 152 SMs x 2 DFMA/clk x 2 flop x 2.07 GHz (probe-measured 2 DFMA/clk/SM)",
                "hbm_write_GBs": achieved_gbs, "hbm_frac_of_measured": achieved_gbs / peaks["hbm_gbs"],
                "algorithmic_flop_per_launch": 2 * fmas, "algorithmic_bytes_per_launch": bytes_written}
    else:
        roof = {"bound": "hbm", "kernel": "k_contract<ArithFF>", "achieved": achieved_gbs, "peak": peaks["hbm_gbs"],
                "unit": "GB/s", "frac": achieved_gbs / peaks["hbm_gbs"], "traffic": None,
                "peak_source": "%s (MEASURED_PEAKS.json copy bandwidth)" % src,
                "algorithmic_bytes_per_launch": bytes_written}
    stages = {"moments_ms": mom_avg, "contract_ms": con_avg,
              "moments_fp64_tflops": 2 * macs / (mom_avg * 1e-3) / 1e12,
              "contract_fp64_tflops": achieved_flops}

    e2e = measure_e2e(args, wl, ctx, prec, dev) if not args.no_e2e else None

    line = None
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "entries/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": workload_config(args, wl),
            "elements_per_s": world * wl.n_elem * args.steps / (total_ms * 1e-3),
            "roofline": roof, "stages": stages, "clocks": clocks,
            "gpu_launches": 2 * args.steps,
        }
        if e2e:
            line["e2e"] = e2e
    del out, mom
    plan.close()
    if rank == 0 and world == 1 and not args.no_cpu:
        v, dt, desc, threads = oracle_sample(wl, cpu_sample_size(args.workload))
        line["cpu_baseline"] = {"value": v, "unit": "entries/s", "cores": threads, "kind": "oracle",
                                "sample": desc + " (%.1f s)" % dt}
    if rank == 0:
        print(json.dumps(line), flush=True)
    ctx.close()
    if world > 1:
        dist.destroy_process_group()


def measure_e2e(args, wl, ctx, prec, dev):
    """Same metric through the public API: pinned host inputs -> device, fill, every output
    entry -> pinned host memory, all inside the timed region.  Outputs stream through a
    two-slot pinned host ring in element chunks on two CUDA streams."""
    import torch

    from paper_1703_09619_gb300 import p2s
    E = wl.n_elem
    per_elem = wl.entries() / E
    chunk = int(max(1, min(E, (2 << 30) // (8 * per_elem))))  # ~2 GB of output per chunk
    starts = list(range(0, E, chunk))
    subs = [wl.subset(np.arange(s, min(E, s + chunk))) for s in starts]
    npts = lambda w: int(w.npts[0]) if (w.npts == w.npts[0]).all() else w.npts
    plans = [p2s.Plan(ctx, w.orders, npts(w), prec, w.types_mask) for w in subs]
    maxn = max(p.output_entries for p in plans)
    host_in = [(torch.from_numpy(np.ascontiguousarray(w.params)).pin_memory(),
                torch.from_numpy(np.ascontiguousarray(w.nodes)).pin_memory(),
                torch.from_numpy(np.ascontiguousarray(w.bulge)).pin_memory()) for w in subs]
    host_out = [torch.empty(maxn, dtype=torch.float64).pin_memory() for _ in range(2)]
    dev_out = [torch.empty(maxn, dtype=torch.float64, device=dev) for _ in range(2)]
    dev_in = [[torch.empty_like(h, device=dev) for h in host_in[0]] for _ in range(2)]
    streams = [torch.cuda.Stream(dev) for _ in range(2)]
    h2d = sum(sum(t.numel() * 8 for t in h) for h in host_in)
    d2h = sum(p.output_entries * 8 for p in plans)

    def one_pass():
        for i, (w, p) in enumerate(zip(subs, plans)):
            s = streams[i % 2]
            with torch.cuda.stream(s):
                di = dev_in[i % 2]
                hi = host_in[i]
                for d, h in zip(di, hi):
                    d[: h.shape[0]].copy_(h, non_blocking=True)
                n = w.n_elem
                p.fill(w.kind, di[0][:n], di[1][:n], di[2][:n], dev_out[i % 2], stream=s)
                host_out[i % 2][: p.output_entries].copy_(dev_out[i % 2][: p.output_entries], non_blocking=True)
        for s in streams:
            s.synchronize()

    one_pass()
    steps = max(1, min(args.steps, 3))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(steps):
        one_pass()
    dt = (time.perf_counter() - t0) / steps
    rc = ctx.sync_status()
    for p in plans:
        p.close()
    if rc != 0:
        raise RuntimeError("device status %d in e2e" % rc)
    return {"value": wl.entries() / dt, "unit": "entries/s", "h2d_bytes_per_step": int(h2d),
            "d2h_bytes_per_step": int(d2h), "steps": steps, "chunks": len(subs),
            "note": "pinned host inputs in, every FP64 entry back to pinned host memory, 2-stream pipeline"}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="c2", choices=["c1", "c2", "c3", "c4", "c5"])
    ap.add_argument("--precision", default="fp64", choices=["fp64", "mixed"])
    ap.add_argument("--elements", type=int, default=None, help="use only the first E elements")
    ap.add_argument("--npts", type=int, default=None, help="override the quadrature size G")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    args = ap.parse_args()
    wl = W.make(args.workload, args.elements)
    if args.npts:
        wl = wl.with_npts(args.npts)
    if args.impl == "reference":
        run_reference(args, wl)
    else:
        run_ours(args, wl)


if __name__ == "__main__":
    main()
