#!/usr/bin/env python
"""Benchmark of the product-to-sum element-matrix fill (one JSON line on stdout).

python bench.py [--gpus N] [--steps K] [--warmup W] [--workload c5] [--mode learned|plain|mixed]
                [--impl ours|reference]

Default: the 32768-element, three-component, N = 4 curved-hexahedron batch (c5) filled by
the learned + mixed-precision path (per-element quadrature picked by the network, float-float
contraction, 2% seeded 48-point FP64 judge with fallback).  `value` is matrix entries per
second of that fill over all ranks, inputs resident in HBM; the plain FP64 fill at 48 points
of the same batch is timed beside it, and every element of the learned fill is compared with
it (max relative error, share above 1e-8).  `e2e` is the same metric through the public API
with pinned host inputs copied in and every FP64 entry copied back to host inside the timed
region.  Under torchrun each rank fills its own batch (weak scaling, no collective on the
data path; one all-reduce of the elapsed time).  --mode plain|mixed times one fixed-G fill of
any workload instead.
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

from paper_1703_09619_gb300 import dist as D  # noqa: E402
from paper_1703_09619_gb300 import workloads as W  # noqa: E402

METRIC = "matrix entries/s: learned+mixed-prec vs plain FP64 fill, one GB300, rel err ≤1e-8"
PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
# FP64 FMA, FP32 FMA and store-only HBM rates are measured in every run by the library's
# probe kernels (p2s_measure_peaks); the values below are the unit-count fallbacks used only
# if that call fails (152 SMs, 2 DFMA / 128 FFMA per clock per SM, 2070 MHz).
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.070e9 / 1e12
# FP64 operations per quadrature point of the metric coupling factor in the moment kernel
# (Jacobian 45, phase 9, sin ~25, cofactors 18, det 3, products 18, division ~10, scale 6)
ALPHA_FLOP_PER_POINT = 134
# The mixed moment kernel runs in double-word (float-float) arithmetic and is bound by FP32
# instruction issue: 152 SMs x 128 lanes x 2.07 GHz lane operations per second.  Its work is
# counted as the FP32 instructions that the double-word algorithms need per operation of the
# method (an FMA counts once):
#   one multiply-accumulate into the lazy accumulator: 12;
#   the metric coupling factor at one point, with the _fast and _lazy double-word operations
#   (sum 11, sum without renormalisation 8, product 4, fused 15 / 12, division 11): 725
#   (Jacobian from row constants 196, phase 30, sin 110 + scale 14, cofactors 144, det 28,
#   division 11, six products 192);
#   the scalar coupling factor at one point: 14;
#   the parity fold of the first mode product, per point and pair: one sum (11) and two
#   shuffles; the first mode product then runs over ceil(G/2) points per row.
FP32_PEAK_TOPS = 152 * 128 * 2.070e9 / 1e12  # FP32 issue slots (lane operations / s), unit counts
DW_MAC_OPS, DW_ALPHA_OPS_METRIC, DW_ALPHA_OPS_SCALAR, DW_FOLD_OPS = 12, 725, 14, 13
# Learned-fill settings: judge share and tolerance.  The class rule's risk comes from the
# checkpoint's metadata, where `python -m paper_1703_09619_gb300.learned --calibrate` keeps the
# largest risk of its sweep whose held-out elements (shard 1 of the training recipe, neither
# trained on nor benchmarked) all stay within 1e-8 of their 48-point FP64 fill.
JUDGE_FRAC, JUDGE_TOL = 0.02, 1e-9
RISK_DEFAULT = 0.002  # only for a checkpoint without a calibrated risk


def log(*a):
    print(*a, file=sys.stderr, flush=True)


def load_peaks():
    try:
        with open(PEAKS_FILE) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


_DEV = {}  # this run's probe results (device_peaks)


def fp64_peak():
    """FP64 FMA rate (TFLOP/s) measured in this run, else the unit-count figure."""
    return _DEV.get("fp64_fma_tflops") or FP64_PEAK_TFLOPS


def fp32_issue_peak():
    """FP32 lane operations per second (T/s): the measured FMA issue rate (half the measured
    FP32 FMA flop rate), else the unit-count figure."""
    v = _DEV.get("fp32_fma_tflops")
    return v / 2 if v else FP32_PEAK_TOPS


def peak_source(kind):
    measured = bool(_DEV.get("fp64_fma_tflops")) and "probes failed" not in _DEV.get("source", "")
    if kind == "fp64":
        return ("FP64 FMA rate of this GPU, measured in this run (p2s_measure_peaks)" if measured
                else "FP64 pipe: 152 SMs x 2 DFMA/clk x 2 flop x 2.07 GHz (unit counts)")
    return ("FP32 FMA issue rate of this GPU, measured in this run (p2s_measure_peaks), one lane operation per FMA"
            if measured else "FP32 issue: 152 SMs x 128 lanes x 2.07 GHz (unit counts)")


def device_peaks(p2s, ctx):
    """FP64 / FP32 FMA and store-only HBM rates of this GPU from the library's probe kernels
    (CUDA events, best of 5); the unit-count figures if the probes fail."""
    try:
        pk = p2s.measure_peaks(ctx, 4 << 30)
        pk["source"] = "p2s_measure_peaks on this GPU in this run (probe kernels, CUDA events, best of 5)"
        _DEV.clear()
        _DEV.update(pk)
        return pk
    except Exception as e:  # noqa: BLE001
        log("peak probes failed: %s" % e)
        return {"fp64_fma_tflops": FP64_PEAK_TFLOPS, "fp32_fma_tflops": 2 * FP32_PEAK_TOPS, "hbm_write_gbs": None,
                "source": "unit counts (probes failed)"}


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
    """Algorithmic FMAs of the sparse three-stage contraction (Eq. (4)) as the library runs
    it: vv and dd blocks gi <= gj, dv blocks all (vd = dv^T when both are selected)."""
    cnt = _runs()
    total = 0
    uniq, counts = np.unique(orders.reshape(orders.shape[0], -1), axis=0, return_counts=True)
    nc = orders.shape[1]
    for row, mult in zip(uniq, counts):
        o = row.reshape(nc, 3)
        s = 0
        for t in range(4):
            if not types_mask & (1 << t):
                continue
            if t == 2 and types_mask & 2:
                continue
            for gi in range(nc):
                for gj in range(nc):
                    if t in (0, 3) and gj < gi:
                        continue
                    Ni, Nj = o[gi], o[gj]
                    K = Ni + Nj - 1
                    cu = cnt[t, :Ni[0], :Nj[0]].sum()
                    cv = cnt[t, :Ni[1], :Nj[1]].sum()
                    cw = cnt[t, :Ni[2], :Nj[2]].sum()
                    s += cu * K[1] * K[2] + Ni[0] * Nj[0] * cv * K[2] + Ni[0] * Ni[1] * Nj[0] * Nj[1] * cw
        total += int(s) * int(mult)
    return total


def operator_fma_count(orders, terms, symmetric):
    """Algorithmic FMAs of the operator contraction: for every element, block and term, the
    three sparse stages with the term's per-axis product types (blocks gi <= gj only when the
    term list is mirror-closed)."""
    cnt = _runs()
    total = 0
    uniq, counts = np.unique(orders.reshape(orders.shape[0], -1), axis=0, return_counts=True)
    nc = orders.shape[1]
    for row, mult in zip(uniq, counts):
        o = row.reshape(nc, 3)
        s = 0
        for tm in terms:
            gi, gj = int(tm[0]), int(tm[1])
            if symmetric and gi > gj:
                continue
            tu, tv, tw = (int(tm[4 + x]) + 2 * int(tm[7 + x]) for x in range(3))
            Ni, Nj = o[gi], o[gj]
            Kv, Kw = Ni[1] + Nj[1] - 1, Ni[2] + Nj[2] - 1
            cu = cnt[tu, :Ni[0], :Nj[0]].sum()
            cv = cnt[tv, :Ni[1], :Nj[1]].sum()
            cw = cnt[tw, :Ni[2], :Nj[2]].sum()
            s += cu * Kv * Kw + Ni[0] * Nj[0] * cv * Kw + Ni[0] * Ni[1] * Nj[0] * Nj[1] * cw
        total += int(s) * int(mult)
    return total


def moment_mac_points(orders, npts, folded=False):
    """Sum-factorised moment MACs, quadrature points and pairs of a batch; with ``folded`` the
    first mode product runs over ceil(G/2) points per row (parity fold of the symmetric rule)."""
    macs = pts = 0
    nc = orders.shape[1]
    npairs = 1 if nc == 1 else 6
    for e in range(orders.shape[0]):
        K = [int(k) for k in 2 * orders[e].max(axis=0) - 1]
        G = int(npts[e])
        ga = (G + 1) // 2 if folded else G
        macs += npairs * (K[0] * ga * G ** 2 + K[0] * K[1] * G ** 2 + K[0] * K[1] * K[2] * G)
        pts += G ** 3
    return macs, pts, npairs


def moment_flop_count(orders, npts, metric=True):
    """Algorithmic FP64 flops of the moment kernel: 2 x the sum-factorised MACs plus the
    coupling-factor evaluation per quadrature point."""
    total = 0
    nc = orders.shape[1]
    npairs = 1 if nc == 1 else 6
    for e in range(orders.shape[0]):
        K = [int(k) for k in 2 * orders[e].max(axis=0) - 1]
        G = int(npts[e])
        total += 2 * npairs * (K[0] * G ** 3 + K[0] * K[1] * G ** 2 + K[0] * K[1] * K[2] * G)
        total += (ALPHA_FLOP_PER_POINT if metric else 8) * G ** 3
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
                                          "--format=csv,noheader,nounits", "-lms", "50"],
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
def sample_indices(wl, n_elem, seed=5):
    rng = np.random.default_rng(seed)
    return np.sort(rng.choice(wl.n_elem, size=min(n_elem, wl.n_elem), replace=False))


def oracle_sample(wl, n_elem, seed=5, keep=False):
    """Time the CPU oracle on a seeded element sample; returns (entries/s, seconds, desc,
    threads), plus (indices, oracle output, its offsets) with ``keep``."""
    import oracle
    idx = sample_indices(wl, n_elem, seed)
    sub = wl.subset(idx)
    threads = oracle.default_threads()
    t0 = time.perf_counter()
    out, off, _ = oracle.fill(sub.orders, sub.kind, sub.params, sub.nodes, sub.bulge, sub.npts, sub.types_mask,
                              threads)
    dt = time.perf_counter() - t0
    res = (sub.entries() / dt, dt, "%d of %d elements (seed %d) at G=%s, every entry, all types" % (
        idx.size, wl.n_elem, seed, ",".join(str(g) for g in sorted(set(sub.npts.tolist())))), threads)
    return res + ((idx, out, off, sub) if keep else ())


def errors_vs_oracle(got_slices, ref, ref_off, sub):
    """Per element max over product types of max|dM| / max|M| (R8) of GPU element slices
    against the oracle's output of the same elements."""
    import oracle
    errs = []
    for e, g in enumerate(got_slices):
        mg = oracle.element_matrices(g, [0], sub.orders[e:e + 1], 0, sub.types_mask)
        mr = oracle.element_matrices(ref, ref_off, sub.orders, e, sub.types_mask)
        errs.append(float(max(np.abs(mg[t] - mr[t]).max() / max(np.abs(mr[t]).max(), 1e-300) for t in mr)))
    return errs


def cpu_sample_size(name):
    # about 5-20 s of oracle work on a 16-core host
    return {"c1": 1, "c2": 3, "c3": 2, "c4": 12, "c5": 4}[name]


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


L2_BYTES = 129 << 20  # GB300 L2 (126 MiB usable, 129 MB nominal)


def l2_note(out_bytes):
    """How a step's output relates to L2 (between timed steps the bench writes 256 MB to flush it)."""
    size = "%.1f GB" % (out_bytes / 1e9) if out_bytes >= 1e8 else "%.2f MB" % (out_bytes / 1e6)
    rel = "exceed L2; L2 also flushed" if out_bytes > L2_BYTES else "fit in L2; L2 flushed"
    return "outputs (%s) %s (256 MB write) between steps" % (size, rel)


def workload_config(args, wl, risk=None, risk_src=None):
    o = wl.orders
    cfg = {"workload": "%s: %s" % (args.workload, wl.description), "elements": wl.n_elem,
           "n_comp": wl.n_comp, "orders": "uniform %d" % o[0, 0, 0] if (o == o[0, 0, 0]).all() else "mixed",
           "mode": args.mode, "entries_per_step": wl.entries(),
           "l2": l2_note(8 * wl.entries())}
    if args.mode == "learned":
        cfg.update({"npts": "learned per element, classes 8/12/16/24/32/48", "plain_npts": 48,
                    "precision": "mixed (float-float contraction, FP64 output)",
                    "risk": RISK_DEFAULT if risk is None else risk,
                    "risk_source": ("held-out calibration kept in the checkpoint: %s" % risk_src.get("holdout")
                                    if risk_src else "default (checkpoint without a calibrated risk)"),
                    "judge": "%.0f%% seeded, re-filled at 48 points in the fill's precision (side stream), tol %.0e; "
                             "failures replaced by the 48-point FP64 fill" % (100 * JUDGE_FRAC, JUDGE_TOL)})
    else:
        cfg.update({"npts": int(wl.npts[0]) if (wl.npts == wl.npts[0]).all() else "per-element",
                    "precision": args.mode})
    return cfg


# ----------------------------------------------------------------------------- GPU helpers
def dist_setup():
    import torch
    world, rank, local = D.init("nccl")
    torch.cuda.set_device(local)
    return world, rank, local


def max_over_ranks(x, world, dev):
    return D.max_over_ranks(x, world, dev)


def barrier(world):
    D.barrier(world)


def time_steps(fn, steps, stream, flush):
    """CUDA-event time (ms) of each call of fn() on `stream`, L2 flushed between calls."""
    import torch
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    for a, b in evs:
        a.record(stream)
        fn()
        b.record(stream)
        flush.zero_()
    torch.cuda.synchronize()
    return [a.elapsed_time(b) for a, b in evs]


def stage_times(p2s, ctx, wl, npts, prec, params, nodes, bulge, dev, stream, flush, steps=3, tile=None):
    """Moment and contraction kernels timed separately on a plan with the given G per element."""
    import torch
    plan = p2s.Plan(ctx, wl.orders, npts, prec, wl.types_mask, tile=tile)
    mom = torch.empty(max(plan.moment_entries, 1), dtype=torch.float64, device=dev)
    out = torch.empty(plan.output_entries, dtype=torch.float64, device=dev)
    plan.moments(wl.kind, params, nodes, bulge, mom, stream=stream)
    plan.contract(mom, out, stream=stream)
    m = time_steps(lambda: plan.moments(wl.kind, params, nodes, bulge, mom, stream=stream), steps, stream, flush)
    c = time_steps(lambda: plan.contract(mom, out, stream=stream), steps, stream, flush)
    del mom, out
    plan.close()
    return float(np.mean(m)), float(np.mean(c))


def contract_kernel(orders, mixed=True, kernel=0):
    """The contraction kernel a plan takes (the library's rule for tile kernel 0)."""
    o = np.asarray(orders)
    arith = "ArithFF" if mixed else "ArithF64"
    if kernel == 1 or o.max() > 8:
        return "k_contract<%s>" % arith
    if not mixed or kernel == 2 or not (o == o.flat[0]).all() or o.flat[0] < 2:
        return "k_contract_ffb<%s>" % arith
    return "k_contract_ffn<%d>" % o.flat[0]


def roofline_for(wl, npts, prec, mom_ms, con_ms, peaks, src, kernel=0):
    """Roofline object of the dominant kernel of a fill (the slower of the two stages).

    Moment stage (a1 + a2): the method's work is 2 x (K G^3 + K^2 G^2 + K^3 G) flop per
    coupling pair (sum-factorised Eq. (4), first mode product unfolded) plus the coupling
    factor's FP64-equivalent operations per point (ALPHA_FLOP_PER_POINT); the mixed form is
    reported against the BF16 dense tensor peak (the roofline the moment contraction is
    assigned) and, beside it, against the measured FP32 FMA rate; `issue_frac` is the
    double-word kernel's FP32 instruction model over the measured FP32 issue rate.  The
    FP64 form is reported against the measured FP64 FMA rate.  Contraction (a4): mixed
    against HBM (8 B per stored entry over the copy bandwidth, and the store-only rate
    beside it), FP64 against the measured FP64 FMA rate."""
    entries = wl.entries()
    fmas = contract_fma_count(wl.orders, wl.types_mask)
    metric = wl.kind == W.KIND_METRIC_EPS
    npts = np.broadcast_to(np.asarray(npts), (wl.n_elem,))
    if mom_ms >= con_ms:
        macs, pts, npairs = moment_mac_points(wl.orders, npts, folded=False)
        alpha_flop = (ALPHA_FLOP_PER_POINT if metric else 8) * pts
        flop = 2 * macs + alpha_flop
        ach = flop / (mom_ms * 1e-3) / 1e12
        model = ("2 x %d MACs (K G^3 + K^2 G^2 + K^3 G per coupling pair, %d pairs) + %d flop per point x %d points"
                 % (macs, npairs, ALPHA_FLOP_PER_POINT if metric else 8, pts))
        if prec == 0:
            pk = fp64_peak()
            return {"bound": "alu", "kernel": "k_moments_fp64", "achieved": ach, "peak": pk,
                    "unit": "TFLOP/s", "frac": ach / pk, "traffic": None, "peak_source": peak_source("fp64"),
                    "algorithmic_flop_per_launch": int(flop), "flop_model": model}
        fmacs, _, _ = moment_mac_points(wl.orders, npts, folded=True)
        per_point = (DW_ALPHA_OPS_METRIC if metric else DW_ALPHA_OPS_SCALAR) + DW_FOLD_OPS * npairs
        ops = DW_MAC_OPS * fmacs + per_point * pts
        iss = ops / (mom_ms * 1e-3) / 1e12
        fp32 = 2 * fp32_issue_peak()
        bf16 = peaks["bf16_tflops"]
        return {"bound": "tensor", "kernel": "k_moments_dw", "achieved": ach, "peak": bf16, "unit": "TFLOP/s",
                "frac": ach / bf16, "traffic": None,
                "traffic_note": "not scalable from a capture of the allowed size: at 1024 elements the moments stay "
                                "in L2 for the contraction (0.45 MB read, 0 written); the full launch writes its "
                                "moments (16.5 KB per element) to DRAM",
                "peak_source": "%s BF16 dense burst (MEASURED_PEAKS.json)" % src,
                "algorithmic_flop_per_launch": int(flop), "flop_model": model,
                "vs_fp32_fma": {"peak": fp32, "frac": ach / fp32, "unit": "TFLOP/s",
                                "peak_source": peak_source("fp32").replace("issue rate", "rate") + " (2 flop per FMA)"},
                "issue_frac": iss / fp32_issue_peak(),
                "issue": {"achieved": iss, "peak": fp32_issue_peak(), "unit": "T FP32 lane-op/s",
                          "peak_source": peak_source("fp32"), "ops_per_launch": int(ops),
                          "op_model": "%d per double-word MAC x %d MACs (first mode product folded) + %d per point x "
                                      "%d points" % (DW_MAC_OPS, fmacs, per_point, pts)}}
    if prec == 0:
        ach = 2 * fmas / (con_ms * 1e-3) / 1e12
        pk = fp64_peak()
        return {"bound": "alu", "kernel": contract_kernel(wl.orders, False, kernel), "achieved": ach,
                "peak": pk, "unit": "TFLOP/s", "frac": ach / pk, "traffic": None, "peak_source": peak_source("fp64"),
                "algorithmic_flop_per_launch": 2 * fmas,
                "hbm_write_GBs": 8 * entries / (con_ms * 1e-3) / 1e9}
    ach = 8 * entries / (con_ms * 1e-3) / 1e9
    kname = contract_kernel(wl.orders, True, kernel)
    roof = {"bound": "hbm", "kernel": kname, "achieved": ach,
            "peak": peaks["hbm_gbs"], "unit": "GB/s", "frac": ach / peaks["hbm_gbs"], "traffic": None,
            "peak_source": "%s copy bandwidth (MEASURED_PEAKS.json)" % src, "algorithmic_bytes_per_launch": 8 * entries}
    if _DEV.get("hbm_write_gbs"):
        roof["vs_store_only"] = {"peak": _DEV["hbm_write_gbs"], "frac": ach / _DEV["hbm_write_gbs"],
                                 "peak_source": "store-only stream measured in this run (p2s_measure_peaks)"}
    return roof


# ----------------------------------------------------------------------------- learned (headline)
def run_learned(args, wl):
    import torch

    from paper_1703_09619_gb300 import learned as LN
    from paper_1703_09619_gb300 import p2s

    world, rank, local = dist_setup()
    dev = torch.device("cuda", local)
    ctx = p2s.Context(local)
    device_peaks(p2s, ctx)
    mlp_params, meta = LN.ensure_trained(ctx)
    risk = float(meta.get("risk", RISK_DEFAULT))
    P = torch.as_tensor(mlp_params, device=dev)
    params, nodes, bulge = p2s.device_inputs(wl, dev)
    stream = torch.cuda.current_stream(dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    lp = p2s.LearnedPlan(ctx, wl.orders, precision=p2s.MIXED, judge_frac=JUDGE_FRAC, seed=1703,
                         judge_tol=JUDGE_TOL, risk=risk, n_nets=LN.n_nets_of(mlp_params))
    out = torch.empty(lp.output_entries, dtype=torch.float64, device=dev)
    npts_d = torch.empty(wl.n_elem, dtype=torch.int32, device=dev)
    step = lambda: lp.fill(wl.kind, params, nodes, bulge, P, out, npts_d, stream=stream)
    for _ in range(args.warmup):
        step()
        flush.zero_()
    torch.cuda.synchronize()
    rep = lp.report(stream)
    barrier(world)
    with ClockSampler(local) as clk:
        ms = time_steps(step, args.steps, stream, flush)
    barrier(world)
    rc = ctx.sync_status(stream)
    if rc != 0:
        raise RuntimeError("device status %d" % rc)
    rep = lp.report(stream)
    total_ms = max_over_ranks(float(sum(ms)), world, dev)
    clocks = clk.summary()
    npts = npts_d.cpu().numpy()

    # the plain FP64 fill at 48 points of the same batch, and the learned fill's error against it
    plain = p2s.Plan(ctx, wl.orders, 48, p2s.FP64)
    ref = torch.empty(plain.output_entries, dtype=torch.float64, device=dev)
    plain.fill(wl.kind, params, nodes, bulge, ref, stream=stream)
    ksteps = max(1, min(args.steps, 3))
    pms = time_steps(lambda: plain.fill(wl.kind, params, nodes, bulge, ref, stream=stream), ksteps, stream, flush)
    plain_ms = max_over_ranks(float(np.mean(pms)), world, dev)
    n, off = p2s.output_entries(wl.orders, offsets=True)
    off_d = torch.as_tensor(off, device=dev)
    err = torch.empty(wl.n_elem, dtype=torch.float64, device=dev)
    p2s.element_errors(ctx, out, off_d, ref, off_d, 4, err, stream=stream)
    err_h = err.cpu().numpy()
    plain.close()
    # the method without the network: the smallest uniform class G whose mixed fill keeps every
    # element of this batch within 1e-8 of the 48-point FP64 fill (chosen on the batch itself)
    uniform = None
    uout = torch.empty_like(out)
    for G in p2s.CLASS_NPTS:
        up = p2s.Plan(ctx, wl.orders, G, p2s.MIXED)
        up.fill(wl.kind, params, nodes, bulge, uout, stream=stream)
        p2s.element_errors(ctx, uout, off_d, ref, off_d, 4, err, stream=stream)
        uerr = err.cpu().numpy()
        if uerr.max() <= 1e-8 or G == p2s.CLASS_NPTS[-1]:
            ums = time_steps(lambda: up.fill(wl.kind, params, nodes, bulge, uout, stream=stream), ksteps, stream, flush)
            ums = max_over_ranks(float(np.mean(ums)), world, dev)
            uniform = {"npts": G, "ms_per_step": ums, "max_rel_err_vs_plain48": float(uerr.max()),
                       "rule": "smallest class G with every element of the batch <= 1e-8 (mixed fill, same plan "
                               "calls as the learned fill's contraction)"}
            up.close()
            break
        up.close()
    del uout, ref
    # the learned fill's elements of the oracle's CPU sample, for the oracle comparison below
    cpu_idx = sample_indices(wl, cpu_sample_size(args.workload))
    cpu_got = [out[int(off[e]):int(off[e + 1])].cpu().numpy() for e in cpu_idx]
    # stage breakdown at the learned G (moments, contraction); the learned fill's moment queue
    # takes elements grouped by G, largest first, so the breakdown fills them in that order
    order = np.argsort(-npts, kind="stable")
    wls = wl.subset(order)
    ps, ns_, bs = p2s.device_inputs(wls, dev)
    mom_ms, con_ms = stage_times(p2s, ctx, wls, npts[order], p2s.MIXED, ps, ns_, bs, dev, stream, flush)
    del ps, ns_, bs
    peaks, src = load_peaks()
    roof = roofline_for(wl, npts, p2s.MIXED, mom_ms, con_ms, peaks, src)
    entries = wl.entries()
    job_entries = D.sum_over_ranks(entries, world, dev)  # each rank fills a batch of its own
    job_elems = D.sum_over_ranks(wl.n_elem, world, dev)
    value = job_entries * args.steps / (total_ms * 1e-3)
    hist = np.bincount([p2s.CLASS_NPTS.index(int(g)) for g in npts], minlength=6).tolist()
    e2e = None if args.no_e2e else measure_e2e_learned(args, wl, ctx, P, dev, risk)
    line = None
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "entries/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32x2", "data": "synthetic",
            "config": workload_config(args, wl, risk=risk, risk_src=meta.get("risk_calibration")),
            "elements_per_s": job_elems * args.steps / (total_ms * 1e-3),
            "uniform_mixed": dict(uniform, value=job_entries / (uniform["ms_per_step"] * 1e-3), unit="entries/s",
                                  learned_speedup=uniform["ms_per_step"] / (total_ms / args.steps)),
            "plain_fp64": {"value": job_entries / (plain_ms * 1e-3), "unit": "entries/s", "ms_per_step": plain_ms,
                           "npts": 48},
            "speedup_vs_plain_fp64": plain_ms / (total_ms / args.steps),
            "accuracy": {"max_rel_err_vs_plain48": float(err_h.max()), "share_above_1e-8": float((err_h > 1e-8).mean()),
                         "median_rel_err": float(np.median(err_h)), "metric": "per element max over types of max|dM|/max|M|"},
            "learned": {"class_hist": hist, "mean_G3": float(np.mean(npts.astype(float) ** 3)),
                        "judged": rep["judged"], "judge_failed": rep["failed"],
                        "max_judged_err": rep["max_judged_err"], "train": meta},
            "roofline": roof,
            "stages": {"moments_ms": mom_ms, "contract_ms": con_ms,
                       "learned_other_ms": total_ms / args.steps - mom_ms - con_ms},
            "clocks": clocks,
            # per learned fill (launch list): gather, judge moments + contraction, features, predict,
            # set_npts, order_by_class, main moments + contraction, elem_err, judge_mask, fallback
            # moments + contraction (masked), judge_fix
            "gpu_launches": 14 * args.steps,
        }
        if e2e:
            line["e2e"] = e2e
    del out
    lp.close()
    if rank == 0 and world == 1 and not args.no_cpu:
        v, dt, desc, threads, idx, ro, roff, sub = oracle_sample(wl.with_npts(48), cpu_sample_size(args.workload),
                                                                 keep=True)
        line["cpu_baseline"] = {"value": v, "unit": "entries/s", "cores": threads, "kind": "oracle",
                                "sample": desc + " (%.1f s)" % dt}
        ev = errors_vs_oracle(cpu_got, ro, roff, sub)
        line["accuracy"]["vs_oracle48_sample"] = {
            "elements": idx.tolist(), "learned_G": [int(npts[e]) for e in idx], "rel_err": ev,
            "note": "learned fill of the oracle's CPU-sample elements against the oracle's direct triple sums at 48 "
                    "points (quadrature difference of the learned rule plus arithmetic)"}
    if rank == 0:
        line["device_peaks"] = dict(_DEV) or None
        print(json.dumps(line), flush=True)
    ctx.close()
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def measure_e2e_learned(args, wl, ctx, P, dev, risk, chunk_elems=4096):
    """Learned fill through the public API with host buffers: per chunk of elements, pinned
    host inputs -> device, learned fill, every FP64 entry -> pinned host memory; two chunks
    in flight on two streams."""
    import torch

    from paper_1703_09619_gb300 import p2s
    E = wl.n_elem
    subs = [wl.subset(np.arange(s, min(E, s + chunk_elems))) for s in range(0, E, chunk_elems)]
    from paper_1703_09619_gb300 import learned as LN
    plans = [p2s.LearnedPlan(ctx, w.orders, precision=p2s.MIXED, judge_frac=JUDGE_FRAC, seed=1703,
                             judge_tol=JUDGE_TOL, risk=risk, n_nets=LN.n_nets_of(P.cpu().numpy())) for w in subs]
    return _e2e_pipeline(args, wl, subs, plans, dev,
                         lambda p, w, di, o, s: p.fill(w.kind, di[0], di[1], di[2], P, o, stream=s))


def _e2e_pipeline(args, wl, subs, plans, dev, fill):
    import torch
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
                for d, h in zip(di, host_in[i]):
                    d[: h.shape[0]].copy_(h, non_blocking=True)
                n = w.n_elem
                fill(p, w, [di[0][:n], di[1][:n], di[2][:n]], dev_out[i % 2], s)
                host_out[i % 2][: p.output_entries].copy_(dev_out[i % 2][: p.output_entries], non_blocking=True)
        for s in streams:
            s.synchronize()

    one_pass()
    steps = max(1, min(args.steps, 3))
    world = D.env()[0]
    torch.cuda.synchronize()
    D.barrier(world)
    t0 = time.perf_counter()
    for _ in range(steps):
        one_pass()
    dt = D.max_over_ranks((time.perf_counter() - t0) / steps, world, dev)
    for p in plans:
        p.close()
    # the host link bounds this figure: every FP64 entry crosses it once.  Its ceiling is taken
    # the way the pipeline uses it: the same two streams copying their chunk buffers at once.
    link = d2h_bandwidth_streams(host_out, dev_out, streams, [p.output_entries for p in plans[:2]])
    single = d2h_bandwidth(host_out[0], dev_out[0])
    return {"value": D.sum_over_ranks(wl.entries(), world, dev) / dt, "unit": "entries/s", "h2d_bytes_per_step": int(h2d),
            "d2h_bytes_per_step": int(d2h), "steps": steps, "chunks": len(subs),
            "d2h_link_gbs": link, "d2h_single_copy_gbs": single, "d2h_achieved_gbs": d2h / dt / 1e9,
            "frac_of_link": d2h / dt / 1e9 / link,
            "note": "pinned host inputs in, every FP64 entry back to pinned host memory, 2-stream pipeline; "
                    "d2h_link_gbs = the two pipeline streams copying a chunk each, concurrently, device to pinned "
                    "host (best of 3), measured in the same process; d2h_single_copy_gbs = one copy alone"}


def d2h_bandwidth_streams(host, devbuf, streams, counts):
    """GB/s of concurrent device-to-host copies, one per stream, of `counts` doubles each
    (best of 3 rounds, after one warm-up round)."""
    import torch
    best = 0.0
    for r in range(4):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for h, d, s, n in zip(host, devbuf, streams, counts):
            with torch.cuda.stream(s):
                h[:n].copy_(d[:n], non_blocking=True)
        for s in streams:
            s.synchronize()
        dt = time.perf_counter() - t0
        if r > 0:
            best = max(best, 8 * sum(counts) / dt / 1e9)
    return best


def d2h_bandwidth(host, devbuf, nbytes=2 << 30):
    """GB/s of one device-to-host copy of up to 2 GB between the given buffers (median of 3)."""
    import torch
    n = min(host.numel(), devbuf.numel(), nbytes // 8)
    ts = []
    for _ in range(4):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        host[:n].copy_(devbuf[:n], non_blocking=True)
        torch.cuda.synchronize()
        ts.append(time.perf_counter() - t0)
    return 8 * n / sorted(ts[1:])[1] / 1e9


# ----------------------------------------------------------------------------- fixed-G fills
def run_fixed(args, wl):
    import torch

    from paper_1703_09619_gb300 import p2s

    world, rank, local = dist_setup()
    dev = torch.device("cuda", local)
    ctx = p2s.Context(local)
    device_peaks(p2s, ctx)
    prec = p2s.MIXED if args.mode == "mixed" else p2s.FP64
    npts = int(wl.npts[0]) if (wl.npts == wl.npts[0]).all() else wl.npts
    params, nodes, bulge = p2s.device_inputs(wl, dev)
    # tile shapes from the autotuner, launches replayed from a graph (on by default)
    tune = args.tune if args.tune is not None else True
    tile = tune_info = None
    if args.tile:
        vals = [int(x) for x in args.tile.split(",")]
        tile = dict(zip(("combo_target", "unit_kbytes", "threads", "kernel"), vals))
        tune_info = {"tile": tile, "candidates": 0, "note": "given on the command line"}
    elif tune:
        from paper_1703_09619_gb300 import tunecache
        sample = min(wl.n_elem, 1024)
        key = tunecache.signature(wl.orders, npts, prec, wl.types_mask, torch.cuda.get_device_name(dev))
        tile, tune_info = tunecache.tuned_tile(
            lambda: p2s.autotune_tiles(ctx, wl.orders, npts, wl.kind, params, nodes, bulge, prec, wl.types_mask,
                                       sample=sample, reps=3),
            key, sample_elements=sample, workload=args.workload)
        log("autotune (%s): %s" % (tune_info["cache"], tile))
    plan = p2s.Plan(ctx, wl.orders, npts, prec, wl.types_mask, tile=tile, graph=bool(tune or args.tile))
    out = torch.empty(plan.output_entries, dtype=torch.float64, device=dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)

    def step():
        plan.fill(wl.kind, params, nodes, bulge, out, stream=stream)

    for _ in range(args.warmup):
        step()
        flush.zero_()
    torch.cuda.synchronize()
    if ctx.sync_status(stream) != 0:
        raise RuntimeError("device status after warm-up")
    barrier(world)
    with ClockSampler(local) as clk:
        ms = time_steps(step, args.steps, stream, flush)
    barrier(world)
    total_ms = max_over_ranks(float(sum(ms)), world, dev)
    clocks = clk.summary()
    mom_ms, con_ms = stage_times(p2s, ctx, wl, npts, prec, params, nodes, bulge, dev, stream, flush, tile=tile)
    peaks, src = load_peaks()
    roof = roofline_for(wl, wl.npts, prec, mom_ms, con_ms, peaks, src, kernel=plan.tile_config()["kernel"])
    entries = wl.entries()
    job_entries = D.sum_over_ranks(entries, world, dev)  # each rank fills a batch of its own
    job_elems = D.sum_over_ranks(wl.n_elem, world, dev)
    value = job_entries * args.steps / (total_ms * 1e-3)
    e2e = None if args.no_e2e else measure_e2e_fixed(args, wl, ctx, prec, dev, tile, bool(tune or args.tile))
    # the elements of the oracle's CPU sample, for the per-element comparison below
    n_, off_ = p2s.output_entries(wl.orders, wl.types_mask, offsets=True)
    cpu_idx = sample_indices(wl, cpu_sample_size(args.workload))
    cpu_got = [out[int(off_[e]):int(off_[e + 1])].cpu().numpy() for e in cpu_idx]
    line = None
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "entries/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32x2" if prec == p2s.MIXED else "f64",
            "data": "synthetic",
            "config": workload_config(args, wl),
            "elements_per_s": job_elems * args.steps / (total_ms * 1e-3),
            "roofline": roof, "stages": {"moments_ms": mom_ms, "contract_ms": con_ms}, "clocks": clocks,
            "gpu_launches": 2 * args.steps,
        }
        if tune_info:
            line["config"]["launch"] = "one CUDA graph per step (queue reset, moment kernel, contraction kernel)"
            line["autotune"] = tune_info
        if e2e:
            line["e2e"] = e2e
    del out
    plan.close()
    if rank == 0 and world == 1 and not args.no_cpu:
        v, dt, desc, threads, idx, ro, roff, sub = oracle_sample(wl, cpu_sample_size(args.workload), keep=True)
        line["cpu_baseline"] = {"value": v, "unit": "entries/s", "cores": threads, "kind": "oracle",
                                "sample": desc + " (%.1f s)" % dt}
        ev = errors_vs_oracle(cpu_got, ro, roff, sub)
        line["accuracy"] = {"vs_oracle": {"elements": idx.tolist(), "rel_err": ev, "max_rel_err": max(ev),
                                          "bar": 1e-12 if prec == p2s.FP64 else 1e-8,
                                          "metric": "per element max over types of max|dM|/max|M| against the "
                                                    "oracle's direct triple sums at the same rule"}}
    if rank == 0:
        line["device_peaks"] = dict(_DEV) or None
        print(json.dumps(line), flush=True)
    ctx.close()
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def run_operator(args, wl):
    """The diffusion stiffness sum_ab alpha_ab d_a phi_i d_b phi_j of one scalar field (the
    workload's first component) as a term-list operator: one n x n matrix per element."""
    import torch

    from paper_1703_09619_gb300 import p2s

    world, rank, local = dist_setup()
    dev = torch.device("cuda", local)
    ctx = p2s.Context(local)
    device_peaks(p2s, ctx)
    prec = p2s.MIXED if args.precision == "mixed" else p2s.FP64
    orders = np.ascontiguousarray(wl.orders[:, :1, :])
    terms, scales = W.diffusion_terms()
    npts = int(wl.npts[0]) if (wl.npts == wl.npts[0]).all() else wl.npts
    params, nodes, bulge = p2s.device_inputs(wl, dev)
    tile = None
    if args.tile:
        vals = [int(x) for x in args.tile.split(",")]
        tile = dict(zip(("combo_target", "unit_kbytes", "threads", "kernel"), vals))
    plan = p2s.OperatorPlan(ctx, orders, npts, terms, scales, wl.kind, prec, tile=tile, graph=True)
    out = torch.empty(plan.output_entries, dtype=torch.float64, device=dev)
    mom = torch.empty(max(plan.moment_entries, 1), dtype=torch.float64, device=dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)

    def step():
        plan.fill(wl.kind, params, nodes, bulge, out, stream=stream)

    for _ in range(args.warmup):
        step()
        flush.zero_()
    torch.cuda.synchronize()
    if ctx.sync_status(stream) != 0:
        raise RuntimeError("device status after warm-up")
    barrier(world)
    with ClockSampler(local) as clk:
        ms = time_steps(step, args.steps, stream, flush)
    barrier(world)
    total_ms = max_over_ranks(float(sum(ms)), world, dev)
    clocks = clk.summary()
    m = time_steps(lambda: plan.moments(wl.kind, params, nodes, bulge, mom, stream=stream), 3, stream, flush)
    c = time_steps(lambda: plan.contract(mom, out, stream=stream), 3, stream, flush)
    mom_ms, con_ms = float(np.mean(m)), float(np.mean(c))
    entries = plan.output_entries
    job_entries = D.sum_over_ranks(entries, world, dev)
    value = job_entries * args.steps / (total_ms * 1e-3)
    fmas = operator_fma_count(orders, terms, symmetric=True)
    if prec == p2s.FP64:
        ach = 2 * fmas / (con_ms * 1e-3) / 1e12
        roof = {"bound": "alu", "kernel": "k_contract<ArithF64> (operator terms)", "achieved": ach,
                "peak": fp64_peak(), "unit": "TFLOP/s", "frac": ach / fp64_peak(), "traffic": None,
                "peak_source": peak_source("fp64"),
                "algorithmic_flop_per_launch": 2 * fmas}
    else:  # float-float MACs: bound by FP32 issue (12 lane operations per MAC, as the moment kernel)
        ops = DW_MAC_OPS * fmas
        ach = ops / (con_ms * 1e-3) / 1e12
        uniform = bool((orders == orders[0, 0, 0]).all()) and 2 <= int(orders[0, 0, 0]) <= 6
        kname = "k_contract_opn<%d> (operator terms)" % orders[0, 0, 0] if uniform else "k_contract<ArithFF> (operator terms)"
        roof = {"bound": "alu", "kernel": kname, "achieved": ach,
                "peak": fp32_issue_peak(), "unit": "T FP32 lane-op/s", "frac": ach / fp32_issue_peak(), "traffic": None,
                "peak_source": peak_source("fp32"),
                "algorithmic_ops_per_launch": ops,
                "op_model": "%d per float-float MAC x %d MACs of the three sparse stages" % (DW_MAC_OPS, fmas),
                "hbm_write_GBs": 8 * entries / (con_ms * 1e-3) / 1e9}
    line = None
    if rank == 0:
        cfg = workload_config(args, wl)
        cfg.update({"operator": "diffusion stiffness of one scalar field, 9 terms alpha_ab d_a d_b (symmetric)",
                    "orders": "uniform %d" % orders[0, 0, 0] if (orders == orders[0, 0, 0]).all() else "mixed",
                    "n_comp": 1, "entries_per_step": entries, "precision": args.precision or "fp64",
                    "launch": "one CUDA graph per step"})
        line = {
            "metric": METRIC, "value": value, "unit": "entries/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64" if prec == p2s.FP64 else "f32x2",
            "data": "synthetic", "config": cfg,
            "elements_per_s": D.sum_over_ranks(wl.n_elem, world, dev) * args.steps / (total_ms * 1e-3),
            "roofline": roof, "stages": {"moments_ms": mom_ms, "contract_ms": con_ms}, "clocks": clocks,
            "gpu_launches": 2 * args.steps,
        }
    del out, mom
    plan.close()
    if rank == 0 and world == 1 and not args.no_cpu:
        import oracle
        sub = wl.subset(np.arange(min(16, wl.n_elem)))
        threads = oracle.default_threads()
        t0 = time.perf_counter()
        _, off, _ = oracle.fill_terms(np.ascontiguousarray(sub.orders[:, :1, :]), sub.kind, sub.params, sub.nodes,
                                      sub.bulge, npts if np.isscalar(npts) else sub.npts, terms, scales, threads)
        dt = time.perf_counter() - t0
        line["cpu_baseline"] = {"value": float(off[-1]) / dt, "unit": "entries/s", "cores": threads, "kind": "oracle",
                                "sample": "first %d elements, every entry of the operator (%.1f s)" % (sub.n_elem, dt)}
    if rank == 0:
        line["device_peaks"] = dict(_DEV) or None
        print(json.dumps(line), flush=True)
    ctx.close()
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def run_assembly(args):
    """Fill plus global assembly of the diffusion stiffness on a conforming structured mesh of
    curved hexahedra (one scalar field, order N per axis): element matrices by the operator fill,
    then the hierarchic-basis transform and the 8-colour scatter into one CSR matrix."""
    import torch

    from paper_1703_09619_gb300 import p2s

    world, rank, local = dist_setup()
    dev = torch.device("cuda", local)
    ctx = p2s.Context(local)
    device_peaks(p2s, ctx)
    prec = p2s.FP64 if args.precision == "fp64" else p2s.MIXED
    nx, ny, nz = (int(x) for x in args.mesh.split(","))
    N, G = args.order, args.npts or 8
    mesh = W.make_mesh(nx, ny, nz, N, G, seed=7 + rank)  # weak scaling: one mesh per rank
    wl = mesh.workload
    terms, scales = W.diffusion_terms()
    asm = p2s.Assembly(ctx, nx, ny, nz, N, G, terms, scales, wl.kind, prec, graph=True)
    params, nodes, bulge = p2s.device_inputs(wl, dev)
    vals = torch.empty(asm.nnz, dtype=torch.float64, device=dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)

    def step():
        asm.fill(wl.kind, params, nodes, bulge, vals, stream=stream)

    for _ in range(args.warmup):
        step()
        flush.zero_()
    torch.cuda.synchronize()
    if ctx.sync_status(stream) != 0:
        raise RuntimeError("device status after warm-up")
    barrier(world)
    with ClockSampler(local) as clk:
        ms = time_steps(step, args.steps, stream, flush)
    barrier(world)
    total_ms = max_over_ranks(float(sum(ms)), world, dev)
    clocks = clk.summary()
    # the assembly stage alone on the last fill: memset + 8 colour launches (fused: the operator
    # contraction from the kept moments + basis change + scatter; otherwise the assembly kernel)
    a = time_steps(lambda: asm.reassemble(vals, stream=stream), 3, stream, flush)
    add_ms = float(np.mean(a))
    fill_ms = total_ms / args.steps - add_ms
    n = N ** 3
    E = wl.n_elem
    contributions = E * n * n
    if asm.fused:  # contraction + basis change + scatter in one kernel: the double-word MACs dominate
        fmas = operator_fma_count(wl.orders, terms, symmetric=True)
        ops = DW_MAC_OPS * fmas
        ach = ops / (add_ms * 1e-3) / 1e12
        roof = {"bound": "alu", "kernel": "k_opn_assemble<%d> (memset + 8 colour launches)" % N, "achieved": ach,
                "peak": fp32_issue_peak(), "unit": "T FP32 lane-op/s", "frac": ach / fp32_issue_peak(), "traffic": None,
                "peak_source": peak_source("fp32"),
                "algorithmic_ops_per_launch": ops,
                "op_model": "%d per float-float MAC x %d MACs of the operator contraction (basis change and "
                            "scatter not counted)" % (DW_MAC_OPS, fmas),
                "hbm_values_GBs": 16 * asm.nnz / (add_ms * 1e-3) / 1e9}
    elif prec == p2s.MIXED:
        peaks, src = load_peaks()
        alg_bytes = 8 * contributions + 8 * asm.nnz
        ach = alg_bytes / (add_ms * 1e-3) / 1e9
        roof = {"bound": "hbm", "kernel": "k_assemble_staged<%d, float-float> (memset + 8 colour launches)" % N,
                "achieved": ach, "peak": peaks["hbm_gbs"], "unit": "GB/s", "frac": ach / peaks["hbm_gbs"],
                "traffic": None, "peak_source": "%s copy bandwidth (MEASURED_PEAKS.json)" % src,
                "algorithmic_bytes_per_launch": alg_bytes,
                "bytes_model": "element matrices read once (8 E n^2) + global values written once (8 nnz)"}
    else:  # the FP64 basis change: 12 FP64 operations per entry (6 axes x subtract + scale)
        ops = 12 * contributions
        ach = ops / (add_ms * 1e-3) / 1e12
        peak = fp64_peak() / 2
        roof = {"bound": "alu", "kernel": "k_assemble_staged<%d, FP64> (memset + 8 colour launches)" % N,
                "achieved": ach, "peak": peak, "unit": "T FP64 op/s", "frac": ach / peak, "traffic": None,
                "peak_source": peak_source("fp64") + ", one operation per DADD/DMUL",
                "algorithmic_ops_per_launch": ops, "op_model": "12 FP64 operations per element-matrix entry"}
    job = D.sum_over_ranks(contributions, world, dev)
    line = None
    if rank == 0:
        cfg = {"workload": "%dx%dx%d conforming curved hexahedra, diffusion stiffness, N=%d, G=%d" % (nx, ny, nz, N, G),
               "elements": E, "order": N, "npts": G, "rows": asm.rows, "nnz": asm.nnz,
               "element_entries": contributions, "precision": "fp64" if prec == p2s.FP64 else "mixed",
               "basis": "hierarchic C0 (vertex + integrated Legendre)",
               "scatter": "8 lattice colours, one red.global.add.f64 per entry (at most one per position and colour)",
               "launch": ("moments, memset, 8 colour launches of the fused contraction + assembly" if asm.fused
                          else "fill from a CUDA graph, memset, 8 colour launches"),
               "path": "fused (no element-matrix scratch)" if asm.fused else "fill, then assembly",
               "l2": "global values (%.2f GB) and element matrices (%.2f GB) exceed L2; L2 flushed between steps"
                     % (8e-9 * asm.nnz, 8e-9 * contributions)}
        line = {
            "metric": "element-matrix entries assembled/s (fill + global CSR assembly)",
            "value": job * args.steps / (total_ms * 1e-3), "unit": "entries/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64" if prec == p2s.FP64 else "f32x2", "data": "synthetic", "config": cfg,
            "nnz_per_s": D.sum_over_ranks(asm.nnz, world, dev) * args.steps / (total_ms * 1e-3),
            "roofline": roof, "stages": {"fill_ms": fill_ms, "assemble_ms": add_ms}, "clocks": clocks,
            "gpu_launches": (9 if asm.fused else 10) * args.steps,  # moments (+ contraction), 8 colours
        }
    del vals
    asm.close()
    if rank == 0 and world == 1 and not args.no_cpu:
        import oracle
        from oracle import assembly as oasm
        sm = W.make_mesh(6, 6, 6, N, G, seed=7)
        sw = sm.workload
        threads = oracle.default_threads()
        t0 = time.perf_counter()
        out, _, _ = oracle.fill_terms(sw.orders, sw.kind, sw.params, sw.nodes, sw.bulge, G, terms, scales, threads)
        oasm.assemble(6, 6, 6, N, out.reshape(sw.n_elem, n, n))
        dt = time.perf_counter() - t0
        line["cpu_baseline"] = {"value": sw.n_elem * n * n / dt, "unit": "entries/s", "cores": threads, "kind": "oracle",
                                "sample": "a 6x6x6 mesh of the same recipe: oracle fill + dense assembly (%.1f s)" % dt}
    if rank == 0:
        line["device_peaks"] = dict(_DEV) or None
        print(json.dumps(line), flush=True)
    ctx.close()
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


# Table I of the paper (M = N): matrix-filling reduction factor, direct / product-to-sum, measured on
# its CPU ("from the left columns") and predicted by the Sec. IV operation count (D/15).
TABLE_I_REDUCTION = {3: (0.96, 0.6), 4: (1.22, 1.0), 6: (2.5, 2.4), 8: (4.8, 4.25), 10: (7.25, 6.7),
                     12: (10.0, 9.6), 14: (13.0, 13.0), 16: (15.0, 17.0), 18: (17.0, 21.6)}


def run_cheb2d(args):
    """The paper's 2-D curl-curl example (Sec. III): stiffness and mass element matrices of the
    Fig. 1 domain meshed into nx x ny curved quadrilaterals, orders M = N of Table I; the
    product-to-sum fill (FP64 and mixed) against direct numerical integration (FP64), same rule."""
    import torch

    from paper_1703_09619_gb300 import p2s

    world, rank, local = dist_setup()
    dev = torch.device("cuda", local)
    ctx = p2s.Context(local)
    device_peaks(p2s, ctx)
    nx, ny = (int(x) for x in args.mesh2d.split(","))
    orders = [int(x) for x in args.orders.split(",")]
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)
    rows, head = [], None
    with ClockSampler(local) as clk:
        for M in orders:
            G = W.cheb2d_npts(M)
            mesh = W.make_mesh2d(nx, ny, M, G)
            n = p2s.cheb2d_dofs(M, M)
            E = mesh.n_elem
            dp = torch.as_tensor(mesh.params, device=dev)
            S = torch.empty((E, n, n), dtype=torch.float64, device=dev)
            Mm = torch.empty_like(S)
            fill = lambda method, prec: p2s.cheb2d_fill(ctx, dp, M, M, G, S, Mm, method, prec, stream=stream)
            times = {}
            for key, method, prec, reps in (("p2s_mixed", p2s.CHEB2D_P2S, p2s.MIXED, args.steps),
                                            ("p2s_fp64", p2s.CHEB2D_P2S, p2s.FP64, args.steps),
                                            ("direct_fp64", p2s.CHEB2D_DIRECT, p2s.FP64, 1 if M >= 14 else 2)):
                for _ in range(args.warmup if method == p2s.CHEB2D_P2S else 1):
                    fill(method, prec)
                torch.cuda.synchronize()
                barrier(world)
                ms = time_steps(lambda: fill(method, prec), reps, stream, flush)
                times[key] = max_over_ranks(float(np.median(ms)), world, dev)
            if ctx.sync_status(stream) != 0:
                raise RuntimeError("device status after the %d-order fills" % M)
            entries = 2 * E * n * n
            ti = TABLE_I_REDUCTION.get(M)
            rows.append({"M": M, "G": G, "dofs": n, "entries": entries, "ms": times,
                         "gpu_reduction_fp64": times["direct_fp64"] / times["p2s_fp64"],
                         "gpu_reduction_mixed": times["direct_fp64"] / times["p2s_mixed"],
                         "table_I_reduction": ti[0] if ti else None, "table_I_model_D_over_15": ti[1] if ti else None})
            head = (M, G, n, E, entries, times)
            del S, Mm
    clocks = clk.summary()
    M, G, n, E, entries, times = head
    peaks, src = load_peaks()
    job = D.sum_over_ranks(entries, world, dev)
    ach = 8 * entries / (times["p2s_mixed"] * 1e-3) / 1e9
    roof = {"bound": "hbm", "kernel": "k_cheb2d_p2s<float-float> (order %d)" % M, "achieved": ach,
            "peak": peaks["hbm_gbs"], "unit": "GB/s", "frac": ach / peaks["hbm_gbs"], "traffic": None,
            "peak_source": "%s copy bandwidth (MEASURED_PEAKS.json)" % src,
            "algorithmic_bytes_per_launch": 8 * entries, "bytes_model": "every FP64 entry of S and M written once"}
    macs = entries * G * G  # the direct method: one multiply-add per point and entry (Sec. IV)
    dach = 2 * macs / (times["direct_fp64"] * 1e-3) / 1e12
    roof_direct = {"bound": "alu", "kernel": "k_cheb2d_direct (order %d)" % M, "achieved": dach,
                   "peak": fp64_peak(), "unit": "TFLOP/s", "frac": dach / fp64_peak(),
                   "peak_source": peak_source("fp64"),
                   "flop_model": "2 flop per Gauss point and entry (the paper's direct count)"}
    if rank == 0:
        line = {
            "metric": "2-D curl-curl element-matrix entries/s (Sec. III example), product to sum, order %d" % M,
            "value": job / (times["p2s_mixed"] * 1e-3), "unit": "entries/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": times["p2s_mixed"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32x2", "data": "synthetic",
            "config": {"workload": "Fig. 1 domain, %dx%d curved quadrilaterals, M = N = %d, G = %d, S and M" % (nx, ny, M, G),
                       "elements": E, "dofs_per_element": n, "orders": orders,
                       "l2": "outputs exceed L2 at the larger orders; L2 flushed (256 MB write) between steps"},
            "orders": rows, "roofline": roof, "roofline_direct": roof_direct, "clocks": clocks,
            "gpu_launches": 1,
        }
        if world == 1 and not args.no_cpu:
            from oracle import cheb2d as oc2
            mesh = W.make_mesh2d(nx, ny, M, G)
            t0 = time.perf_counter()
            oc2.element_matrices(mesh.params[0], M, M, G)
            dt = time.perf_counter() - t0
            line["cpu_baseline"] = {"value": 2 * n * n / dt, "unit": "entries/s", "cores": 1, "kind": "oracle",
                                    "sample": "element 0 at order %d: S and M by direct sums in numpy (%.1f s)" % (M, dt)}
        line["device_peaks"] = dict(_DEV) or None
        print(json.dumps(line), flush=True)
    ctx.close()
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def measure_e2e_fixed(args, wl, ctx, prec, dev, tile=None, graph=False):
    from paper_1703_09619_gb300 import p2s
    E = wl.n_elem
    per_elem = wl.entries() / E
    chunk = int(max(1, min(E, (2 << 30) // (8 * per_elem))))
    subs = [wl.subset(np.arange(s, min(E, s + chunk))) for s in range(0, E, chunk)]
    npts = lambda w: int(w.npts[0]) if (w.npts == w.npts[0]).all() else w.npts
    plans = [p2s.Plan(ctx, w.orders, npts(w), prec, w.types_mask, tile=tile, graph=graph) for w in subs]
    return _e2e_pipeline(args, wl, subs, plans, dev,
                         lambda p, w, di, o, s: p.fill(w.kind, di[0], di[1], di[2], o, stream=s))


def run_mode1(args, n_src=65536, n_rows=1 << 24):
    """The first mode product of the moments (the a-axis sum of Eq. (4), K = 7) in its two
    forms on the same rows: double-word SIMT (the moment kernel's phase B) and the
    split-precision tensor-core form (tcgen05, 4 and 5 slices).  Rows are double-word
    samples of a c5-like coupling factor, read from a 65 536-row source (L2-resident) so
    that arithmetic, not HBM, is timed; 16.8 M rows per launch, CUDA events, L2 flushed
    between launches.  Reports time per row and per point for each G of the learned classes."""
    import torch

    from paper_1703_09619_gb300 import p2s

    world, rank, local = dist_setup()
    dev = torch.device("cuda", local)
    ctx = p2s.Context(local)
    device_peaks(p2s, ctx)
    stream = torch.cuda.current_stream(dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    out = torch.empty((n_rows, 8, 2), dtype=torch.float32, device=dev)
    rng = np.random.default_rng(17)
    res = {}
    for G in (16, 24, 32, 48):
        u = np.polynomial.legendre.leggauss(G)[0]
        x = 1 + 0.8 * np.sin(rng.uniform(1, 40, (n_src, 1)) * u + rng.uniform(0, 6, (n_src, 1)))
        x *= rng.uniform(0.5, 2.0, (n_src, 1))
        hi = x.astype(np.float32)
        xs = np.stack([hi, (x - hi).astype(np.float32)], axis=-1)
        xd = torch.as_tensor(np.ascontiguousarray(xs), device=dev)
        row = {}
        ref = None
        for name, method, sl in (("simt", p2s.MODE1_SIMT, 4), ("tc4", p2s.MODE1_TC, 4), ("tc5", p2s.MODE1_TC, 5)):
            call = lambda: p2s.mode1_product(ctx, method, G, xd, n_rows, out, slices=sl, stream=stream)
            for _ in range(args.warmup):
                call()
            ms = float(np.median(time_steps(call, max(3, args.steps), stream, flush)))
            o = out[:n_src].double()
            T = (o[..., 0] + o[..., 1]).cpu().numpy()
            if ref is None:
                ref = T
            row[name] = {"ms": ms, "ns_per_row": 1e6 * ms / n_rows, "ns_per_point": 1e6 * ms / (n_rows * G),
                         "max_rel_diff_vs_simt": float(np.abs(T - ref).max() / np.abs(ref).max())}
        row["tc4_speedup"] = row["simt"]["ms"] / row["tc4"]["ms"]
        row["tc5_speedup"] = row["simt"]["ms"] / row["tc5"]["ms"]
        res["G%d" % G] = row
        log("mode1 G=%d: %s" % (G, json.dumps(row)))
    rc = ctx.sync_status()
    line = None
    if rank == 0:
        g = res["G24"]
        line = {"metric": "first-mode moment product rows/s (Eq. (4) a-axis sum, K = 7), tensor core vs SIMT",
                "value": n_rows / (g["tc4"]["ms"] * 1e-3), "unit": "rows/s", "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": g["tc4"]["ms"], "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f16x4 slices, f32 accumulate", "data": "synthetic",
                "config": {"workload": "mode1: %d rows per launch from a %d-row L2-resident source, G = 16..48"
                                       % (n_rows, n_src), "rows": n_rows},
                "results": res, "device_status": rc, "gpu_launches": 3 * 4 * (args.warmup + max(3, args.steps))}
        line["device_peaks"] = dict(_DEV) or None
        print(json.dumps(line), flush=True)
    ctx.close()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="c5", choices=["c1", "c2", "c3", "c4", "c5"])
    ap.add_argument("--mode", default=None, choices=["learned", "plain", "mixed", "operator", "assembly", "cheb2d", "mode1"])
    ap.add_argument("--mesh2d", default="32,32", help="cheb2d mode: elements nx,ny (ny even)")
    ap.add_argument("--orders", default="3,4,6,8,10,12,14,16,18", help="cheb2d mode: orders M = N (Table I)")
    ap.add_argument("--mesh", default="32,32,32", help="assembly mode: elements per axis nx,ny,nz")
    ap.add_argument("--order", type=int, default=4, help="assembly mode: order N per axis")
    ap.add_argument("--precision", default=None, choices=["fp64", "mixed"], help="alias of --mode plain|mixed")
    ap.add_argument("--elements", type=int, default=None, help="use only the first E elements")
    ap.add_argument("--npts", type=int, default=None, help="override the quadrature size G")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--tune", dest="tune", action="store_true", default=None,
                    help="autotune the contraction tiles and replay fills from a CUDA graph (default: on)")
    ap.add_argument("--no-tune", dest="tune", action="store_false")
    ap.add_argument("--tile", default=None,
                    help="contraction tile combo_target,unit_kbytes,threads[,kernel] (skips the autotuner)")
    args = ap.parse_args()
    if args.mode is None:
        args.mode = {"fp64": "plain", "mixed": "mixed"}.get(args.precision) or (
            "learned" if args.workload == "c5" else "plain")
    if args.mode == "assembly" and args.impl == "ours":
        run_assembly(args)
        return
    if args.mode == "cheb2d" and args.impl == "ours":
        run_cheb2d(args)
        return
    if args.mode == "mode1" and args.impl == "ours":
        run_mode1(args)
        return
    wl = W.make(args.workload, args.elements, shard=D.env()[1])  # weak scaling: a batch per rank
    if args.npts:
        wl = wl.with_npts(args.npts)
    if args.impl == "reference":
        if args.mode == "learned":
            wl = wl.with_npts(48)
        run_reference(args, wl)
    elif args.mode == "operator":
        if wl.kind != W.KIND_METRIC_EPS:
            raise SystemExit("the operator mode takes the metric coupling of a curved workload (c2, c4, c5)")
        run_operator(args, wl)
    elif args.mode == "learned":
        if wl.kind != W.KIND_METRIC_EPS:
            raise SystemExit("the learned mode needs a three-component metric workload (c2, c4, c5)")
        run_learned(args, wl)
    else:
        run_fixed(args, wl)


if __name__ == "__main__":
    main()
