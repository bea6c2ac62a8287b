#!/usr/bin/env python3
"""Throughput benchmark: LLG node-steps/s of adaptive Dormand-Prince 5(4) integration with the full
effective field (exchange, uniaxial anisotropy, FFT demag), FP32 field evaluation with FP64 state
(the library's NM_F32 mode), beside the plain FP64 path, on one GB300 per rank.

One "step" is one DP5 step attempt of the whole hot path: six effective-field evaluations (node->cell
average, five demag FFT passes, fused local stencil and LLG right-hand side with stage formation),
the FP64 error norm with device-side step control, and the accepted update with renormalisation.

  python bench.py [--gpus N --steps K --warmup W] [--grid 1024x1024x32] [--impl ours|reference]

The line also carries `serving`: Poisson streams of mixed-size LLG runs (grids 64..256 x 64..256 x 1..8
cells, per-run material, field and duration) through the library's request loop at 0.7x and 1.2x the
one-at-a-time capacity, with p50/p99 latency, throughput and occupancy (--serve-requests 0 skips it).

Prints one JSON line (rank 0).  Under torchrun every rank integrates its own replica (no data-path
collective: independent runs shard trivially); the time is the max over ranks.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import nm_inputs as inp  # noqa: E402

METRIC = "LLG node-steps/s (h_eff incl. FFT demag) FP32 vs plain FP64; serving p50/p99"
UNIT = "node-steps/s"


# ----------------------------------------------------------------------------------------- helpers
def parse_grid(s):
    v = tuple(int(x) for x in s.lower().split("x"))
    assert len(v) == 3
    return v


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def csrc_hash():
    h = hashlib.sha256()
    d = os.path.join(ROOT, "paper_2411_11725_gb300", "csrc")
    for f in sorted(os.listdir(d)):
        with open(os.path.join(d, f), "rb") as fh:
            h.update(f.encode() + fh.read())
    return h.hexdigest()[:16]


class ClockSampler:
    """nvidia-smi clock/throttle sampling while the timed region runs."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.th = threading.Thread(target=self._read, daemon=True)
            self.th.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.th.join(timeout=2)
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax = float(f[2])
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


def algorithmic_bytes(name, stage, n, b, with_maps):
    """Bytes a launch must move at minimum: its inputs read once and its outputs written once, with the
    zero padding of the FFT grid neither read nor written (the pruned passes skip it).
    n = (N1, N2, N3); b = bytes per real (4 or 8); stage = DP5 stage index of node kernels."""
    N1, N2, N3 = n
    Nn = (N1 + 1) * (N2 + 1) * (N3 + 1)
    Nc = N1 * N2 * N3

    def pad(v):
        if v == 1:
            return 1
        p = 1
        while p < 2 * v - 1:
            p *= 2
        return p
    P1, P2, P3 = pad(N1), pad(N2), pad(N3)
    X = P1 // 2 + 1
    H2, H3 = P2 // 2 + 1, P3 // 2 + 1
    c = 2 * b  # complex
    ms = b * Nc if with_maps else 0
    if name == "demag_x_fwd":
        return 3 * b * Nn + ms + 3 * c * X * N2 * N3
    if name == "demag_y_fwd":
        return 3 * c * X * N2 * N3 + 3 * c * X * P2 * N3
    if name == "demag_z_conv":
        return 2 * 3 * c * X * P2 * N3 + 6 * b * X * H2 * H3
    if name == "demag_y_inv":
        return 3 * c * X * P2 * N3 + 3 * c * X * N2 * N3
    if name == "demag_y_conv":
        return 2 * 3 * c * X * N2 + 6 * b * X * H2
    if name == "demag_x_inv":
        return 3 * c * X * N2 * N3 + ms + 3 * b * Nc
    # stage inputs and the error scale read the FP64 m (24 B/node), or in the FP32 path its FP32 copy
    mb = 3 * b if b == 4 else 24
    if name == "node_llg_stage":
        # y_s, Ms*H_c, 1/mass in; k_s out; for s < 7 also m, the k_j with non-zero a_{s+1,j}
        # (j < s), and y_{s+1} out
        base = 3 * b * Nn + 3 * b * Nc + b * Nn + 3 * b * Nn
        if stage < 7:
            nk = {2: 1, 3: 2, 4: 3, 5: 4, 6: 4}[stage]
            base += mb * Nn + nk * 3 * b * Nn + 3 * b * Nn
        return base
    if name == "stage_input":
        return mb * Nn + 3 * b * Nn + 3 * b * Nn
    if name == "dp5_error_control":
        return mb * Nn + 6 * 3 * b * Nn + b * Nn
    if name == "dp5_update":
        # m in and out (FP64), b_j k_j (j = 1, 3..6) and k7 in, k1 <- k7 out, FP32 copy of m out
        return 24 * Nn + 6 * 3 * b * Nn + 24 * Nn + 3 * b * Nn + (3 * b * Nn if b == 4 else 0)
    return 0


def fp64_line(nmgb, value64, ms64, k64, value32, prof64, nn, wl_key):
    """The plain FP64 path: node-steps/s, and its roofline against GB300's FP64 rate (ALU-bound: the FP64
    pipe is far slower than HBM here).  peak = the library's FP64 fused multiply-add probe; FP64
    operations per node and step from the committed ncu counts (profiles/fp64_flops.txt: DADD + DMUL +
    2 DFMA of one step, per node), used only while the sources match the capture."""
    out = {"value": value64, "unit": UNIT, "ms_per_step": ms64 / k64 if k64 else None, "steps": k64,
           "fp32_over_fp64": value32 / value64 if value64 else None}
    if not value64:
        return out
    if prof64:
        out["kernels_ms"] = {}
        for name, t in prof64:
            out["kernels_ms"][name] = out["kernels_ms"].get(name, 0.0) + t
    try:
        peak = nmgb.measure_peak(1)
    except Exception as e:
        out["roofline"] = {"error": f"{type(e).__name__}: {e}"}
        return out
    flops_node = None
    try:
        with open(os.path.join(ROOT, "profiles", "fp64_flops.txt")) as f:
            d = json.load(f)
        if d.get("csrc_sha") == csrc_hash():
            flops_node = float(d["flops_per_node_step"])
    except Exception:
        pass
    achieved = flops_node * nn * (value64 / nn) / 1e12 if flops_node else None
    out["roofline"] = {"bound": "alu", "unit": "TFLOP/s", "peak": peak / 1e12,
                       "peak_source": "nm_measure_peak(FP64): fused multiply-add chains on every SM",
                       "flops_per_node_step": flops_node, "achieved": achieved,
                       "frac": achieved / (peak / 1e12) if achieved else None}
    return out


def traffic_for(name, workload_key):
    """dram bytes per launch from the committed ncu summary, if it matches the current kernels."""
    p = os.path.join(ROOT, "profiles", "dram_traffic.txt")
    try:
        with open(p) as f:
            d = json.load(f)
    except Exception:
        return None
    if d.get("csrc_sha") != csrc_hash():
        return None
    ent = d.get("kernels", {}).get(name)
    if not ent:
        return None
    scale = ent.get("scale_to", {}).get(workload_key)
    v = ent.get("bytes_per_launch")
    if v is None:
        return None
    return float(v) * (scale if scale else 1.0) if (scale or ent.get("workload") == workload_key) else None


class RankReducer:
    """Max / sum of a scalar over the ranks of a process group (or the value itself without one), and a
    barrier.  Timing takes the max over ranks; counts are summed."""

    def __init__(self, dist=None, device="cuda"):
        self.dist, self.device = dist, device

    def _reduce(self, x, op):
        if self.dist is None:
            return float(x)
        import torch
        t = torch.tensor([float(x)], dtype=torch.float64, device=self.device)
        self.dist.all_reduce(t, op=op)
        return float(t.item())

    def max(self, x):
        return self._reduce(x, None if self.dist is None else self.dist.ReduceOp.MAX)

    def sum(self, x):
        return self._reduce(x, None if self.dist is None else self.dist.ReduceOp.SUM)

    def barrier(self):
        if self.dist is not None:
            self.dist.barrier()


def whole_job_rate(red, units_per_item, items_this_rank, seconds_this_rank):
    """Aggregate rate of all ranks: units processed by all ranks / the slowest rank's time."""
    return units_per_item * red.sum(items_this_rank) / red.max(seconds_this_rank)


# ----------------------------------------------------------------------------------------- arms
def oracle_sample(seconds=15.0, grid=(32, 32, 4), max_steps=None, threads=None):
    """Time the FP64 oracle (direct-sum demag) on a bounded sample: DP5 steps on a smaller cuboid of
    the same material and cell size, on all host cores or on `threads` of them.  Returns (node-steps/s,
    cores, steps, seconds, description)."""
    import oracle
    oracle.build()
    all_threads = oracle.num_threads()
    if threads:
        oracle.set_num_threads(threads)
    p = inp.throughput(grid, 0)
    me = oracle.Mesh(p.n, p.dx)
    me.set_material(p.Ms, p.A, p.Ku, p.axis, p.alpha, p.gamma)
    st = me.dp5_stepper(p.m0, 0.0, 1e-15, p.terms, rtol=1e-5, atol=1e-5)
    me.tensor()  # set-up outside the timed sample
    t0 = time.perf_counter()
    steps = 0
    while True:
        st.step()
        steps += 1
        el = time.perf_counter() - t0
        if el > seconds or (max_steps and steps >= max_steps):
            break
    nn = int(np.prod(p.nodes))
    desc = (f"oracle DP5(4) steps on {grid[0]}x{grid[1]}x{grid[2]} cells (same material and 3 nm cells, "
            f"direct O(N^2) demag, FP64), {steps} steps in {el:.1f} s; the oracle's cost per node grows "
            f"with N, so this over-states its rate on the full grid")
    used = oracle.num_threads()
    if threads:
        oracle.set_num_threads(all_threads)
    return nn * st.n_acc / el, used, steps, el, desc


def run_reference(args, rank, world):
    if rank != 0:
        return
    W, K = args.warmup, args.steps
    import oracle
    oracle.build()
    p = inp.throughput((32, 32, 4), 0)
    me = oracle.Mesh(p.n, p.dx)
    me.set_material(p.Ms, p.A, p.Ku, p.axis, p.alpha, p.gamma)
    me.tensor()
    st = me.dp5_stepper(p.m0, 0.0, 1e-15, p.terms, rtol=1e-5, atol=1e-5)
    for _ in range(W):
        st.step()
    a0 = st.n_acc
    t0 = time.perf_counter()
    for _ in range(K):
        st.step()
    el = time.perf_counter() - t0
    nn = int(np.prod(p.nodes))
    v = nn * (st.n_acc - a0) / el
    desc = (f"FP64 CPU oracle, DP5(4) steps on 32x32x4 cells of the throughput material (direct-sum demag); "
            f"a bounded sample of the {args.grid} workload, which the O(N^2) oracle cannot run")
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": world, "steps": K,
            "warmup": W, "ms_per_step": el / K * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"cuboid {args.grid} cells, 3 nm, Ms=1e6 A/m, A=1.5e-11 J/m, Ku=5e5 J/m^3 "
                                   f"along z, DP5(4) rtol=atol=1e-5 (sampled on 32x32x4)"},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
                             "sample": desc},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_ours(args, rank, world, dist):
    import torch
    import paper_2411_11725_gb300 as nmgb

    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    n = parse_grid(args.grid)
    W, K = args.warmup, args.steps
    p = inp.throughput(n, seed=rank, with_m0=False)
    m0 = inp.unit_vectors(np.random.default_rng(rank), p.nodes)
    nn = int(np.prod(p.nodes))
    stream = torch.cuda.Stream()

    def make(prec):
        me = nmgb.Mesh(p.n, p.dx, prec, stream=stream)
        me.set_material(p.Ms, p.A, p.Ku, p.axis, p.alpha, p.gamma)
        me.set_terms(p.terms)
        me.set_state(m0, 0.0, 1e-15)
        return me

    red = RankReducer(dist, "cuda")

    def barrier():
        red.barrier()

    def timed_steps(me, k):
        torch.cuda.synchronize()
        barrier()
        torch.cuda.synchronize()
        a0, r0, _ = me.counters()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        me.run_steps(k, nmgb.DP54, 1e-5, 1e-5)
        e1.record(stream)
        e1.synchronize()
        torch.cuda.synchronize()
        barrier()
        ms = e0.elapsed_time(e1)
        a1, r1, err = me.counters()
        return ms, a1 - a0, r1 - r0

    max_over_ranks = red.max
    sum_over_ranks = red.sum

    # ---- FP32 (mixed) path: the headline
    me = make(nmgb.F32)
    me.run_steps(W, nmgb.DP54, 1e-5, 1e-5)
    me.sync()
    clk = ClockSampler(local)
    clk.start()
    ms, acc, rej = timed_steps(me, K)
    clocks = clk.stop()
    value = whole_job_rate(red, nn, acc, ms * 1e-3)
    ms_max = max_over_ranks(ms)
    acc_tot = sum_over_ranks(acc)
    evals = 6 * (acc + rej)  # DP5(4) with FSAL: six field evaluations per attempted step
    evals_tot = sum_over_ranks(evals)
    # per-launch timing for the roofline (CUDA events between launches on the mesh stream)
    prof = me.profile_step(nmgb.DP54, reps=3)
    # ---- e2e: the public API with host buffers, every step: H2D of m, one step, D2H of m
    e2e_value, ke = None, 0
    if args.e2e_steps > 0:
        m_host = torch.from_numpy(m0.copy()).pin_memory()
        me.set_state(m_host.numpy(), 0.0, me.get_state()[2])
        ke = max(2, min(K, args.e2e_steps))
        dt_e = me.get_state()[2]
        # one untimed pass of the loop: the step graph is captured again after the per-launch profile
        me.set_state_host_ptr(m_host, 0.0, dt_e)
        me.run_steps(1, nmgb.DP54, 1e-5, 1e-5)
        me.mean_m()
        torch.cuda.synchronize()
        barrier()
        t_e = time.perf_counter()
        acc_e = 0
        mean_hist = []
        for _ in range(ke):
            me.set_state_host_ptr(m_host, 0.0, dt_e)
            me.run_steps(1, nmgb.DP54, 1e-5, 1e-5)
            mean_hist.append(me.mean_m())
            acc_e += me.counters()[0]
        torch.cuda.synchronize()
        el_e = max_over_ranks(time.perf_counter() - t_e)
        e2e_value = nn * sum_over_ranks(acc_e) / el_e
    me.close()
    del me
    # ---- plain FP64 path on the same workload (fewer steps: it is several times slower)
    value64, ms64, k64, prof64 = None, None, 0, None
    if args.fp64_steps > 0:
        k64 = max(2, min(K, args.fp64_steps))
        me = make(nmgb.F64)
        me.run_steps(min(W, 3), nmgb.DP54, 1e-5, 1e-5)
        me.sync()
        ms64, acc64, _ = timed_steps(me, k64)
        ms64 = max_over_ranks(ms64)
        value64 = nn * sum_over_ranks(acc64) / (ms64 * 1e-3)
        # one step launch by launch inside an NVTX range (the ncu capture of its FP64 operations selects it)
        torch.cuda.nvtx.range_push("fp64_profile_step")
        prof64 = me.profile_step(nmgb.DP54, reps=1)
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_pop()
        me.close()
        del me

    if rank != 0:
        return
    # roofline of the dominant kernel (largest share of the step time)
    b = 4
    groups = {}
    stage = 1
    rows = []
    for name, t in prof:
        if name == "node_llg_stage":
            stage += 1
        byts = algorithmic_bytes(name, stage, n, b, False)
        rows.append((name, stage, t, byts))
        g = groups.setdefault(name, [0.0, 0, 0.0])
        g[0] += t
        g[1] += 1
        g[2] += byts
    step_ms = sum(r[2] for r in rows)
    dom = max(groups.items(), key=lambda kv: kv[1][0])
    dname, (dms, dcount, dbytes) = dom
    peak, peak_src = measured_peaks()
    achieved = (dbytes / dcount) / (dms / dcount * 1e-3) / 1e9
    wl_key = f"{n[0]}x{n[1]}x{n[2]}"
    traffic = traffic_for(dname, wl_key)
    step_bytes = sum(r[3] for r in rows)
    kernels = {k: {"launches_per_step": v[1], "ms_per_launch": v[0] / v[1], "share": v[0] / step_ms,
                   "GBps": (v[2] / v[1]) / (v[0] / v[1] * 1e-3) / 1e9,
                   "frac_of_peak": (v[2] / v[1]) / (v[0] / v[1] * 1e-3) / 1e9 / peak}
               for k, v in groups.items()}
    launches_per_step = len(prof) + 1  # dp5_error_control is two kernels
    serving = None
    if args.serve_requests > 0:
        serving = run_serving(args.serve_requests, int(args.serve_budget_gb * (1 << 30)), args.serve_max_active)
    film = wire = None
    if args.film_steps > 0 and rank == 0:
        try:
            film = run_film(nmgb, args.film_steps)
        except Exception as e:  # a side measurement: report it, keep the headline line
            film = {"error": f"{type(e).__name__}: {e}"}
        try:
            wire = run_wire(nmgb, args.film_steps)
        except Exception as e:
            wire = {"error": f"{type(e).__name__}: {e}"}
    workloads = None
    if args.workloads and rank == 0:
        try:
            workloads = run_workloads(nmgb)
        except Exception as e:  # a side measurement: report it, keep the headline line
            workloads = {"error": f"{type(e).__name__}: {e}"}
    cufft = None
    if args.cufft_reps > 0 and rank == 0:
        dem = [k for k in groups if k.startswith("demag_")]
        own_ms = sum(groups[k][0] for k in dem) / 6  # six field evaluations per step
        own_b = sum(groups[k][2] for k in dem) / 6
        try:
            cufft = run_cufft_baseline(n, args.cufft_reps, own_ms, own_b)
        except Exception as e:  # a side measurement: report it, keep the headline line
            cufft = {"error": f"{type(e).__name__}: {e}"}
    gradients = None
    if args.grad_steps > 0 and rank == 0:
        try:
            gradients = run_gradients(nmgb, args.grad_steps)
        except Exception as e:  # a side measurement: report it, keep the headline line
            gradients = {"error": f"{type(e).__name__}: {e}"}
    cpu_v, cpu_v1, cores, cs_desc = None, None, None, "skipped (--cpu-seconds 0)"
    if args.cpu_seconds > 0:
        cpu_v, cores, cs_steps, cs_el, cs_desc = oracle_sample(seconds=args.cpu_seconds)
        cpu_v1 = oracle_sample(seconds=max(2.0, args.cpu_seconds / 4), threads=1)[0]
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K, "warmup": W,
        "ms_per_step": ms_max / K, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32", "data": "synthetic",
        "config": {"workload": f"cuboid {wl_key} cells of 3 nm, Ms=1e6 A/m, A=1.5e-11 J/m, Ku=5e5 J/m^3 along z, "
                               f"exchange+anisotropy+FFT demag, random unit m0, DP5(4) rtol=atol=1e-5",
                   "nodes": nn, "cells": int(np.prod(n)), "precision": "FP32 field evaluation, FP64 state, "
                   "error norm and step control", "l2": "working set larger than L2 (no flush needed)",
                   "accepted_steps": int(acc_tot), "rejected_steps": int(sum_over_ranks(rej)),
                   "parallelism": f"replicas x{world}"},
        "h_eff": {"evals_per_s": evals_tot / (ms_max * 1e-3), "ns_per_node_per_eval": ms_max * 1e6 / (evals * nn),
                  "evals": evals_tot,
                  "note": "the paper's timing metric: integration time / number of field evaluations (six per "
                          "DP5(4) step with FSAL, accepted or rejected), here per node"},
        "fp64": fp64_line(nmgb, value64, ms64, k64, value, prof64, nn, wl_key),
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": int(24 * nn),
                "d2h_bytes_per_step": 32 + 128, "steps": ke,
                "note": "per step through the public API: nm_set_state from pinned host m (the step's input), "
                        "one DP5 step (with the FSAL slope of the new state), and the step's result read "
                        "back: the volume-weighted mean of m (nm_mean_m) and the step counters"},
        "roofline": {"bound": "hbm", "kernel": dname, "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": traffic, "peak_source": peak_src,
                     "algorithmic_bytes_per_launch": dbytes / dcount,
                     "step_achieved": step_bytes / (step_ms * 1e-3) / 1e9,
                     "step_frac": step_bytes / (step_ms * 1e-3) / 1e9 / peak},
        "kernels": kernels,
        "cpu_baseline": {"value": cpu_v, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": cs_desc,
                         "value_1_core": cpu_v1},
        "serving": serving,
        "gradients": gradients,
        "cufft_baseline": cufft,
        "workloads": workloads,
        "thin_film_2d_basis": film,
        "wire_1d_basis": wire,
        "clocks": clocks,
        "gpu_launches": int(launches_per_step * K),
    }
    print(json.dumps(line), flush=True)


def run_cufft_baseline(n, reps, own_demag_ms, own_demag_bytes):
    """Timed baseline only, never on the library's path: the conventional demag convolution with cuFFT
    (through torch.fft) on the zero-padded P1 x P2 x P3 grid in FP32, as a library FFT pipeline does it:
    copy the cell field into the zeroed padded grid, 3D real-to-complex transforms of the three
    components, the product with the six-component tensor on the full half spectrum (torch elementwise
    operations), 3D complex-to-real transforms, and the crop back to the cells.  Reported per field
    evaluation beside the library's own demag passes of the same mesh."""
    import torch

    def pad(v):
        if v == 1:
            return 1
        p = 1
        while p < 2 * v - 1:
            p *= 2
        return p
    N1, N2, N3 = n
    P1, P2, P3 = pad(N1), pad(N2), pad(N3)
    dev = "cuda"
    g = torch.Generator(device=dev).manual_seed(0)
    cells = torch.randn((3, N3, N2, N1), device=dev, dtype=torch.float32, generator=g)
    Nt = torch.randn((6, P3, P2, P1 // 2 + 1), device=dev, dtype=torch.float32, generator=g)
    Mp = torch.zeros((3, P3, P2, P1), device=dev, dtype=torch.float32)
    out = torch.empty_like(cells)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(6)]
    acc = np.zeros(5)

    def once(timed):
        if timed:
            ev[0].record()
        Mp.zero_()
        Mp[:, :N3, :N2, :N1] = cells
        if timed:
            ev[1].record()
        S = torch.fft.rfftn(Mp, dim=(1, 2, 3))
        if timed:
            ev[2].record()
        Hx = Nt[0] * S[0] + Nt[3] * S[1] + Nt[4] * S[2]
        Hy = Nt[3] * S[0] + Nt[1] * S[1] + Nt[5] * S[2]
        Hz = Nt[4] * S[0] + Nt[5] * S[1] + Nt[2] * S[2]
        H = torch.stack((Hx, Hy, Hz))
        del Hx, Hy, Hz, S
        if timed:
            ev[3].record()
        h = torch.fft.irfftn(H, s=(P3, P2, P1), dim=(1, 2, 3))
        if timed:
            ev[4].record()
        out.copy_(h[:, :N3, :N2, :N1])
        if timed:
            ev[5].record()
        del H, h

    for _ in range(2):
        once(False)
    torch.cuda.synchronize()
    for _ in range(reps):
        once(True)
        torch.cuda.synchronize()
        acc += np.array([ev[i].elapsed_time(ev[i + 1]) for i in range(5)])
    acc /= reps
    res = {"workload": f"padded grid {P1}x{P2}x{P3} (cells {N1}x{N2}x{N3}), 3 components, FP32, cuFFT through "
                       f"torch.fft {torch.version.cuda}",
           "unit": "ms per field evaluation",
           "pad_ms": acc[0], "r2c_ms": acc[1], "tensor_product_ms": acc[2], "c2r_ms": acc[3], "crop_ms": acc[4],
           "cufft_transforms_ms": acc[1] + acc[3], "total_ms": float(acc.sum()),
           "own_demag_ms": own_demag_ms, "own_demag_algorithmic_GB": own_demag_bytes / 1e9,
           "own_over_cufft_transforms": own_demag_ms / (acc[1] + acc[3]),
           "own_over_cufft_total": own_demag_ms / float(acc.sum())}
    del cells, Nt, Mp, out
    torch.cuda.empty_cache()
    return res


def run_film(nmgb, n_steps, grid=(1024, 1024, 1)):
    """A single-layer film (3 nm cells of the throughput material, 1 nm thick), FP32 DP5(4) steps with
    the trilinear basis (2 node layers) and with the 2D basis (1 node layer, section "Low-Dimensional
    Geometries"): wall time per step (graph replays, synchronised) and node-steps/s of each."""
    p = inp.throughput(grid, seed=5, with_m0=False)
    out = run_bases(nmgb, n_steps, p, (p.dx[0], p.dx[1], 1e-9), (3, 2), 5,
                    f"film {grid[0]}x{grid[1]}x{grid[2]} cells of 3x3x1 nm")
    out["step_time_ratio_3d_over_2d"] = out["basis3"]["ms_per_step"] / out["basis2"]["ms_per_step"]
    return out


def run_wire(nmgb, n_steps, grid=(1024, 4, 4)):
    """A wire of 4 x 4 cells across (3 nm cells of the throughput material), FP32 DP5(4) steps with the
    trilinear basis (5 x 5 nodes across) and with the 1D basis (one node per position along the wire,
    section "Low-Dimensional Geometries"): wall time per step and node-steps/s of each."""
    p = inp.throughput(grid, seed=6, with_m0=False)
    out = run_bases(nmgb, n_steps, p, p.dx, (3, 1), 6, f"wire {grid[0]}x{grid[1]}x{grid[2]} cells of 3 nm")
    out["step_time_ratio_3d_over_1d"] = out["basis3"]["ms_per_step"] / out["basis1"]["ms_per_step"]
    return out


def run_bases(nmgb, n_steps, p, dx, bases, seed, what):
    """FP32 DP5(4) steps of the problem p on cells dx with each nodal basis in `bases`."""
    rng = np.random.default_rng(seed)
    out = {"workload": f"{what}, throughput material, FP32 field, DP5(4) rtol=atol=1e-5, random unit m0, "
                       f"{n_steps} timed steps"}
    for basis in bases:
        me = nmgb.Mesh(p.n, dx, nmgb.F32, basis=basis)
        me.set_material(p.Ms, p.A, p.Ku, p.axis, p.alpha, p.gamma)
        me.set_terms(p.terms)
        m0 = inp.unit_vectors(rng, me.nodes)
        me.set_state(m0, 0.0, 1e-15)
        me.run_steps(3, nmgb.DP54, 1e-5, 1e-5)  # warm-up
        me.sync()
        a0, r0, _ = me.counters()
        t0 = time.perf_counter()
        me.run_steps(n_steps, nmgb.DP54, 1e-5, 1e-5)
        me.sync()
        ms = (time.perf_counter() - t0) * 1e3
        a1, r1, _ = me.counters()
        nn = int(np.prod(me.nodes))
        out[f"basis{basis}"] = {"nodes": nn, "ms_per_step": ms / max(1, (a1 - a0) + (r1 - r0)),
                                "node_steps_per_s": nn * (a1 - a0) / (ms * 1e-3)}
        me.close()
    return out


def run_gradients(nmgb, n_steps, grid=(256, 256, 8), dt=1e-14):
    """Wall time of the two gradient methods against the forward integration they differentiate (FP32
    field, the throughput material): n RK4 steps forward; the discrete adjoint (nm_adjoint_run,
    checkpointed, exact gradient of the discrete map); the continuous adjoint (nm_adjoint_continuous,
    backward integration of Eq. adjoint_system).  Also the relative L2 gap between their Ms gradients."""
    p = inp.throughput(grid, seed=7, with_m0=False)
    rng = np.random.default_rng(7)
    m0 = inp.unit_vectors(rng, p.nodes)
    Wt = rng.uniform(0.5, 1.5, p.nodes + (3,))
    tgt = inp.unit_vectors(rng, p.nodes)
    T = n_steps * dt

    def mesh():
        me = nmgb.Mesh(p.n, p.dx, nmgb.F32)
        me.set_material(p.Ms, p.A, p.Ku, p.axis, p.alpha, p.gamma)
        me.set_terms(p.terms)
        me.set_state(m0, 0.0, dt)
        return me

    out = {"workload": f"cuboid {grid[0]}x{grid[1]}x{grid[2]} cells, throughput material, FP32 field, "
                       f"{n_steps} RK4 steps of {dt:g} s, final-time quadratic loss", "unit": "ms"}
    me = mesh()
    me.run_steps(n_steps, nmgb.RK4, 0.0, 0.0)  # warm-up (graphs, workspaces)
    me.set_state(m0, 0.0, dt)
    me.sync()
    t0 = time.perf_counter()
    me.run_steps(n_steps, nmgb.RK4, 0.0, 0.0)
    me.sync()
    out["forward_ms"] = (time.perf_counter() - t0) * 1e3
    me.set_state(m0, 0.0, dt)
    me.adjoint_run(T, Wt, tgt, method=nmgb.RK4, dt0=dt)  # warm-up
    me.set_state(m0, 0.0, dt)
    t0 = time.perf_counter()
    _, gd, _, _ = me.adjoint_run(T, Wt, tgt, method=nmgb.RK4, dt0=dt)
    out["discrete_adjoint_ms"] = (time.perf_counter() - t0) * 1e3
    me.set_state(m0, 0.0, dt)
    me.adjoint_continuous(T, n_steps, Wt, tgt)  # warm-up
    me.set_state(m0, 0.0, dt)
    t0 = time.perf_counter()
    _, _, gc, _, m0r = me.adjoint_continuous(T, n_steps, Wt, tgt)
    out["continuous_adjoint_ms"] = (time.perf_counter() - t0) * 1e3
    me.close()
    out["ms_gradient_rel_l2_gap"] = float(np.linalg.norm(gc - gd) / np.linalg.norm(gd))
    out["m0_reconstruction_max_err"] = float(np.abs(m0r - m0).max())
    return out


def run_workloads(nmgb, sweep_steps=10):
    """Absolute node-steps/s of the other workloads (wall time, synchronised, FP32 field with FP64 state
    and plain FP64): the 16x16x4 cuboid over its 1000 RK4 steps, the 200x50x1 film by Dormand-Prince to
    1 ns (with the FP32-FP64 gap of the time-averaged mean m), the 256x256x8 and 512x512x16 throughput
    cuboids over `sweep_steps` DP5 steps, and the 256x64x1 waveguide over 2 ns with its Ms gradient
    (loss on the right 16 cells, RK4 steps of 0.25 ps, checkpoints every ceil(sqrt(n)) steps)."""
    import math
    out = {}

    def timed(fn):
        t0 = time.perf_counter()
        r = fn()
        return r, time.perf_counter() - t0

    # cuboid 16x16x4, 1000 RK4 steps of 1e-14 s
    p = inp.cuboid_rk4(0)
    nn = int(np.prod(p.nodes))
    res = {"workload": "cuboid 16x16x4 cells of 2 nm, exchange + demag + Zeeman, 1000 RK4 steps of 1e-14 s"}
    for prec, name in ((nmgb.F32, "fp32"), (nmgb.F64, "fp64")):
        me = nmgb.Mesh(p.n, p.dx, prec)
        me.set_material(p.Ms, p.A, p.Ku, p.axis, p.alpha, p.gamma)
        me.set_zeeman(p.h_uniform)
        me.set_terms(p.terms)
        me.set_state(p.m0, 0.0, 1e-14)
        me.run_until(2e-13, nmgb.RK4, dt0=1e-14)  # warm-up (graphs)
        me.set_state(p.m0, 0.0, 1e-14)
        (_, na, _), el = timed(lambda: me.run_until(1e-11, nmgb.RK4, dt0=1e-14))
        res[name] = {"node_steps_per_s": nn * na / el, "ms_per_step": el / na * 1e3, "steps": na}
        me.close()
    out["cuboid_16x16x4_rk4"] = res
    # thin film 200x50x1 to 1 ns
    p = inp.thin_film(0)
    x = p.extra
    nn = int(np.prod(p.nodes))
    res = {"workload": "film 200x50x1 cells of 2.5x2.5x3 nm, exchange + demag + Zeeman, DP5(4) to 1 ns, "
                       "rtol=atol=1e-5, 1 ps samples of the mean m"}
    avg = {}
    for prec, name in ((nmgb.F32, "fp32"), (nmgb.F64, "fp64")):
        me = nmgb.Mesh(p.n, p.dx, prec)
        me.set_material(p.Ms, p.A, p.Ku, p.axis, p.alpha, p.gamma)
        me.set_zeeman(p.h_uniform)
        me.set_terms(p.terms)
        me.set_state(p.m0, 0.0, x["dt0"])
        me.run_until(2e-12, nmgb.DP54, x["rtol"], x["atol"], dt0=x["dt0"])  # warm-up
        me.set_state(p.m0, 0.0, x["dt0"])
        (smp, na, nr), el = timed(lambda: me.run_until(x["t_end"], nmgb.DP54, x["rtol"], x["atol"], dt0=x["dt0"],
                                                       sample_dt=x["sample_dt"]))
        res[name] = {"node_steps_per_s": nn * na / el, "ms_per_step": el / (na + nr) * 1e3, "accepted": na,
                     "rejected": nr}
        avg[name] = (0.5 * (smp[0] + smp[-1]) + smp[1:-1].sum(axis=0)) / (len(smp) - 1)
        me.close()
    res["time_averaged_mean_m_gap_fp32_fp64"] = float(np.abs(avg["fp32"] - avg["fp64"]).max())
    out["thin_film_200x50x1_dp5_1ns"] = res
    # throughput sweep points
    for grid in ((256, 256, 8), (512, 512, 16)):
        p = inp.throughput(grid, seed=3, with_m0=False)
        m0 = inp.unit_vectors(np.random.default_rng(3), p.nodes)
        nn = int(np.prod(p.nodes))
        res = {"workload": f"cuboid {grid[0]}x{grid[1]}x{grid[2]} cells of 3 nm, throughput material, DP5(4) "
                           f"rtol=atol=1e-5, {sweep_steps} steps"}
        for prec, name in ((nmgb.F32, "fp32"), (nmgb.F64, "fp64")):
            me = nmgb.Mesh(p.n, p.dx, prec)
            me.set_material(p.Ms, p.A, p.Ku, p.axis, p.alpha, p.gamma)
            me.set_terms(p.terms)
            me.set_state(m0, 0.0, 1e-15)
            me.run_steps(3, nmgb.DP54, 1e-5, 1e-5)
            me.sync()
            a0, r0, _ = me.counters()
            _, el = timed(lambda: (me.run_steps(sweep_steps, nmgb.DP54, 1e-5, 1e-5), me.sync()))
            a1, r1, _ = me.counters()
            res[name] = {"node_steps_per_s": nn * (a1 - a0) / el, "ms_per_step": el / ((a1 - a0) + (r1 - r0)) * 1e3}
            me.close()
        res["fp32_over_fp64"] = res["fp32"]["node_steps_per_s"] / res["fp64"]["node_steps_per_s"]
        out[f"cuboid_{grid[0]}x{grid[1]}x{grid[2]}"] = res
    # waveguide inverse problem over 2 ns
    p = inp.waveguide(0)
    T, sdt, dt = p.extra["t_end"], p.extra["sample_dt"], 2.5e-13
    n_steps = int(round(T / dt))
    C = math.ceil(math.sqrt(n_steps))
    nn = int(np.prod(p.nodes))
    W = np.zeros(p.nodes + (3,))
    W[p.n[0] - 16:, :, :, 1] = 1.0
    W /= W[..., 1].sum() * int(round(T / sdt))
    res = {"workload": f"waveguide 256x64x1 cells of 4x4x10 nm, Ms map, 2 GHz drive, loss = mean m_y^2 over the "
                       f"right 16 cells and 1 ps samples in [0, 2 ns], {n_steps} RK4 steps of 0.25 ps, "
                       f"checkpoints every {C} steps, FP32 field"}
    me = nmgb.Mesh(p.n, p.dx, nmgb.F32)
    me.set_material(p.Ms_cells(), p.A, 0.0, p.axis, p.alpha, p.gamma)
    me.set_zeeman((0, 0, 0), h_cell=p.h_cell, cell_freq=p.cell_freq, cell_phase=p.cell_phase)
    me.set_terms(p.terms)
    me.set_state(p.m0, 0.0, dt)
    me.adjoint_run(2e-11, W, None, nmgb.RK4, dt0=dt, sample_dt=sdt, checkpoint_every=C)  # warm-up
    me.set_state(p.m0, 0.0, dt)
    (fwd, el_f) = timed(lambda: me.adjoint_run(T, W, None, nmgb.RK4, dt0=dt, sample_dt=sdt, checkpoint_every=C,
                                               loss_only=True))
    me.set_state(p.m0, 0.0, dt)
    (grad, el_g) = timed(lambda: me.adjoint_run(T, W, None, nmgb.RK4, dt0=dt, sample_dt=sdt, checkpoint_every=C))
    me.close()
    res.update({"forward_s": el_f, "forward_node_steps_per_s": nn * fwd[3] / el_f, "gradient_s": el_g,
                "gradient_over_forward": el_g / el_f, "steps": fwd[3], "loss": fwd[0]})
    out["waveguide_256x64x1_gradient_2ns"] = res
    return out


def serving_kwargs(i, p):
    return dict(n=p.n, dx=p.dx, m0=inp.serving_m0(p), t_end=p.extra["t_end"], Ms=p.Ms, A=p.A, Ku=p.Ku,
                axis=p.axis, alpha=p.alpha, gamma=p.gamma, h=p.h_uniform, terms=p.terms, rtol=p.extra["rtol"],
                atol=p.extra["atol"], dt0=p.extra["dt0"], tag=i)


def run_serving(n_requests, budget_bytes, max_active, loads=(0.7, 1.2, 8.0), n_capacity=8):
    """Poisson streams of mixed-size LLG runs through the library's request loop.  Capacity = 1 / mean
    service time of runs executed one at a time; each load level replays the same requests with arrival
    rate = load x capacity.  Latency = submit -> result on the host.  The 8x level keeps the queue full:
    its throughput is the ceiling of the request loop with up to max_active runs on the GPU at once."""
    from paper_2411_11725_gb300.serve import Server, replay
    reqs = inp.serving_requests(max(n_requests, n_capacity), seed=0, rate_hz=1.0)
    stream = [(t, serving_kwargs(i, p)) for i, (t, p) in enumerate(reqs[:n_requests])]
    nodes = {i: int(np.prod(p.nodes)) for i, (_, p) in enumerate(reqs)}
    out = {"requests": n_requests, "hbm_budget_bytes": int(budget_bytes), "max_active": max_active,
           "distribution": "grids N1,N2 in {64,128,256} x N3 in {1,2,4,8} cells of 3 nm, Ms~U[4e5,1.2e6], "
                           "A~U[5e-12,2e-11], alpha~U[0.01,0.5], |mu0 h|~U[0,100] mT, T~U[0.2,2] ns, "
                           "DP5(4) rtol=atol=1e-5, FP32 field, seed 0"}
    with Server(budget_bytes, max_active=max_active) as s:
        # warm the mesh pool: one short run per shape (tensor spectra resident, as in steady state)
        shapes = {}
        for i, (_, kw) in enumerate(stream):
            shapes.setdefault(tuple(kw["n"]), i)
        for i in shapes.values():
            s.submit(**dict(stream[i][1], t_end=1e-13, tag=10**6 + i))
        s.drain(len(shapes))
        # capacity: runs one at a time
        service = []
        for i in range(n_capacity):
            s.submit(**serving_kwargs(i, reqs[i][1]))
            (r,) = s.drain(1)
            service.append(r["run_s"])
        cap = 1.0 / float(np.mean(service))
        out["capacity_req_s"] = cap
        out["capacity_sample"] = f"{n_capacity} requests run one at a time, mean service {np.mean(service):.3f} s"
        levels = []
        for load in loads:
            rate = load * cap
            st0 = s.stats()
            t0 = time.perf_counter()
            res = replay(s, stream, time_scale=1.0 / rate, timeout_s=900)
            wall = time.perf_counter() - t0
            st1 = s.stats()
            ok = [r for r in res if r["status"] == 0]
            lat = np.array([r["latency_s"] for r in ok])
            ns = sum(nodes[r["tag"]] * r["n_accepted"] for r in ok)
            levels.append({
                "load": load, "rate_req_s": rate, "completed": len(ok), "failed": len(res) - len(ok),
                "p50_s": float(np.percentile(lat, 50)), "p99_s": float(np.percentile(lat, 99)),
                "mean_s": float(lat.mean()), "max_s": float(lat.max()),
                "mean_queue_s": float(np.mean([r["queue_s"] for r in ok])),
                "throughput_req_s": len(ok) / wall, "node_steps_s": ns / wall, "wall_s": wall,
                "busy_frac": (st1["busy_s"] - st0["busy_s"]) / wall,
                "mean_active": (st1["active_s"] - st0["active_s"]) / wall,
                "peak_active": st1["peak_active"], "peak_bytes": st1["peak_bytes"],
                "meshes_created": st1["meshes_created"], "meshes_evicted": st1["meshes_evicted"]})
        out["levels"] = levels
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--grid", default="1024x1024x32")
    ap.add_argument("--e2e-steps", type=int, default=5)
    ap.add_argument("--fp64-steps", type=int, default=4)
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--serve-requests", type=int, default=500, help="requests per serving load level (0: skip)")
    ap.add_argument("--serve-budget-gb", type=float, default=2.0)
    ap.add_argument("--serve-max-active", type=int, default=16)
    ap.add_argument("--grad-steps", type=int, default=16, help="RK4 steps of the gradient timing leg (0: skip)")
    ap.add_argument("--film-steps", type=int, default=10, help="DP5 steps of the 2D-basis film and 1D-basis wire legs (0: skip)")
    ap.add_argument("--workloads", type=int, default=1, help="absolute rates of the other workloads (0: skip)")
    ap.add_argument("--cufft-reps", type=int, default=3,
                    help="timed repetitions of the cuFFT zero-padded convolution baseline (0: skip)")
    args = ap.parse_args()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    dist = None
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    if world > 1:
        import torch
        import torch.distributed as tdist
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
        tdist.init_process_group("nccl")
        dist = tdist
    try:
        run_ours(args, rank, world, dist)
    finally:
        if dist is not None:
            dist.destroy_process_group()


if __name__ == "__main__":
    main()
