#!/usr/bin/env python3
"""Benchmark: pairwise interactions/s of the block-step Hermite hot path on B300.

One step = one full block cycle of the 6th-order scheme on the galactic-nucleus
workload (2^20 Plummer stars + two unsoftened 0.005 black holes, star softening
1e-5): block scheduler, predictor of all N, force of every particle on every
particle (the synchronised block of a hierarchical block-step run), corrector
and new steps.  Mixed precision (double-single positions, FP32 pair chain,
compensated sums) unless --precision fp64.

Printed JSON line (rank 0): value = interactions/s over the timed steps with
the state resident in HBM; e2e = the same through the C ABI with host state
copied in and out every step; roofline of the force kernel (CUDA events on its
stream); the FP64 path on a 4096-particle block of the same system; the force
rate of both paths on each single-system workload and on the nucleus at 4th
order; energy error and
whole-run throughput of both paths on the 65536-particle Plummer sphere
(host-driven, CUDA-graph and autotuned cycles); energy and binary-element
drift of both paths on the 8th-order cusp nucleus; the 256-cluster ensemble;
the CPU oracle on the host cores as a baseline (cpu_baseline: its rate on a
sample of the nucleus, and on that sample the parity of the GPU force against
it; the 1024-particle Plummer run end to end against the FP64 path's blocks).
The oracle runs in that leg only (and in the reference arm).

  python bench.py [--steps K] [--warmup W] [--gpus N] [--impl ours|reference]
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

METRIC = "pairwise interactions/s & % CUDA-core peak at N=2^20, mixed vs FP64 at stated dE/E"
FLOPS_PER_INTERACTION = {4: 60, 6: 97, 8: 144}   # direct N-body flop convention
SM_COUNT, FP32_LANES, SM_MAX_MHZ = 148, 128, 2032.0
FP32_PEAK_TFLOPS = SM_COUNT * FP32_LANES * 2 * SM_MAX_MHZ * 1e6 / 1e12   # 76.96, FMA = 2 flops
FP64_PEAK_TFLOPS = 1.25                                                     # nominal dense FP64
# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) of one mixed force
# launch over the whole nucleus system (N_act = N = 2^20 + 2, 13 j-splits), from
# a one-pass ncu capture of that launch (the command is the profiling case
# `bench.py --profile-force --n-act 1048578 --repeat 1`).
FORCE_TRAFFIC_BYTES = {("nucleus_plummer_n1048576_2bh", "mixed"): 911.70e6 + 1163.57e6}


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=5)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", choices=["ours", "reference"], default="ours")
    p.add_argument("--precision", choices=["mixed", "fp64"], default="mixed")
    p.add_argument("--block-step", type=float, default=2.0 ** -12)
    p.add_argument("--quick", action="store_true", help="skip the FP64, energy, ensemble and CPU legs")
    p.add_argument("--ensemble-t", type=float, default=1.0 / 64, help="end time of the ensemble leg")
    p.add_argument("--energy-t", type=float, default=1.0, help="end time of the energy-budget legs")
    p.add_argument("--energy-n", type=int, default=16384,
                   help="Plummer sphere of the both-paths energy-budget leg (FP64 to --energy-t)")
    p.add_argument("--cusp-fp64", action="store_true",
                   help="also run the full-size cusp on the FP64 path (about two minutes)")
    p.add_argument("--nucleus-full", action="store_true",
                   help="also run the 2^20 nucleus to t = 1/16 on the mixed path (about two minutes)")
    p.add_argument("--nucleus-fp64", type=float, default=0.0, metavar="T",
                   help="also run the 2^20 nucleus to t = T with dt_max = T on both paths (T = 2^-10: about "
                        "ten minutes, most of it the FP64 start-up and energies)")
    p.add_argument("--nucleus-trend", action="store_true",
                   help="also run the nucleus recipe with 2^14 and 2^17 stars to t = 1/16 on both paths (about "
                        "two minutes)")
    p.add_argument("--profile-force", action="store_true",
                   help="instead of the benchmark: a small force case for profilers (see profile_force)")
    p.add_argument("--profile-step", action="store_true",
                   help="instead of the benchmark: block steps of one small active set (see profile_step)")
    p.add_argument("--n-act", type=int, default=4096, help="active particles of the profiling cases")
    p.add_argument("--repeat", type=int, default=2, help="force launches / block steps of the profiling cases")
    p.add_argument("--workload", choices=["nucleus", "cusp", "plummer65k"], default="nucleus",
                   help="system of the profiling cases")
    return p.parse_args()


# --------------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi samples every 200 ms while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index=0):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for nm, val in zip(names, f[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "samples": len(sm), "reasons": sorted(reasons)}


# ---------------------------------------------------------------- ranks
def aggregate(ms_local: float, steps: int, inter_per_step: float, dist=None, device="cpu"):
    """Whole-job throughput over ranks that each ran `steps` steps of their own
    replica: elapsed = the slowest rank's (MAX over ranks), value = every
    rank's interactions / that elapsed time.  Returns (ms_max, value, world)."""
    world = 1
    ms = float(ms_local)
    if dist is not None and dist.is_initialized():
        import torch
        world = dist.get_world_size()
        t = torch.tensor([ms], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    return ms, world * steps * inter_per_step / (ms * 1e-3), world


# ------------------------------------------------------------------- helpers
def nucleus():
    from paper_1312_1789_b300 import ics
    return ics.standard_workload(2)


def make_ctx(nb, wl, precision, stream):
    ctx = nb.NBody(wl.n, wl.order, 0.0, precision)
    ctx.set_stream(stream)
    ctx.set_softening(np.sqrt(wl.eps2))
    ctx.set_params(wl.eta, wl.eta_s, wl.dt_max, 2.0 ** -40)
    ctx.set_particles(wl.m, wl.x, wl.v)
    return ctx


def oracle_rate(wl, n_target_s=12.0, nthreads=None):
    """Oracle direct-sum interactions/s on the host cores for a sample of
    active particles against all N (about n_target_s seconds of work)."""
    import oracle as orc
    nthreads = nthreads or os.cpu_count() or 1
    rng = np.random.default_rng(0)
    n_cal = max(nthreads, 16)
    idx = rng.choice(wl.n, n_cal, replace=False).astype(np.int32)
    t0 = time.perf_counter()
    orc.force(wl.m, wl.eps2, wl.x, wl.v, np.zeros_like(wl.x), None, order=wl.order, idx=idx, nthreads=nthreads)
    dt_cal = time.perf_counter() - t0
    n_s = int(min(wl.n, max(n_cal, n_cal * n_target_s / max(dt_cal, 1e-3))))
    n_s = max(nthreads, (n_s // nthreads) * nthreads)
    return n_s, nthreads


def run_reference(args):
    """The CPU oracle timed on the host cores on a bounded sample per step."""
    import oracle as orc
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    wl = nucleus()
    n_s, nth = oracle_rate(wl, n_target_s=max(2.0, 60.0 / max(1, args.steps + args.warmup)))
    rng = np.random.default_rng(1)
    times = []
    for k in range(args.warmup + args.steps):
        idx = np.sort(rng.choice(wl.n, n_s, replace=False)).astype(np.int32)
        t0 = time.perf_counter()
        orc.force(wl.m, wl.eps2, wl.x, wl.v, np.zeros_like(wl.x), None, order=wl.order, idx=idx, nthreads=nth)
        if k >= args.warmup:
            times.append(time.perf_counter() - t0)
    inter = n_s * wl.n
    val = inter * len(times) / sum(times)
    sample = f"force of {n_s} sampled particles on all {wl.n} (long-double direct sum) per step"
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": val, "unit": "interactions/s", "n_gpus": 0,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sum(times) / len(times),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f80 (x87 long double)",
        "data": "synthetic", "config": {"workload": wl.name, "n": wl.n, "order": wl.order},
        "cpu_baseline": {"value": val, "unit": "interactions/s", "cores": nth, "kind": "oracle", "sample": sample},
        "e2e": {"value": val, "unit": "interactions/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


# ---------------------------------------------------------------- our arm
def run_ours(args):
    import torch

    from paper_1312_1789_b300 import build, ics, nb
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA device")
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    # one rank compiles (if the library is stale), the others wait and load it
    if rank == 0:
        build.build()
    if dist:
        dist.barrier()
    nb.lib()
    stream = torch.cuda.current_stream()
    prec = nb.NB_MIXED if args.precision == "mixed" else nb.NB_FP64
    wl = nucleus()
    n = wl.n
    h = args.block_step
    ctx = make_ctx(nb, wl, prec, stream)
    inter_step = n * n
    flop_pi = FLOPS_PER_INTERACTION[wl.order]

    def step():
        ctx.set_block_step(h)
        tb, na = ctx.block_step()
        assert na == n, (na, n)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    ctx.set_profiling(True)
    _, launches0 = ctx.get_profile()
    clocks = ClockSampler(local)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(args.steps):
        step()
    ev1.record(stream)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clk = clocks.stop()
    ms = ev0.elapsed_time(ev1)
    prof, launches1 = ctx.get_profile()
    ctx.set_profiling(False)
    ms, value, world = aggregate(ms, args.steps, inter_step, dist, device="cuda")
    force_ms, force_n = prof["force"]
    t_force = force_ms / max(force_n, 1) * 1e-3
    achieved = flop_pi * inter_step / t_force / 1e12
    out = {
        "metric": METRIC, "value": value, "unit": "interactions/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32 pair chain, double-single x, f64 state" if prec == nb.NB_MIXED else "f64",
        "data": "synthetic",
        "config": {"workload": wl.name, "n": n, "order": wl.order, "n_act": n,
                   "precision": args.precision, "block_step": h,
                   "l2": "state (~250 MB) and j-store (64 MB) stream every step; inputs exceed L2",
                   "parallelism": f"replicas x{world}" if world > 1 else "1 GPU"},
        "tflops_convention": value * flop_pi / world / 1e12 if world else None,
        "roofline": {"bound": "alu", "achieved": achieved, "peak": FP32_PEAK_TFLOPS, "unit": "TFLOP/s",
                     "frac": achieved / FP32_PEAK_TFLOPS,
                     "traffic": FORCE_TRAFFIC_BYTES.get((wl.name, args.precision)),
                     "traffic_unit": "DRAM bytes per force launch (ncu)",
                     "note": f"force kernel, {flop_pi} flops per interaction (direct N-body convention); peak "
                             "= 148 SMs x 128 FP32 lanes x 2 x 2032 MHz"},
        "phases_ms_per_step": {k: v[0] / args.steps for k, v in prof.items()},
        "gpu_launches": int(launches1 - launches0),
        "clocks": clk,
    }
    try:
        fp32 = ctx.fma_peak(False)
        fp64 = ctx.fma_peak(True)
        out["measured_fma_peak"] = {"fp32_tflops": fp32, "fp64_tflops": fp64,
                                    "force_frac_of_measured_fp32": achieved / fp32,
                                    "note": "independent FFMA / DFMA chains on every SM (nb_fma_peak), best of 3, "
                                            "at the clock of this run"}
    except Exception as e:  # pragma: no cover
        out["measured_fma_peak"] = {"error": repr(e)}
    if rank == 0 and not args.quick:
        extras(args, nb, ics, wl, ctx, stream, out, prec)
    ctx.close()
    if rank == 0:
        print(json.dumps(out))
    if dist:
        dist.destroy_process_group()


def momentum_drift(S0, S1, m):
    """|P1 - P0| / sum_i m_i |v_i| (at the start) of the total momentum."""
    p0 = (m[:, None] * S0["v"]).sum(axis=0)
    p1 = (m[:, None] * S1["v"]).sum(axis=0)
    return float(np.linalg.norm(p1 - p0) / (m * np.linalg.norm(S0["v"], axis=1)).sum())


def binary_elements(S, m):
    """Two-body semi-major axis and eccentricity of the last two particles."""
    r = S["x"][-2] - S["x"][-1]
    u = S["v"][-2] - S["v"][-1]
    mu = m[-2] + m[-1]
    en = 0.5 * float(u @ u) - mu / float(np.linalg.norm(r))
    h = np.cross(r, u)
    return -mu / (2.0 * en), math.sqrt(max(0.0, 1.0 + 2.0 * en * float(h @ h) / mu ** 2))


def cusp_run(nb, w, p, stream, torch, t_end, dt_max=None):
    c = nb.NBody(w.n, w.order, 0.0, p)
    c.set_stream(stream)
    c.set_softening(np.sqrt(w.eps2))
    c.set_params(w.eta, w.eta_s, dt_max or w.dt_max, 2.0 ** -40)
    c.set_particles(w.m, w.x, w.v)
    c.set_precision(nb.NB_FP64)
    e0 = sum(c.energy())
    S0 = c.get_state()
    a0, ec0 = binary_elements(S0, w.m)
    c.set_precision(p)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    nblk, ni = c.step_until(t_end)
    torch.cuda.synchronize()
    el = time.perf_counter() - t0
    c.set_precision(nb.NB_FP64)
    e1 = sum(c.energy())
    S1 = c.get_state()
    a1, ec1 = binary_elements(S1, w.m)
    c.close()
    return {"dE_E": (e1 - e0) / abs(e0), "dP_rel": momentum_drift(S0, S1, w.m), "binary_a": [a0, a1],
            "binary_e": [ec0, ec1], "blocks": nblk,
            "interactions": ni, "seconds": el, "whole_run_interactions_per_s": ni / el}


def nucleus_run(nb, w, p, stream, torch, t_end, graph=0, dt_max=None):
    c = nb.NBody(w.n, w.order, 0.0, p)
    c.set_stream(stream)
    c.set_softening(np.sqrt(w.eps2))
    c.set_params(w.eta, w.eta_s, dt_max or w.dt_max, 2.0 ** -40)
    c.set_particles(w.m, w.x, w.v)
    c.set_precision(nb.NB_FP64)
    e0 = sum(c.energy())
    S0 = c.get_state()
    c.set_precision(p)
    c.set_graph(graph)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    nblk, ni = c.step_until(t_end)
    torch.cuda.synchronize()
    el = time.perf_counter() - t0
    c.set_precision(nb.NB_FP64)
    e1 = sum(c.energy())
    dp = momentum_drift(S0, c.get_state(), w.m)
    c.close()
    return {"dE_E": (e1 - e0) / abs(e0), "dP_rel": dp, "blocks": nblk, "interactions": ni, "seconds": el,
            "whole_run_interactions_per_s": ni / el}


def cusp_leg(args, nb, ics, stream, torch):
    """Dehnen gamma=1 cusp with a central black-hole binary, 8th order.  The
    two-body elements are not conserved (the stellar mass inside the orbit
    exceeds the binary's); the comparison of interest is mixed vs FP64."""
    res = {}
    small = ics.cusp_nucleus(1 << 14, 1003, 1e-4, 1.0 / 16, 8)
    res["reduced"] = {"workload": small.name + " to t=1/16",
                      "mixed": cusp_run(nb, small, nb.NB_MIXED, stream, torch, 1.0 / 16),
                      "fp64": cusp_run(nb, small, nb.NB_FP64, stream, torch, 1.0 / 16)}
    r = res["reduced"]
    r["mixed_dE_within_2x_of_fp64"] = abs(r["mixed"]["dE_E"]) <= 2 * abs(r["fp64"]["dE_E"])
    full = ics.standard_workload(3)
    res["full"] = {"workload": full.name + " to t=1/16", "mixed": cusp_run(nb, full, nb.NB_MIXED, stream, torch,
                                                                           1.0 / 16)}
    if args.cusp_fp64:
        w = {"workload": full.name + " to t=1/256 with dt_max=1/256"}
        for name, p in (("mixed", nb.NB_MIXED), ("fp64", nb.NB_FP64)):
            w[name] = cusp_run(nb, full, p, stream, torch, 1.0 / 256, dt_max=1.0 / 256)
        # the drift of the holes' two-body elements that the precision causes:
        # mixed minus FP64 at the same time (the elements themselves are not
        # conserved, the stars inside the orbit outweigh the binary)
        w["binary_a_mixed_minus_fp64"] = w["mixed"]["binary_a"][1] - w["fp64"]["binary_a"][1]
        w["binary_e_mixed_minus_fp64"] = w["mixed"]["binary_e"][1] - w["fp64"]["binary_e"][1]
        res["full_short"] = w
    r["binary_a_mixed_minus_fp64"] = r["mixed"]["binary_a"][1] - r["fp64"]["binary_a"][1]
    r["binary_e_mixed_minus_fp64"] = r["mixed"]["binary_e"][1] - r["fp64"]["binary_e"][1]
    return res


def extras(args, nb, ics, wl, ctx, stream, out, prec):
    import torch
    n = wl.n
    h = args.block_step
    flop_pi = FLOPS_PER_INTERACTION[wl.order]
    # ---- e2e through the C ABI with host state in and out every step, from
    #      and to page-locked host memory
    try:
        def pinned(*shape):
            return torch.empty(shape, dtype=torch.float64, pin_memory=True).numpy()

        S = {"x": pinned(n, 3), "v": pinned(n, 3), "d": pinned(n, 6, 3), "t": pinned(n), "dt": pinned(n)}
        R = {"x": pinned(n, 3), "v": pinned(n, 3), "d": pinned(n, 6, 3), "t": pinned(n), "dt": pinned(n)}
        ctx.get_state(out=S)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            ctx.set_state(S["x"], S["v"], S["d"], S["t"], S["dt"])
            ctx.set_block_step(h)
            ctx.block_step()
            ctx.get_state(out=R)
        el = time.perf_counter() - t0
        per = 8 * (3 + 3 + 18 + 1 + 1)
        out["e2e"] = {"value": args.steps * n * n / el, "unit": "interactions/s", "h2d_bytes_per_step": per * n,
                      "d2h_bytes_per_step": per * n,
                      "path": "nb_set_state (pinned host) + nb_set_block_step + nb_block_step + nb_get_state (pinned host)"}
        del R
    except Exception as e:  # pragma: no cover
        out["e2e"] = {"error": repr(e)}
    # ---- FP64 path vs mixed on the same 4096-particle block
    try:
        rng = np.random.default_rng(7)
        blk = np.sort(rng.choice(n, 4096, replace=False)).astype(np.int32)
        res = {}
        for name, p in (("fp64", nb.NB_FP64), ("mixed", nb.NB_MIXED)):
            ctx.set_precision(p)
            ctx.set_state(S["x"], S["v"], S["d"], S["t"], S["dt"])
            t_next = float(S["t"][0]) + h
            ctx.predict(t_next)
            ctx.force(blk)
            ctx.set_profiling(True)
            reps = 2 if name == "fp64" else 10
            for _ in range(reps):
                ctx.force(blk)
            prof, _ = ctx.get_profile()
            ctx.set_profiling(False)
            fms = prof["force"][0] / reps
            res[name] = len(blk) * n / (fms * 1e-3)
        ctx.set_precision(prec)
        out["fp64"] = {"interactions_per_s": res["fp64"], "tflops_convention": res["fp64"] * flop_pi / 1e12,
                       "frac_of_fp64_peak": res["fp64"] * flop_pi / 1e12 / FP64_PEAK_TFLOPS,
                       "block": f"{len(blk)} active of {n}"}
        out["mixed_same_block"] = {"interactions_per_s": res["mixed"]}
        out["mixed_vs_fp64"] = res["mixed"] / res["fp64"]
    except Exception as e:  # pragma: no cover
        out["fp64"] = {"error": repr(e)}
    # ---- the GPU force of every particle of the nucleus on a predicted
    #      store; the cpu_baseline leg times the oracle on a sample of the same
    #      particles and store and compares the two (the parity gate of the
    #      test suite)
    held = {}
    try:
        ctx.set_state(S["x"], S["v"], S["d"], S["t"], S["dt"])
        ctx.predict(float(S["t"][0]) + h)
        ctx.force(np.arange(n, dtype=np.int32))
        held["G"] = ctx.get_force(n)
        held["pred"] = ctx.get_predicted()[:3]
    except Exception as e:  # pragma: no cover
        held["error"] = repr(e)
    # ---- per-N_act curve of the mixed force on the 2^20 store (powers of two)
    try:
        ctx.set_state(S["x"], S["v"], S["d"], S["t"], S["dt"])
        ctx.predict(float(S["t"][0]) + h)
        rng = np.random.default_rng(11)
        curve = {}
        for k in range(0, 21):
            na = min(1 << k, n)
            blk = np.sort(rng.choice(n, na, replace=False)).astype(np.int32)
            ctx.force(blk)
            ctx.set_profiling(True)
            reps = 2 if na >= 262144 else 3 if na >= 65536 else 10
            for _ in range(reps):
                ctx.force(blk)
            prof, _ = ctx.get_profile()
            ctx.set_profiling(False)
            fms = (prof["force"][0] + prof["reduce"][0]) / reps
            curve[str(na)] = na * n / (fms * 1e-3)
        out["nact_curve_interactions_per_s"] = curve
    except Exception as e:  # pragma: no cover
        out["nact_curve_interactions_per_s"] = {"error": repr(e)}
    # ---- energy error of both paths after one time unit: a Plummer sphere of
    #      --energy-n particles (the FP64 path finishes it in well under a
    #      minute) on both paths; then the 65536-particle sphere to the same
    #      time on the mixed path as host-driven cycles, CUDA-graph replays of 64
    #      device-driven cycles, and graph replays with autotuned shapes
    try:
        t_end = args.energy_t

        def energy_run(w, p, cyc, tune=0):
            c2 = nb.NBody(w.n, 6, math.sqrt(w.eps2[0]), p)
            c2.set_stream(stream)
            c2.set_params(w.eta, w.eta_s, w.dt_max, 2.0 ** -40)
            c2.set_particles(w.m, w.x, w.v)
            c2.set_precision(nb.NB_FP64)
            e0 = sum(c2.energy())
            S0 = c2.get_state()
            c2.set_precision(p)
            c2.set_graph(cyc)
            rec = {}
            if tune:  # after set_graph: tuned with the kernels graph cycles run
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                c2.autotune(tune)
                rec["autotune_seconds"] = time.perf_counter() - t0
            c2.get_nact_histogram(reset=True)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            nblk, ni = c2.step_until(t_end)
            torch.cuda.synchronize()
            el = time.perf_counter() - t0
            hist = c2.get_nact_histogram()
            rec["nact_histogram"] = {f"{1 << k}-{(2 << k) - 1}": int(hist[k]) for k in np.nonzero(hist)[0]}
            S1 = c2.get_state()
            xf = S1["x"]
            c2.set_precision(nb.NB_FP64)
            e1 = sum(c2.energy())
            c2.close()
            rec.update({"dE_E": (e1 - e0) / abs(e0), "dP_rel": momentum_drift(S0, S1, w.m), "blocks": nblk,
                        "interactions": ni,
                        "whole_run_interactions_per_s": ni / el, "seconds": el})
            return rec, xf

        ws = ics.plummer_cluster(args.energy_n, 1001, 1e-4, 6, t_end)
        both = {}
        for name, p in (("fp64", nb.NB_FP64), ("mixed", nb.NB_MIXED)):
            both[name], _ = energy_run(ws, p, 64)
        both["mixed_within_2x"] = abs(both["mixed"]["dE_E"]) <= 2 * abs(both["fp64"]["dE_E"])
        both["time_to_solution_ratio"] = both["fp64"]["seconds"] / both["mixed"]["seconds"]
        pw = ics.standard_workload(1)
        de, final = {}, {}
        for name, cyc, tune in (("mixed_host", 0, 0), ("mixed_graph", 64, 0), ("mixed_graph_tuned", 64, 3)):
            de[name], final[name] = energy_run(pw, nb.NB_MIXED, cyc, tune)
        de["mixed_graph"]["same_state_as_host_driven"] = bool(np.array_equal(final["mixed_host"],
                                                                              final["mixed_graph"]))
        out["energy_budget"] = {"workload": ws.name + f" to t={t_end}, graph replays, both paths", **both,
                                "plummer65k": {"workload": pw.name + f" to t={t_end}, mixed", **de}}
    except Exception as e:  # pragma: no cover
        out["energy_budget"] = {"error": repr(e)}
    # ---- Plummer N = 1024 to t = 0.125 end to end on both GPU paths (the
    #      cpu_baseline leg runs the oracle on it: the FP64 path must take the
    #      oracle's blocks)
    try:
        w0 = ics.standard_workload(0)
        rec = {"workload": w0.name + f" to t={w0.t_end}"}
        states = {}
        for name, p in (("fp64", nb.NB_FP64), ("mixed", nb.NB_MIXED)):
            c0 = nb.NBody(w0.n, w0.order, math.sqrt(w0.eps2[0]), p)
            c0.set_stream(stream)
            c0.set_params(w0.eta, w0.eta_s, w0.dt_max, 2.0 ** -40)
            c0.set_particles(w0.m, w0.x, w0.v)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            nblk, ni = c0.step_until(w0.t_end)
            torch.cuda.synchronize()
            el = time.perf_counter() - t0
            states[name] = c0.get_state()
            rec[name] = {"blocks": nblk, "interactions": ni, "seconds": el, "interactions_per_s": ni / el}
            c0.close()
        out["plummer_1k_end_to_end"] = rec
        held["w0"], held["fp64_1k"] = w0, (rec["fp64"], states["fp64"])
    except Exception as e:  # pragma: no cover
        out["plummer_1k_end_to_end"] = {"error": repr(e)}
    # ---- force kernel at N_act = N on each single-system workload (mixed),
    #      and the FP64 path on a 4096-particle block of each; last, the
    #      nucleus at 4th order (acc and jerk only, 60 flops per interaction)
    try:
        import dataclasses
        table = {}
        for k in range(5):
            w = ics.standard_workload(k) if k not in (2, 4) else wl
            if k == 4:
                w = dataclasses.replace(wl, order=4, name=wl.name + "_order4")
            fl = FLOPS_PER_INTERACTION[w.order]
            row = {"n": w.n, "order": w.order}
            for name, p, na in (("mixed", nb.NB_MIXED, w.n), ("fp64", nb.NB_FP64, min(4096, w.n))):
                c3 = make_ctx(nb, w, p, stream) if k != 2 else ctx
                c3.set_precision(p)
                c3.predict(2.0 ** -12)
                blk = np.arange(w.n, dtype=np.int32) if na == w.n else \
                    np.sort(np.random.default_rng(k).choice(w.n, na, replace=False)).astype(np.int32)
                c3.force(blk)
                reps = 5 if name == "mixed" else 2
                c3.set_profiling(True)
                for _ in range(reps):
                    c3.force(blk)
                pr, _ = c3.get_profile()
                c3.set_profiling(False)
                fms = (pr["force"][0] + pr["reduce"][0]) / reps
                rate = na * w.n / (fms * 1e-3)
                peak = FP32_PEAK_TFLOPS if name == "mixed" else FP64_PEAK_TFLOPS
                row[name] = {"n_act": na, "interactions_per_s": rate, "gflops_convention": rate * fl / 1e9,
                             "frac_of_peak": rate * fl / 1e12 / peak}
                if k != 2:
                    c3.close()
            ctx.set_precision(prec)
            table[w.name] = row
        out["per_workload_force"] = {"note": "force + split reduction at N_act = N (mixed) and on a 4096 block "
                                             "(FP64); peaks: FP32 lanes x 2 x 2032 MHz / nominal FP64 1.25 TFLOP/s",
                                     **table}
    except Exception as e:  # pragma: no cover
        out["per_workload_force"] = {"error": repr(e)}
    # ---- galactic nucleus: energy error of both paths on the 2^16-star
    #      version of the benchmark system to t = 1/16 (FP64 cannot finish the
    #      2^20 one); the 2^20 mixed run with --nucleus-full
    try:
        nuc = {}
        ws = ics.plummer_nucleus(1 << 16, 1002, 1e-5, 1.0 / 16)
        nuc["reduced"] = {"workload": ws.name + " to t=1/16"}
        for name, p in (("mixed", nb.NB_MIXED), ("fp64", nb.NB_FP64)):
            nuc["reduced"][name] = nucleus_run(nb, ws, p, stream, torch, 1.0 / 16)
        r = nuc["reduced"]
        r["mixed_dE_within_2x_of_fp64"] = abs(r["mixed"]["dE_E"]) <= 2 * abs(r["fp64"]["dE_E"])
        if args.nucleus_trend:
            for k in (14, 17):
                wk = ics.plummer_nucleus(1 << k, 1002, 1e-5, 1.0 / 16)
                rk = {"workload": wk.name + " to t=1/16"}
                for name, p in (("mixed", nb.NB_MIXED), ("fp64", nb.NB_FP64)):
                    rk[name] = nucleus_run(nb, wk, p, stream, torch, 1.0 / 16, graph=64)
                rk["mixed_dE_within_2x_of_fp64"] = abs(rk["mixed"]["dE_E"]) <= 2 * abs(rk["fp64"]["dE_E"])
                nuc[f"stars_2p{k}"] = rk
        if args.nucleus_full:
            nuc["full"] = {"workload": wl.name + " to t=1/16",
                           "mixed": nucleus_run(nb, wl, nb.NB_MIXED, stream, torch, 1.0 / 16, graph=64)}
        if args.nucleus_fp64 > 0:
            T = args.nucleus_fp64
            r = {"workload": wl.name + f" to t={T} with dt_max={T}, every path started and measured in its own "
                             "precision (energies in FP64)"}
            for name, p in (("mixed", nb.NB_MIXED), ("fp64", nb.NB_FP64)):
                r[name] = nucleus_run(nb, wl, p, stream, torch, T, graph=64, dt_max=T)
            # over so short a horizon neither path has a truncation error above the rounding of the energy
            # sum: the FP64 figure is that rounding, the mixed one the floor of its FP32 pair terms
            r["note"] = "short horizon: energy errors are rounding floors, not truncation errors"
            r["whole_run_rate_ratio"] = (r["mixed"]["whole_run_interactions_per_s"] /
                                         r["fp64"]["whole_run_interactions_per_s"])
            nuc["full_short_both"] = r
        out["nucleus_energy"] = nuc
    except Exception as e:  # pragma: no cover
        out["nucleus_energy"] = {"error": repr(e)}
    # ---- cusp nucleus, order 8: energy and binary-element drift of both paths
    try:
        out["cusp8"] = cusp_leg(args, nb, ics, stream, torch)
    except Exception as e:  # pragma: no cover
        out["cusp8"] = {"error": repr(e)}
    # ---- ensemble: 256 Plummer clusters, batched vs one context per cluster
    try:
        clusters = ics.ensemble()
        sizes = [c.n for c in clusters]
        t_ens = args.ensemble_t
        m = np.concatenate([c.m for c in clusters])
        x = np.concatenate([c.x for c in clusters])
        v = np.concatenate([c.v for c in clusters])
        # the plan's wave count, autotuned on a copy of the ensemble (the
        # tuning cycles advance the state they run on)
        bt = nb.Batch(sizes, 6, math.sqrt(clusters[0].eps2[0]), nb.NB_MIXED)
        bt.set_stream(stream)
        bt.set_params(0.2, 0.01, 1.0 / 16, 2.0 ** -40)
        bt.set_particles(m, x, v)
        t0 = time.perf_counter()
        tuned_waves, tune_ms = bt.autotune(cycles=48, reps=2)
        tune_s = time.perf_counter() - t0
        bt.close()
        runs = {}
        for name, cyc, waves in (("host", 0, 4), ("graph", 32, 4), ("graph_tuned", 32, tuned_waves)):
            bt = nb.Batch(sizes, 6, math.sqrt(clusters[0].eps2[0]), nb.NB_MIXED)
            bt.set_stream(stream)
            bt.set_params(0.2, 0.01, 1.0 / 16, 2.0 ** -40)
            bt.set_graph(cyc)
            bt.set_waves(waves)
            bt.set_particles(m, x, v)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            ncyc, ni_b = bt.step_until(t_ens)
            torch.cuda.synchronize()
            runs[name] = (ncyc, ni_b, time.perf_counter() - t0, bt.get_state()["x"])
            bt.close()
        ncyc, ni_b, el_b, xb = runs["graph"]
        same = bool(np.array_equal(xb, runs["host"][3]))
        ni_s, el_s = 0, 0.0
        for c in clusters:
            cx = nb.NBody(c.n, 6, math.sqrt(c.eps2[0]), nb.NB_MIXED)
            cx.set_stream(stream)
            cx.set_particles(c.m, c.x, c.v)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            _, ni = cx.step_until(t_ens)
            torch.cuda.synchronize()
            el_s += time.perf_counter() - t0
            ni_s += ni
            cx.close()
        out["ensemble"] = {"workload": f"{len(sizes)} Plummer clusters, N_k log-uniform in [1024, 32768] "
                                       f"({int(sum(sizes))} particles), order 6, mixed, to t={t_ens}",
                           "batched_interactions_per_s": ni_b / el_b, "batched_cycles": ncyc,
                           "batched_seconds": el_b, "batched": "CUDA-graph replays of 32 device-planned cycles",
                           "batched_host_cycles_interactions_per_s": runs["host"][1] / runs["host"][2],
                           "batched_autotuned": {"waves": tuned_waves, "tune_ms_per_wave_count": tune_ms,
                                                 "tune_seconds": tune_s,
                                                 "interactions_per_s": runs["graph_tuned"][1] / runs["graph_tuned"][2]},
                           "graph_state_equals_host_cycles": same,
                           "per_cluster_interactions_per_s": ni_s / el_s,
                           "per_cluster_seconds": el_s, "interactions": ni_b,
                           "speedup": (ni_b / el_b) / (ni_s / el_s)}
    except Exception as e:  # pragma: no cover
        out["ensemble"] = {"error": repr(e)}
    # ---- CPU baseline: the oracle on the host cores (bounded samples), the
    #      one place this arm runs it
    cpu_baseline_leg(wl, prec, held, out)
    torch.cuda.synchronize()


def cpu_baseline_leg(wl, prec, held, out):
    """The oracle timed on the host cores: the force of a sample of the
    nucleus (both holes among them) on the GPU's predicted store, whose
    results are also compared with the GPU's for the same particles; the same
    on one thread; and the 1024-particle Plummer run end to end, whose blocks
    the FP64 path must reproduce."""
    n = wl.n
    try:
        import oracle as orc
        from oracle import parity
        n_s, nth = oracle_rate(wl)
        rng = np.random.default_rng(3)
        idx = np.unique(np.concatenate([rng.choice(n - 2, max(n_s - 2, 1), replace=False),
                                        [n - 2, n - 1]])).astype(np.int32)
        xp, vp, ap = held["pred"]
        t0 = time.perf_counter()
        O = orc.force(wl.m, wl.eps2, xp, vp, ap, None, order=wl.order, idx=idx, nthreads=nth)
        el = time.perf_counter() - t0
        out["cpu_baseline"] = {"value": len(idx) * n / el, "unit": "interactions/s", "cores": nth, "kind": "oracle",
                               "sample": f"force of {len(idx)} of {n} particles (both holes among them) on all {n} "
                                         f"of the GPU's predicted store (long-double direct sum), {el:.1f} s"}
        G = held["G"]
        st = parity.force_parity({k: G[k][idx] for k in G}, O, wl.order, prec)
        out["cpu_baseline"]["parity_on_sample"] = {
            "within_gate": all(r["worst"] <= 1.0 for r in st.values()),
            **{k: {"strict_pass": r["strict_pass"], "worst_over_gate": r["worst"], "worst_rel_err": r["rel_err"],
                   "worst_cond": r["cond"]} for k, r in st.items()}}
        # the same oracle on one host thread
        n_1, _ = oracle_rate(wl, n_target_s=4.0, nthreads=1)
        idx = np.sort(np.random.default_rng(4).choice(n, n_1, replace=False)).astype(np.int32)
        t0 = time.perf_counter()
        orc.force(wl.m, wl.eps2, wl.x, wl.v, np.zeros_like(wl.x), None, order=wl.order, idx=idx, nthreads=1)
        el = time.perf_counter() - t0
        out["cpu_baseline"]["one_thread"] = {
            "value": n_1 * n / el, "unit": "interactions/s", "cores": 1,
            "sample": f"force of {n_1} of {n} particles on all {n}, {el:.1f} s"}
        # the 1024-particle Plummer sphere end to end
        if "w0" in held:
            w0 = held["w0"]
            rec64, st64 = held["fp64_1k"]
            so = orc.State(w0.m, w0.eps2, w0.x, w0.v)
            t0 = time.perf_counter()
            nblk_o = int(orc.integrate(so, order=w0.order, t_end=w0.t_end, eta=w0.eta, nthreads=nth))
            el = time.perf_counter() - t0
            out["cpu_baseline"]["plummer_1k_end_to_end"] = {
                "workload": w0.name + f" to t={w0.t_end}", "seconds": el, "cores": nth, "blocks": nblk_o,
                "interactions_per_s": rec64["interactions"] / el,
                "fp64_blocks_equal_oracle": rec64["blocks"] == nblk_o,
                "fp64_steps_equal_oracle": bool(np.array_equal(st64["dt"], so.dt)),
                "fp64_max_position_difference": float(np.max(np.abs(st64["x"] - so.x)))}
    except Exception as e:  # pragma: no cover
        out["cpu_baseline"] = {"error": repr(e)}


# ------------------------------------------------------------ profiling cases
def _profile_workload(args):
    from paper_1312_1789_b300 import ics
    return ics.standard_workload({"nucleus": 2, "cusp": 3, "plummer65k": 1}[args.workload])


def profile_force(args):
    """Small, self-contained force case for ncu.

    Builds the workload (default: the 2^20-star nucleus, order 6; cusp: 2^18
    stars and a binary, order 8), runs the start-up in mixed precision (mixed
    force launches over every particle: 2 at order 6, 3 at order 8), predicts
    in --precision, then launches the force --repeat times on one block of
    --n-act particles.  With ncu, `-k regex:k_force_mixed -s 2 -c 1` (order 6;
    -s 3 at order 8) or `-k regex:k_force_fp64 -s 0 -c 1` captures the first
    block launch."""
    from paper_1312_1789_b300 import build, nb
    build.build()
    wl = _profile_workload(args)
    prec = nb.NB_MIXED if args.precision == "mixed" else nb.NB_FP64
    # start-up in mixed precision (an FP64 start-up of 2^20 particles takes
    # minutes), then the block in the requested precision
    ctx = nb.NBody(wl.n, wl.order, 0.0, nb.NB_MIXED)
    ctx.set_softening(np.sqrt(wl.eps2))
    ctx.set_particles(wl.m, wl.x, wl.v)
    ctx.set_precision(prec)
    ctx.predict(2.0 ** -12)
    blk = np.sort(np.random.default_rng(7).choice(wl.n, min(args.n_act, wl.n), replace=False)).astype(np.int32)
    ctx.set_profiling(True)
    for _ in range(args.repeat):
        ctx.force(blk)
    prof, _ = ctx.get_profile()
    ms = prof["force"][0] / max(prof["force"][1], 1)
    print(f"{wl.name} {args.precision}: block {len(blk)}, launch {ctx.get_launch()}, force kernel {ms:.3f} ms, "
          f"{len(blk) * wl.n / (ms * 1e-3):.3e} interactions/s")
    ctx.close()


def profile_step(args):
    """Block steps whose active set is the first --n-act particles, for ncu
    captures of the scheduler, predictor and corrector: after the start-up
    (mixed), every particle gets the step 2^-12, then those of the first n-act
    particles are halved; each of the --repeat block steps then runs the
    scheduler's two passes (the second with the predictor), the force and the
    corrector on those n-act particles (whose new steps are reset before the
    next one)."""
    from paper_1312_1789_b300 import build, nb
    build.build()
    wl = _profile_workload(args)
    prec = nb.NB_MIXED if args.precision == "mixed" else nb.NB_FP64
    ctx = nb.NBody(wl.n, wl.order, 0.0, nb.NB_MIXED)
    ctx.set_softening(np.sqrt(wl.eps2))
    ctx.set_particles(wl.m, wl.x, wl.v)
    ctx.set_precision(prec)
    S = ctx.get_state()
    na = min(args.n_act, wl.n)
    ctx.set_profiling(True)
    for _ in range(args.repeat):
        dt = np.full(wl.n, 2.0 ** -12)
        dt[:na] = 2.0 ** -13
        ctx.set_state(S["x"], S["v"], S["d"], S["t"], dt)
        tb, n_act = ctx.block_step()
        assert n_act == na, (n_act, na)
    prof, launches = ctx.get_profile()
    print(f"{wl.name} {args.precision}: {args.repeat} block steps of {na} active; per step (ms): " +
          ", ".join(f"{k} {v[0] / args.repeat:.4f}" for k, v in prof.items()) + f"; launches {launches}")
    ctx.close()


def main():
    args = parse()
    if args.profile_force:
        profile_force(args)
        return
    if args.profile_step:
        profile_step(args)
        return
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
