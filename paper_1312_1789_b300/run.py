"""Run a simulation from a JSON configuration.

Block steps to t_end with an output every dt_out: one JSON line of run metrics
per output (time, blocks, interactions, wall seconds, interactions/s, energy
error, momentum drift, block-size histogram of the interval), a checkpoint of
the state at each output, and resumption from a checkpoint.  Every step runs in
libnb's kernels through nb.NBody; this module only sequences the calls.

Configuration keys (DEFAULTS below fills the rest):
  workload      "plummer1k", "plummer65k", "nucleus", "cusp" (the standard
                problems of ics.standard_workload), a dict
                {"model": "plummer", "n": N, "seed": S, "eps": E}, or
                {"model": "ensemble", "clusters": K, "lo": N0, "hi": N1}
                (independent Plummer clusters stepped together, order 6;
                outputs give the per-cluster energy errors; no checkpoints)
  order         4, 6 or 8 (default: the workload's)
  precision     "mixed" or "fp64"
  eta, eta_s, dt_max, dt_min   time-step parameters (default: the workload's)
  t_end         end time; dt_out the output interval: both multiples of
                dt_max, so that every particle is at the output time
  graph_cycles  > 0: device-driven cycles replayed as a CUDA graph
  autotune      reps of the launch-shape autotuner (0: the analytic rule)
  tuning        path of a table NBody.save_tuning wrote (instead of autotune)
  checkpoint    path prefix: the state at every output goes to
                <prefix>_t<time>.npz, and <prefix>_last.npz
  resume        a checkpoint file to continue from (its workload is rebuilt
                from the same configuration; the state comes from the file).
                A resumed run takes the same blocks with the same bits as an
                uninterrupted one when the launch shapes are the same: the
                analytic rule or a saved table, not a fresh autotune.

    python -m paper_1312_1789_b300.run config.json [--log run.jsonl]
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import sys
import time

import numpy as np

from . import ics, nb

DEFAULTS = {
    "workload": "plummer1k", "order": None, "precision": "mixed", "eta": None, "eta_s": None, "dt_max": None,
    "dt_min": 2.0 ** -40, "t_end": None, "dt_out": None, "graph_cycles": 64, "autotune": 0, "tuning": None,
    "checkpoint": None, "resume": None,
}
STANDARD = {"plummer1k": 0, "plummer65k": 1, "nucleus": 2, "cusp": 3}


def load_config(cfg: dict) -> dict:
    """The configuration with defaults filled in and checked (ValueError)."""
    unknown = set(cfg) - set(DEFAULTS)
    if unknown:
        raise ValueError(f"unknown configuration keys: {sorted(unknown)}")
    c = dict(DEFAULTS, **cfg)
    wl = c["workload"]
    if isinstance(wl, str) and wl not in STANDARD:
        raise ValueError(f"workload must be one of {sorted(STANDARD)} or a dict")
    if isinstance(wl, dict) and wl.get("model") not in ("plummer", "ensemble"):
        raise ValueError("a custom workload is {'model': 'plummer', 'n': N, 'seed': S, 'eps': E} or "
                         "{'model': 'ensemble', 'clusters': K, 'lo': N0, 'hi': N1}")
    if isinstance(wl, dict) and wl.get("model") == "ensemble":
        if c["checkpoint"] or c["resume"] or c["tuning"] or c["autotune"]:
            raise ValueError("an ensemble run takes no checkpoint, resume or launch tuning")
        if c["order"] not in (None, 6):
            raise ValueError("ensembles run at order 6")
    if c["precision"] not in ("mixed", "fp64"):
        raise ValueError("precision must be 'mixed' or 'fp64'")
    if c["order"] is not None and c["order"] not in (4, 6, 8):
        raise ValueError("order must be 4, 6 or 8")
    return c


def build_workload(c: dict) -> ics.Workload:
    wl = c["workload"]
    if isinstance(wl, str):
        w = ics.standard_workload(STANDARD[wl])
    else:
        w = ics.plummer_cluster(int(wl["n"]), int(wl.get("seed", 1000)), float(wl.get("eps", 1e-4)))
    for key in ("order", "eta", "eta_s", "dt_max", "t_end"):
        if c[key] is not None:
            setattr(w, key, type(getattr(w, key))(c[key]))
    return w


def _steps(c: dict, w: ics.Workload):
    """Output times: multiples of dt_out up to t_end, each a multiple of dt_max."""
    dt_out = c["dt_out"] if c["dt_out"] is not None else w.t_end
    for val, name in ((dt_out, "dt_out"), (w.t_end, "t_end")):
        q = val / w.dt_max
        if not (q >= 1 and q == math.floor(q)):
            raise ValueError(f"{name} = {val} must be a positive multiple of dt_max = {w.dt_max}")
    q = w.t_end / dt_out
    if q != math.floor(q):
        raise ValueError(f"t_end = {w.t_end} must be a multiple of dt_out = {dt_out}")
    return [dt_out * (k + 1) for k in range(int(q))]


def _momentum(S, m):
    return (m[:, None] * S["v"]).sum(axis=0), float((m * np.linalg.norm(S["v"], axis=1)).sum())


def _energy(ctx, prec):
    # every output time is a multiple of dt_max, so all particles are there;
    # the energy is taken in FP64 whatever the integration's precision
    ctx.set_precision(nb.NB_FP64)
    e = sum(ctx.energy())
    ctx.set_precision(prec)
    return e


def fingerprint(w: ics.Workload) -> str:
    """Digest of a workload's initial conditions (a checkpoint names the run it belongs to)."""
    h = hashlib.sha256()
    for a in (w.m, w.x, w.v, w.eps2):
        h.update(np.ascontiguousarray(a, dtype=np.float64).tobytes())
    return h.hexdigest()


def save_checkpoint(path: str, S, w, cfg, t, e0, p0, pscale, blocks, inter, fp):
    """Write the state S (NBody.get_state) and the run's bookkeeping to path."""
    d = os.path.dirname(path)
    if d:
        os.makedirs(d, exist_ok=True)
    np.savez(path, x=S["x"], v=S["v"], d=S["d"], t=S["t"], dt=S["dt"],
             meta=json.dumps({"config": cfg, "time": t, "e0": e0, "p0": [float(q) for q in p0], "pscale": pscale,
                              "blocks": blocks, "interactions": inter, "workload": w.name,
                              "fingerprint": fp}))


def _run_ensemble(c: dict, log, stream):
    wl = c["workload"]
    clusters = ics.ensemble(int(wl.get("clusters", 256)), int(wl.get("lo", 1024)), int(wl.get("hi", 32768)))
    w0 = clusters[0]
    dt_max = c["dt_max"] if c["dt_max"] is not None else w0.dt_max
    t_end = c["t_end"] if c["t_end"] is not None else w0.t_end
    probe = ics.Workload("ensemble", w0.m, w0.x, w0.v, w0.eps2, dt_max=dt_max, t_end=t_end)
    outs = _steps(c, probe)
    prec = nb.NB_MIXED if c["precision"] == "mixed" else nb.NB_FP64
    sizes = [w.n for w in clusters]
    b = nb.Batch(sizes, 6, math.sqrt(w0.eps2[0]), prec)
    try:
        if stream is not None:
            b.set_stream(stream)
        b.set_params(c["eta"] if c["eta"] is not None else w0.eta, c["eta_s"] if c["eta_s"] is not None else w0.eta_s,
                     dt_max, c["dt_min"])
        b.set_particles(np.concatenate([w.m for w in clusters]), np.concatenate([w.x for w in clusters]),
                        np.concatenate([w.v for w in clusters]))
        b.set_graph(int(c["graph_cycles"]))
        ek, ep = b.energy()
        e0 = ek + ep
        cycles, inter, records = 0, 0, []
        for t_out in outs:
            t0 = time.perf_counter()
            nc, ni = b.step_until(t_out)
            el = time.perf_counter() - t0
            cycles, inter = cycles + nc, inter + ni
            ek, ep = b.energy()
            de = np.abs((ek + ep - e0) / np.abs(e0))
            rec = {"workload": f"ensemble_{len(sizes)}_clusters", "t": t_out, "cycles": cycles,
                   "interactions": inter, "seconds": el, "interactions_per_s": ni / el if el > 0 else None,
                   "dE_E_median": float(np.median(de)), "dE_E_worst": float(de.max())}
            records.append(rec)
            if log is not None:
                log.write(json.dumps(rec) + "\n")
                log.flush()
        return records
    finally:
        b.close()


def run(cfg: dict, log=None, stream=None):
    """Integrate as the configuration says; returns the list of output records
    (also written, one JSON line each, to the file object `log`)."""
    c = load_config(cfg)
    if isinstance(c["workload"], dict) and c["workload"]["model"] == "ensemble":
        return _run_ensemble(c, log, stream)
    w = build_workload(c)
    prec = nb.NB_MIXED if c["precision"] == "mixed" else nb.NB_FP64
    outs = _steps(c, w)
    fp = fingerprint(w)
    ctx = nb.NBody(w.n, w.order, 0.0, prec)
    try:
        if stream is not None:
            ctx.set_stream(stream)
        ctx.set_softening(np.sqrt(w.eps2))
        ctx.set_params(w.eta, w.eta_s, w.dt_max, c["dt_min"])
        t_now, blocks, inter = 0.0, 0, 0
        if c["resume"]:
            ck = np.load(c["resume"])
            meta = json.loads(str(ck["meta"]))
            if meta["fingerprint"] != fp:
                raise ValueError(f"the checkpoint belongs to another run ({meta['workload']})")
            ctx.set_particles(w.m, ck["x"], ck["v"])
            ctx.set_state(ck["x"], ck["v"], ck["d"], ck["t"], ck["dt"])
            t_now, blocks, inter = meta["time"], meta["blocks"], meta["interactions"]
            e0, p0, pscale = meta["e0"], np.array(meta["p0"]), meta["pscale"]
            outs = [t for t in outs if t > t_now]
        else:
            ctx.set_particles(w.m, w.x, w.v)
            e0 = _energy(ctx, prec)
            p0, pscale = _momentum(ctx.get_state(), w.m)
        # graph mode first: the autotuner times the kernels of the current mode
        ctx.set_graph(int(c["graph_cycles"]))
        if c["tuning"]:
            ctx.load_tuning(c["tuning"])
        elif c["autotune"] > 0:
            ctx.autotune(int(c["autotune"]))
        ctx.get_nact_histogram(reset=True)
        records = []
        for t_out in outs:
            t0 = time.perf_counter()
            nblk, ni = ctx.step_until(t_out)  # returns once the device is done
            el = time.perf_counter() - t0
            blocks, inter = blocks + nblk, inter + ni
            e = _energy(ctx, prec)
            S = ctx.get_state()
            p, _ = _momentum(S, w.m)
            h = ctx.get_nact_histogram(reset=True)
            rec = {"workload": w.name, "t": t_out, "blocks": blocks, "interactions": inter, "seconds": el,
                   "interactions_per_s": ni / el if el > 0 else None, "dE_E": (e - e0) / abs(e0),
                   "dP_rel": float(np.linalg.norm(p - p0) / pscale),
                   "nact_histogram": {f"{1 << k}-{(2 << k) - 1}": int(h[k]) for k in np.nonzero(h)[0]}}
            if c["checkpoint"]:
                for path in (f"{c['checkpoint']}_t{t_out:.10g}.npz", f"{c['checkpoint']}_last.npz"):
                    save_checkpoint(path, S, w, cfg, t_out, e0, p0, pscale, blocks, inter, fp)
                rec["checkpoint"] = f"{c['checkpoint']}_last.npz"
            records.append(rec)
            if log is not None:
                log.write(json.dumps(rec) + "\n")
                log.flush()
        return records
    finally:
        ctx.close()


def main(argv=None):
    p = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    p.add_argument("config", help="JSON configuration file")
    p.add_argument("--log", help="JSON-lines output (default: stdout)")
    args = p.parse_args(argv)
    with open(args.config) as f:
        cfg = json.load(f)
    if args.log:
        with open(args.log, "a") as log:
            run(cfg, log)
    else:
        run(cfg, sys.stdout)


if __name__ == "__main__":
    main()
