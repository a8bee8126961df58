"""Small, self-contained force case for profilers (ncu) and quick timing.

    python -m paper_1312_1789_b300.profile_case [--n-act 4096] [--precision mixed|fp64] [--repeat 2]
                                                [--workload nucleus|cusp]

Builds the galactic-nucleus system (2^20 Plummer stars + two black holes,
6th order) or the cusp (2^18 Dehnen stars + a black-hole binary, 8th order),
runs the start-up in mixed precision (mixed force launches over every
particle: 2 at order 6, 3 at order 8), predicts in --precision, then launches
the force kernel --repeat times on one block of --n-act particles.  With ncu,
`-k regex:k_force_mixed -s 2 -c 1` (order 6; -s 3 at order 8) or
`-k regex:k_force_fp64 -s 0 -c 1` captures the first block launch.
"""
from __future__ import annotations

import argparse

import numpy as np

from . import ics, nb


def main():
    p = argparse.ArgumentParser()
    p.add_argument("--n-act", type=int, default=4096)
    p.add_argument("--precision", choices=["mixed", "fp64"], default="mixed")
    p.add_argument("--repeat", type=int, default=2)
    p.add_argument("--workload", choices=["nucleus", "cusp"], default="nucleus")
    a = p.parse_args()
    wl = ics.standard_workload(2 if a.workload == "nucleus" else 3)
    prec = nb.NB_MIXED if a.precision == "mixed" else nb.NB_FP64
    # start-up in mixed precision (an FP64 start-up of 2^20 particles takes
    # minutes), then the block in the requested precision
    ctx = nb.NBody(wl.n, wl.order, 0.0, nb.NB_MIXED)
    ctx.set_softening(np.sqrt(wl.eps2))
    ctx.set_particles(wl.m, wl.x, wl.v)
    ctx.set_precision(prec)
    ctx.predict(2.0 ** -12)
    blk = np.sort(np.random.default_rng(7).choice(wl.n, min(a.n_act, wl.n), replace=False)).astype(np.int32)
    ctx.set_profiling(True)
    for _ in range(a.repeat):
        ctx.force(blk)
    prof, _ = ctx.get_profile()
    ms = prof["force"][0] / max(prof["force"][1], 1)
    print(f"{wl.name} {a.precision}: block {len(blk)}, launch {ctx.get_launch()}, force kernel {ms:.3f} ms, "
          f"{len(blk) * wl.n / (ms * 1e-3):.3e} interactions/s")
    ctx.close()


if __name__ == "__main__":
    main()
