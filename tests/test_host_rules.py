"""Host-side launch and conversion rules of the CUDA library, checked on the CPU
against brute force and an independent definition.  A host-only harness is
compiled with nvcc from the library's own inline functions (no GPU needed):

  makespan_split   the j-split count a force launch takes (host rule and the
                   device-driven gate share it): its span ceil(it*s/slots)/s
                   must be within the rule's 1 % hysteresis of the best span
                   over every s it may choose;
  eps2_threshold   the uniform-softening threshold: the float nearest to x
                   toward zero, as the predictor stores eps^2.
"""
import os
import shutil
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1312_1789_b300", "csrc")
INCLUDE = os.path.join(ROOT, "include")

HARNESS = r"""
#include <cstdio>
#include "nb_internal.cuh"
int main()
{
    char op;
    while (std::scanf(" %c", &op) == 1) {
        if (op == 'M') {
            int it, ntiles, slots;
            long long cap;
            if (std::scanf("%d %d %d %lld", &it, &ntiles, &slots, &cap) != 4) return 1;
            std::printf("%d\n", nb::makespan_split(it, ntiles, slots, cap));
        } else if (op == 'E') {
            double x;
            if (std::scanf("%lf", &x) != 1) return 1;
            std::printf("%.17g\n", (double)nb::eps2_threshold(x));
        } else {
            return 1;
        }
    }
    return 0;
}
"""


def _nvcc():
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    pytest.skip("nvcc not found")


@pytest.fixture(scope="module")
def harness(tmp_path_factory):
    d = tmp_path_factory.mktemp("host_rules")
    src, exe = d / "harness.cu", d / "harness"
    src.write_text(HARNESS)
    subprocess.run([_nvcc(), "-std=c++17", "-gencode", "arch=compute_103a,code=sm_103a", "-I", INCLUDE, "-I", CSRC,
                    "-o", str(exe), str(src)], check=True, capture_output=True)

    def run(lines):
        out = subprocess.run([str(exe)], input="\n".join(lines) + "\n", capture_output=True, text=True, check=True)
        return out.stdout.split()
    return run


def _s_max(it, ntiles, slots, cap):
    return max(1, min(max(4 * slots // it + 4, 16), ntiles, cap))


def test_makespan_split_within_half_a_percent_of_brute_force(harness):
    rng = np.random.default_rng(11)
    cases = []
    for slots in (148, 444, 592):            # SMs x resident CTAs of the force variants
        for ntiles in (8, 33, 512, 2049, 8193):  # j tiles: 1k .. 2^20 particles
            for it in (1, 2, 3, 7, 37, 64, 148, 149, 600, 4097):
                cases.append((it, ntiles, slots, 1 << 40))
    for _ in range(300):                     # random shapes, some capped by the partial buffer
        cases.append((int(rng.integers(1, 5000)), int(rng.integers(1, 9000)), int(rng.integers(1, 700)),
                      int(rng.integers(1, 3000))))
    got = [int(s) for s in harness([f"M {it} {nt} {sl} {cap}" for it, nt, sl, cap in cases])]
    for (it, nt, sl, cap), s in zip(cases, got):
        smax = _s_max(it, nt, sl, cap)
        assert 1 <= s <= smax, (it, nt, sl, cap, s)
        span = lambda k: -(-it * k // sl) / k  # noqa: E731  waves x (1/k) of the one-split time
        best = min(span(k) for k in range(1, smax + 1))
        assert span(s) <= best / 0.995 * (1 + 1e-12), (it, nt, sl, cap, s, span(s), best)


def test_eps2_threshold_rounds_toward_zero(harness):
    rng = np.random.default_rng(12)
    xs = np.concatenate([[1e-10, 1e-8, 2.5e-9, 1e-4, 1.0, 3.0, 0.0, 1e-45, 1e-40, 3.5e38, 1e300],
                         10.0 ** rng.uniform(-44, 38, 400)])
    got = np.array([float(s) for s in harness([f"E {x:.17e}" for x in xs])])
    for x, g in zip(xs, got):
        with np.errstate(over="ignore"):
            f = np.float32(x)                # nearest float (inf past the range)
        if abs(float(f)) > abs(x):           # rounded away from zero: step back
            f = np.nextafter(f, np.float32(0))
        assert g == float(f), (x, g, float(f))
        assert g <= x
