"""Small, self-contained runs of one plan for kernel profiling (ncu) and quick timing.

    python paper_2406_14084_gb300/profile_slab.py KIND N REPS [option=value ...]

KIND: hsweep (ten H gates on seeded random qubits, complex64: one memory-bound slab pass),
layered64 / layered128 (layered depth 40, seed 1002), qft128 (no-swap QFT, complex128).
Options are qs_options fields (slab_bits=12, stage_bits=4, factor=1, ...).  Each repetition
applies the whole plan with per-step CUDA-event timing (qs_plan_profile) on a fresh state and
prints the step times and the per-pass HBM rate 2 * 2^N * s / t.
"""
import os
import sys
import time

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

import torch  # noqa: E402

from paper_2406_14084_gb300 import qs  # noqa: E402
from paper_2406_14084_gb300 import workloads as W  # noqa: E402


def circuit(kind: str, n: int):
    if kind == "hsweep":
        rng = W.SplitMix64(1008 + n)
        return qs.QS_C64, [W.Gate("H", (rng.below(n),)) for _ in range(10)]
    if kind == "layered128":
        return qs.QS_C128, W.layered(n, 40, 1002)
    if kind == "qft128":
        return qs.QS_C128, W.qft(n)
    if kind == "layered64":
        return qs.QS_C64, W.layered(n, 40, 1002)
    raise SystemExit(f"unknown kind {kind}")


def main():
    kind, n, reps = sys.argv[1], int(sys.argv[2]), int(sys.argv[3])
    extra = {k: int(v) for k, v in (a.split("=") for a in sys.argv[4:])}
    dt, gates = circuit(kind, n)
    plan = qs.qs_fuse(gates, n, qs.options(dtype=dt, **extra))
    nst = qs.qs_plan_features(plan).shape[0]
    s = 8 if dt == qs.QS_C64 else 16
    with qs.State(n, dt) as st:
        for _ in range(reps):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            ms = qs.qs_plan_profile(st.h, plan, nst)
            torch.cuda.synchronize()
            print(kind, n, "steps", len(ms), "total ms", round(float(ms.sum()), 3),
                  "wall s", round(time.perf_counter() - t0, 3),
                  "first steps", [round(float(x), 3) for x in ms[:8]])
        print("GB/s per step", [round(2 * (1 << n) * s / (float(x) / 1e3) / 1e9, 1) for x in ms[:8] if x > 0])
    qs.qs_plan_destroy(plan)


if __name__ == "__main__":
    main()
