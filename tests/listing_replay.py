"""Replay of an optimized listing (circuit_io.plan_listing) with the FP64 oracle, for tests."""
import numpy as np

import oracle
from paper_2406_14084_gb300.workloads import Gate


def replay_listing(text: str, n: int, state):
    """Apply an optimized listing with the FP64 oracle on physical positions; returns the layout
    (physical position of each logical qubit)."""
    layout = list(range(n))
    for row in text.splitlines():
        f = row.split()
        if not f:
            continue
        head = f[0]
        if head == "LAYOUT":
            layout = [int(v) for v in f[1:]]
            continue
        if head == "SQS":
            k = int(f[1])
            A = [int(v) for v in f[2:2 + k]]
            B = [int(v) for v in f[2 + k:2 + 2 * k]]
            oracle.remap(state, n, A, B)
            continue
        rest = f[1:]
        ctl = ()
        if "C" in rest:
            ci = rest.index("C")
            # controls run until the first token that is not an integer position
            j = ci + 1
            while j < len(rest) and rest[j].lstrip("-").isdigit() and "." not in rest[j]:
                j += 1
            ctl = tuple(int(v) for v in rest[ci + 1:j])
            rest = rest[:ci] + rest[j:]
        if head.startswith("U") or head.startswith("D"):
            k = int(head[1:])
            t = tuple(int(v) for v in rest[:k])
            vals = [float(v) for v in rest[k:]]
            z = np.array(vals[0::2]) + 1j * np.array(vals[1::2])
            if head.startswith("U"):
                g = Gate("UNITARY", t, ctl, (), z.reshape(1 << k, 1 << k))
            else:
                g = Gate("DIAG", t, ctl, (), z)
        elif head == "X":
            g = Gate("X", (int(rest[0]),), ctl)
        elif head == "SWAP":
            g = Gate("SWAP", (int(rest[0]), int(rest[1])), ctl)
        elif head == "PHASE":
            vals = [float(v) for v in rest]
            p = vals[0] + 1j * vals[1]
            # a phase on the amplitudes where all controls are 1
            if ctl:
                g = Gate("DIAG", (ctl[0],), ctl[1:], (), np.array([1.0, p]))
            else:
                state *= p
                continue
        else:
            raise ValueError(f"unknown listing line {row!r}")
        oracle.apply_circuit(n, [g], state)
    return layout
