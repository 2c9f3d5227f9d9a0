"""Replay a plan listing (qs_plan_dump) with the FP64 oracle, in physical bit positions.

Used by the CPU planner tests: the library's host planner (fusion products, diagonal tables,
slab assignment, remaps and relabels) is checked without a GPU by executing its listing one op
at a time on the oracle and comparing with the unfused circuit.
"""
import numpy as np

import oracle
from paper_2406_14084_gb300.workloads import Gate


def parse_dump(text):
    items = []
    n = None
    layout = None
    for line in text.splitlines():
        f = line.split()
        if not f:
            continue
        if f[0] == "N":
            n = int(f[1])
        elif f[0] == "PASS":
            items.append(("PASS", int(f[1]), int(f[2]), [int(v) for v in f[3:]]))
        elif f[0] == "UNBLOCKED":
            items.append(("UNBLOCKED",))
        elif f[0] == "REMAP":
            k = int(f[1])
            items.append(("REMAP", [int(v) for v in f[2:2 + k]], [int(v) for v in f[2 + k:2 + 2 * k]]))
        elif f[0] == "OP":
            kind, k = f[1], int(f[2])
            i = 3
            assert f[i] == "t"
            i += 1
            t = []
            while i < len(f) and f[i] != "c":
                t.append(int(f[i]))
                i += 1
            i += 1
            c = []
            while i < len(f) and f[i] != "m":
                c.append(int(f[i]))
                i += 1
            m = None
            if i < len(f) and f[i] == "m":
                vals = np.array([float(v) for v in f[i + 1:]])
                m = vals[0::2] + 1j * vals[1::2]
                if kind == "DENSE":
                    m = m.reshape(1 << k, 1 << k)
            items.append(("OP", kind, t, c, m))
        elif f[0] == "LAYOUT":
            layout = [int(v) for v in f[1:]]
    return n, items, layout


def op_gate(kind, t, c, m):
    if kind == "DENSE":
        return Gate("UNITARY", tuple(t), tuple(c), (), m)
    if kind == "DIAG":
        return Gate("DIAG", tuple(t), tuple(c), (), m)
    if kind == "PERMX":
        return Gate("CX" if c else "X", tuple(t), tuple(c))
    if kind == "SWAP":
        return Gate("SWAP", tuple(t), tuple(c))
    raise ValueError(kind)


ORACLE_MAX_DIAG = 12  # widest DIAG gate the oracle takes


def apply_wide_diag(state, n, t, c, m):
    """A diagonal wider than the oracle's DIAG gate, by its definition (Eq. 3 with a diagonal
    matrix): amplitude x is multiplied by m[sum_j bit(x, t_j) 2^j] where every control bit is 1."""
    x = np.arange(1 << n, dtype=np.int64)
    idx = np.zeros_like(x)
    for j, q in enumerate(t):
        idx |= ((x >> q) & 1) << j
    on = np.ones(1 << n, dtype=bool)
    for q in c:
        on &= ((x >> q) & 1) == 1
    state[on] *= m[idx[on]]


def replay(text, state):
    """Execute the listing on `state` (complex128, physical order) in place; returns layout."""
    n, items, layout = parse_dump(text)
    stats = {"passes": 0, "remaps": 0, "unblocked": 0, "ops": 0, "max_b": 0}
    for it in items:
        if it[0] == "PASS":
            stats["passes"] += 1
            stats["max_b"] = max(stats["max_b"], it[1])
            slab = set(range(it[2])) | set(it[3])
            cur_slab = slab
        elif it[0] == "UNBLOCKED":
            stats["unblocked"] += 1
            cur_slab = None
        elif it[0] == "REMAP":
            stats["remaps"] += 1
            oracle.remap(state, n, it[1], it[2])
        else:
            _, kind, t, c, m = it
            if cur_slab is not None and kind != "DIAG":
                # non-diagonal targets must be slab-resident
                assert set(t) <= cur_slab, (kind, t, sorted(cur_slab))
            stats["ops"] += 1
            if kind == "DIAG" and len(t) > ORACLE_MAX_DIAG:
                apply_wide_diag(state, n, t, c, m)
            else:
                oracle.apply_circuit(n, [op_gate(kind, t, c, m)], state)
    return layout, stats


def to_logical(state_phys, n, layout):
    """state_phys[x_phys] with logical qubit q at physical bit layout[q] -> logical order."""
    idx = np.arange(1 << n)
    phys_index = np.zeros_like(idx)
    for q in range(n):
        phys_index |= ((idx >> q) & 1) << layout[q]
    return state_phys[phys_index]
