"""Circuit text I/O in the paper's formats (artifact appendix of arXiv 2406.14084).

Raw circuits: one gate per line, ``<gate type> <target qubits...> <gate ID> [parameters...]``;
``#`` starts a comment.  Controlled kinds list the control first (``CX c t``).  Parameters are
angles in radians (RX/RY/RZ/P/CP/RZZ one, U3 three); a missing angle is read as the gate ID
when ``angle_from_id`` is set (the worked example prints no RZZ angles and its fused values
equal cos of the IDs).

Optimized listings (``plan_listing``): the plan's steps in order, on physical positions --
``SQS k o1..ok i1..ik`` for an in-memory swap (remap pass, Alg. 4) exchanging positions o_j and
i_j, ``D<k> t1..tk d...`` for a diagonal table, ``U<k> t1..tk m...`` for a dense unitary
(row-major, re im pairs), ``X t`` / ``SWAP a b`` for relabels, each with ``C c...`` controls when
present, and a final ``LAYOUT`` line (physical position of each logical qubit).
"""
from __future__ import annotations

from . import qs
from .workloads import Gate

ONE_QUBIT = {"H", "X", "Y", "Z", "S", "T", "SDG", "TDG", "RX", "RY", "RZ", "P", "U3"}
TWO_QUBIT = {"CX", "CZ", "CP", "SWAP", "RZZ"}
N_ANGLES = {"RX": 1, "RY": 1, "RZ": 1, "P": 1, "CP": 1, "RZZ": 1, "U3": 3}


def parse_circuit(text: str, angle_from_id: bool = False):
    """Returns (n, gates, ids): n = 1 + the largest qubit index used."""
    gates, ids, nq = [], [], 0
    for lineno, line in enumerate(text.splitlines(), 1):
        line = line.split("#", 1)[0].strip()
        if not line:
            continue
        f = line.split()
        kind = f[0].upper()
        if kind in ONE_QUBIT:
            nt = 1
        elif kind in TWO_QUBIT:
            nt = 2
        else:
            raise ValueError(f"line {lineno}: unknown gate type {f[0]!r}")
        if len(f) < nt + 1:
            raise ValueError(f"line {lineno}: expected {nt} qubits and an ID")
        qubits = tuple(int(v) for v in f[1:1 + nt])
        gid = int(f[1 + nt]) if len(f) > 1 + nt else len(gates)
        params = tuple(float(v) for v in f[2 + nt:])
        need = N_ANGLES.get(kind, 0)
        if len(params) < need:
            if angle_from_id and need == 1 and not params:
                params = (float(gid),)
            else:
                raise ValueError(f"line {lineno}: {kind} needs {need} angle(s)")
        params = params[:need]
        if kind == "CX":
            g = Gate("CX", (qubits[1],), (qubits[0],), params)
        else:
            g = Gate(kind, qubits, (), params)
        if len(set(qubits)) != len(qubits) or min(qubits) < 0:
            raise ValueError(f"line {lineno}: bad qubits")
        nq = max(nq, max(qubits) + 1)
        gates.append(g)
        ids.append(gid)
    return nq, gates, ids


def write_circuit(gates, ids=None) -> str:
    """Inverse of parse_circuit for the kinds it reads."""
    out = []
    for i, g in enumerate(gates):
        gid = ids[i] if ids is not None else i
        if g.kind == "CX":
            qubits = (g.controls[0], g.targets[0])
        elif g.controls:
            raise ValueError("only CX may carry a control in the text format")
        else:
            qubits = g.targets
        parts = [g.kind] + [str(q) for q in qubits] + [str(gid)] + [repr(float(p)) for p in g.params]
        out.append(" ".join(parts))
    return "\n".join(out) + "\n"


def plan_listing(plan) -> str:
    """The plan as an optimized listing on physical positions (see module docstring)."""
    lines = []
    for row in qs.qs_plan_dump(plan).splitlines():
        f = row.split()
        if not f:
            continue
        if f[0] == "REMAP":
            k = int(f[1])
            lines.append("SQS " + " ".join(f[1:2 + 2 * k]))
        elif f[0] == "OP":
            kind, k = f[1], int(f[2])
            ti, ci, mi = f.index("t"), f.index("c"), f.index("m") if "m" in f else len(f)
            t, c, m = f[ti + 1:ci], f[ci + 1:mi], f[mi + 1:]
            ctl = (" C " + " ".join(c)) if c else ""
            if kind == "DENSE":
                lines.append(f"U{k} " + " ".join(t) + ctl + " " + " ".join(m))
            elif kind == "DIAG":
                lines.append(f"D{len(t)} " + " ".join(t) + ctl + " " + " ".join(m))
            elif kind == "PERMX":
                lines.append("X " + " ".join(t) + ctl)
            elif kind == "SWAP":
                lines.append("SWAP " + " ".join(t) + ctl)
            elif kind == "PHASE":
                lines.append("PHASE" + ctl + " " + " ".join(m))
            else:
                raise ValueError(f"unknown op {kind}")
        elif f[0] == "LAYOUT":
            lines.append(row)
    return "\n".join(lines) + "\n"
