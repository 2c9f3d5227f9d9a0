"""Seeded synthetic circuits shaped like the paper's benchmark workloads.

This module holds no simulation arithmetic: it only draws gate lists (kinds, qubits and
angles) from a counter-based generator, so that the CUDA path and the FP64 oracle can be fed
identical inputs.  It imports nothing else from the package.

Random numbers come from SplitMix64 (Steele, Lea & Flood, "Fast splittable pseudorandom
number generators", OOPSLA 2014): state += 0x9E3779B97F4A7C15, then two xor-shift-multiply
rounds; a double in [0, 1) is the top 53 bits times 2^-53.

Workload shapes (arXiv 2406.14084, Sec. VI-A, Tables 1-2; the generator files the paper used
are not available, these synthetic circuits stand in for them):
  * ``random_circuit``: uniform draws over a gate alphabet with uniform distinct targets;
  * ``qft``: the quantum Fourier transform without the final swap layer (the paper's 31-qubit
    QFT has 496 gates = 31 H + 465 CP, Table 2);
  * ``layered``: a U3 layer on every qubit, then CZ on alternating neighbour pairs;
  * ``vqe_circuit``: hardware-efficient ansatz (RY layer, RZ layer, CX ladder) repeated L times;
  * ``qaoa_like``: H layer, RZZ on ring edges, RX mixer, p rounds (QAOA shape of Table 2);
  * ``gate_sweep``: one gate kind applied to every qubit, ``reps`` times (Table 1 benchmark).
"""
from __future__ import annotations

import math
from typing import NamedTuple, Optional, Sequence

import numpy as np

MASK64 = (1 << 64) - 1
TWO_PI = 2.0 * math.pi


class Gate(NamedTuple):
    kind: str
    targets: tuple
    controls: tuple = ()
    params: tuple = ()
    matrix: Optional[np.ndarray] = None


class SplitMix64:
    def __init__(self, seed: int):
        self.state = seed & MASK64

    def next_u64(self) -> int:
        self.state = (self.state + 0x9E3779B97F4A7C15) & MASK64
        z = self.state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK64
        return z ^ (z >> 31)

    def uniform(self) -> float:
        return (self.next_u64() >> 11) * (1.0 / 9007199254740992.0)

    def below(self, m: int) -> int:
        """Integer uniform in [0, m) (multiply-shift; bias < 2^-40 for the sizes used here)."""
        return (self.next_u64() * m) >> 64

    def angle(self) -> float:
        return TWO_PI * self.uniform()

    def distinct(self, n: int, k: int) -> list:
        out = []
        while len(out) < k:
            q = self.below(n)
            if q not in out:
                out.append(q)
        return out


# ----------------------------------------------------------------------------- circuits

CONFIG1_ALPHABET = ("H", "X", "S", "T", "RZ", "U3", "CX", "CZ", "SWAP")


def random_circuit(n: int, ngates: int, seed: int, alphabet: Sequence[str] = CONFIG1_ALPHABET):
    """Gates drawn uniformly from ``alphabet``; qubits uniform and distinct within a gate."""
    rng = SplitMix64(seed)
    gates = []
    for _ in range(ngates):
        kind = alphabet[rng.below(len(alphabet))]
        if kind in ("H", "X", "Y", "Z", "S", "SDG", "T", "TDG"):
            gates.append(Gate(kind, (rng.below(n),)))
        elif kind in ("RX", "RY", "RZ", "P"):
            gates.append(Gate(kind, (rng.below(n),), (), (rng.angle(),)))
        elif kind == "U3":
            q = rng.below(n)
            gates.append(Gate(kind, (q,), (), (rng.angle(), rng.angle(), rng.angle())))
        elif kind == "CX":
            c, t = rng.distinct(n, 2)
            gates.append(Gate("CX", (t,), (c,)))
        elif kind in ("CZ", "SWAP"):
            a, b = rng.distinct(n, 2)
            gates.append(Gate(kind, (a, b)))
        elif kind in ("CP", "RZZ"):
            a, b = rng.distinct(n, 2)
            gates.append(Gate(kind, (a, b), (), (rng.angle(),)))
        else:
            raise ValueError(kind)
    return gates


def qft(n: int):
    """QFT without final swaps: for j = n-1 .. 0: H(j), then CP(pi / 2^(j-i)) on (i, j), i < j."""
    gates = []
    for j in range(n - 1, -1, -1):
        gates.append(Gate("H", (j,)))
        for i in range(j - 1, -1, -1):
            gates.append(Gate("CP", (i, j), (), (math.pi / (1 << (j - i)),)))
    return gates


def random_basis(n: int, seed: int) -> int:
    return SplitMix64(seed).next_u64() & ((1 << n) - 1)


def layered(n: int, depth: int, seed: int):
    """``depth`` layers of (U3 on every qubit; CZ on (0,1),(2,3),.. for even layers and on
    (1,2),(3,4),.. for odd layers)."""
    rng = SplitMix64(seed)
    gates = []
    for layer in range(depth):
        for q in range(n):
            gates.append(Gate("U3", (q,), (), (rng.angle(), rng.angle(), rng.angle())))
        for a in range(layer % 2, n - 1, 2):
            gates.append(Gate("CZ", (a, a + 1)))
    return gates


def vqe_circuit(n: int, L: int, seed: int):
    """Hardware-efficient ansatz: L x (RY on all, RZ on all, CX ladder 0->1->..->n-1)."""
    rng = SplitMix64(seed)
    gates = []
    for _ in range(L):
        for q in range(n):
            gates.append(Gate("RY", (q,), (), (rng.angle(),)))
        for q in range(n):
            gates.append(Gate("RZ", (q,), (), (rng.angle(),)))
        for q in range(n - 1):
            gates.append(Gate("CX", (q + 1,), (q,)))
    return gates


def vqe_batch(count: int, seed: int, nmin: int = 10, nmax: int = 24, lmin: int = 2, lmax: int = 12):
    """``count`` circuits with n ~ U{nmin..nmax}, L ~ U{lmin..lmax}; returns [(n, gates)]."""
    rng = SplitMix64(seed)
    out = []
    for i in range(count):
        n = nmin + rng.below(nmax - nmin + 1)
        L = lmin + rng.below(lmax - lmin + 1)
        sub = rng.next_u64()
        out.append((n, vqe_circuit(n, L, sub)))
    return out


def zz_chain_hamiltonian(n: int):
    """H = sum_i Z_i + 0.5 sum_{i<n-1} Z_i Z_{i+1} as (coeff, xmask, zmask) terms (open chain)."""
    terms = [(1.0, 0, 1 << i) for i in range(n)]
    terms += [(0.5, 0, (1 << i) | (1 << (i + 1))) for i in range(n - 1)]
    return terms


def qaoa_like(n: int, p: int, seed: int):
    """QAOA-shaped circuit: H on all; p rounds of RZZ on ring edges (i, i+1 mod n) and RX."""
    rng = SplitMix64(seed)
    gates = [Gate("H", (q,)) for q in range(n)]
    for _ in range(p):
        gamma, beta = rng.angle(), rng.angle()
        for i in range(n):
            gates.append(Gate("RZZ", (i, (i + 1) % n), (), (gamma,)))
        for q in range(n):
            gates.append(Gate("RX", (q,), (), (beta,)))
    return gates


def qaoa_complete(n: int, p: int, seed: int):
    """QAOA on the complete graph: H on all; p rounds of RZZ on every pair (i < j) and RX on all.
    n + p (n (n - 1) / 2 + n) gates: 2,511 for n = 31, p = 5 (the paper's QAOA size)."""
    rng = SplitMix64(seed)
    gates = [Gate("H", (q,)) for q in range(n)]
    for _ in range(p):
        gamma, beta = rng.angle(), rng.angle()
        for i in range(n):
            for j in range(i + 1, n):
                gates.append(Gate("RZZ", (i, j), (), (gamma,)))
        for q in range(n):
            gates.append(Gate("RX", (q,), (), (beta,)))
    return gates


def gate_sweep(n: int, kind: str, reps: int, seed: int):
    """``kind`` applied to every qubit ``reps`` times (two-qubit kinds on (q, q+1 mod n))."""
    rng = SplitMix64(seed)
    gates = []
    for _ in range(reps):
        for q in range(n):
            r = (q + 1) % n
            if kind in ("H", "X", "Y", "Z", "S", "T"):
                gates.append(Gate(kind, (q,)))
            elif kind in ("RX", "RY", "RZ", "P"):
                gates.append(Gate(kind, (q,), (), (rng.angle(),)))
            elif kind == "U3":
                gates.append(Gate(kind, (q,), (), (rng.angle(), rng.angle(), rng.angle())))
            elif kind == "CX":
                gates.append(Gate("CX", (r,), (q,)))
            elif kind in ("CZ", "SWAP"):
                gates.append(Gate(kind, (q, r)))
            elif kind in ("CP", "RZZ"):
                gates.append(Gate(kind, (q, r), (), (rng.angle(),)))
            else:
                raise ValueError(kind)
    return gates


def random_unitary(k: int, seed: int) -> np.ndarray:
    """Haar-ish random 2^k x 2^k unitary: QR of a complex Gaussian matrix (seeded draws)."""
    rng = SplitMix64(seed)
    d = 1 << k
    u = np.array([[rng.uniform() for _ in range(2 * d)] for _ in range(d)])
    # Box-Muller on pairs of uniforms
    u1, u2 = np.clip(u[:, 0::2], 1e-300, 1.0), u[:, 1::2]
    r = np.sqrt(-2.0 * np.log(u1))
    z = r * np.cos(TWO_PI * u2) + 1j * r * np.sin(TWO_PI * u2)
    q, rr = np.linalg.qr(z)
    ph = np.diag(rr) / np.abs(np.diag(rr))
    return q * ph[None, :]


def random_diag(k: int, seed: int) -> np.ndarray:
    rng = SplitMix64(seed)
    return np.array([np.exp(1j * rng.angle()) for _ in range(1 << k)])
