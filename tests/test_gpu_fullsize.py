"""Parity at the benchmark's full sizes, in the bench's launch configuration (default options).

A full state is too large for the oracle, so these checks use properties that hold at any
size:
- the no-swap QFT of a basis state |x> (32 qubits, complex128, 64 GiB) has the closed form
  a(y) = 2^{-n/2} exp(2 pi i x rev(y) / 2^n), compared on sampled runs of amplitudes
  (the same closed form pins the oracle);
- a layered circuit followed by its inverse (32 qubits complex128, 64 GiB; 34 qubits complex64,
  128 GiB) returns the basis state it started from, the norm is preserved, and the marginal
  probabilities of sampled qubits are those of the basis state.
"""
import math

import numpy as np
import pytest

from paper_2406_14084_gb300 import qs
from paper_2406_14084_gb300 import workloads as W
from paper_2406_14084_gb300.workloads import Gate

pytestmark = pytest.mark.gpu


def free_gib():
    import torch

    free, _ = torch.cuda.mem_get_info()
    return free / 2**30


def bitrev(v, n):
    return int(format(v, f"0{n}b")[::-1], 2)


def test_qft32_complex128_closed_form_sampled():
    n = 32
    if free_gib() < 70:
        pytest.skip("needs 64 GiB of free device memory")
    x = W.random_basis(n, 1002)
    s = qs.State(n, qs.QS_C128)
    try:
        s.set_basis(x)
        s.apply(W.qft(n), qs.options(dtype=qs.QS_C128))
        assert abs(s.norm2() - 1.0) <= 1e-12
        rng = np.random.default_rng(5)
        starts = [0, (1 << n) - 512] + [int(v) * 512 for v in rng.integers(0, (1 << n) // 512, size=14)]
        worst = 0.0
        for first in starts:
            got = qs.qs_copy_to_host(s.h, n, qs.QS_C128, first, 512)
            y = np.arange(first, first + 512, dtype=np.int64)
            rev = np.array([bitrev(int(v), n) for v in y], dtype=np.float64)
            # x * rev(y) mod 2^n keeps the phase argument exact in FP64
            ph = np.array([(x * int(r)) % (1 << n) for r in rev], dtype=np.float64)
            want = 2.0 ** (-n / 2) * np.exp(2j * np.pi * ph / (1 << n))
            worst = max(worst, float(np.max(np.abs(got - want))))
        assert worst <= 1e-12, worst
    finally:
        s.close()


def inverse_layered(gates):
    """U3(t, p, l)^-1 = U3(-t, -l, -p); CZ is its own inverse."""
    out = []
    for g in reversed(gates):
        if g.kind == "U3":
            t, p, l = g.params
            out.append(Gate("U3", g.targets, (), (-t, -l, -p)))
        else:
            out.append(g)
    return out


def test_layered34_complex64_inverse_returns_basis_state():
    n = 34
    if free_gib() < 135:
        pytest.skip("needs 128 GiB of free device memory")
    g = W.layered(n, 40, 1002)
    x0 = 0x2A5A5A5A5 & ((1 << n) - 1)
    s = qs.State(n, qs.QS_C64)
    try:
        s.set_basis(x0)
        s.apply(g, qs.options(dtype=qs.QS_C64))
        assert abs(s.norm2() - 1.0) <= 1e-4
        s.apply(inverse_layered(g), qs.options(dtype=qs.QS_C64))
        a = qs.qs_copy_to_host(s.h, n, qs.QS_C64, x0, 1)[0]
        assert abs(abs(a) - 1.0) <= 1e-4, a
        # the global phase of U^-1 U is 1 up to rounding
        assert abs(a - 1.0) <= 1e-4, a
        p = s.probs([0, 33, 17])
        want = np.zeros(8)
        want[(x0 & 1) | ((x0 >> 33) & 1) << 1 | ((x0 >> 17) & 1) << 2] = 1.0
        assert np.max(np.abs(p - want)) <= 2e-4
    finally:
        s.close()


def test_layered32_complex128_inverse_returns_basis_state():
    """The 32-qubit complex128 layered circuit of depth 40 with the bench's default options, then
    its inverse: back to the start state within 1e-10 (the complex128 amplitude bar is 1e-12
    per amplitude for one circuit; U then U^-1 doubles the rounding)."""
    n = 32
    if free_gib() < 70:
        pytest.skip("needs 64 GiB of free device memory")
    g = W.layered(n, 40, 1002)
    x0 = 0x9C3A5A17 & ((1 << n) - 1)
    s = qs.State(n, qs.QS_C128)
    try:
        s.set_basis(x0)
        s.apply(g, qs.options(dtype=qs.QS_C128))
        assert abs(s.norm2() - 1.0) <= 1e-12
        mid = s.probs([0, 31, 16, 7])
        assert abs(mid.sum() - 1.0) <= 1e-12 and np.all(mid >= 0)
        s.apply(inverse_layered(g), qs.options(dtype=qs.QS_C128))
        assert abs(s.norm2() - 1.0) <= 1e-12
        a = qs.qs_copy_to_host(s.h, n, qs.QS_C128, x0, 1)[0]
        assert abs(a - 1.0) <= 1e-10, a
        rng = np.random.default_rng(3)
        for _ in range(3):
            qubits = [int(q) for q in rng.choice(n, size=5, replace=False)]
            p = s.probs(qubits)
            want = np.zeros(32)
            want[sum(((x0 >> q) & 1) << j for j, q in enumerate(qubits))] = 1.0
            assert np.max(np.abs(p - want)) <= 1e-10
        # amplitudes around the start state are zero
        near = qs.qs_copy_to_host(s.h, n, qs.QS_C128, (x0 & ~511), 512)
        near[x0 & 511] = 0.0
        assert np.max(np.abs(near)) <= 1e-10
    finally:
        s.close()
