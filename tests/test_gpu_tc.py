"""Tensor-core path (complex64, BF16x3 and TF32x3 split products, FP32 accumulate, 6- and
7-qubit fused blocks) against the FP64 oracle.

The bar is infidelity <= 1e-6 (1 - |<psi_oracle|psi>|^2 / (|psi_oracle|^2 |psi|^2)); the largest
amplitude error is reported and held to the complex64 tolerance of 1e-5.
"""
import numpy as np
import pytest

import oracle
from paper_2406_14084_gb300 import qs
from paper_2406_14084_gb300 import workloads as W
from paper_2406_14084_gb300.workloads import Gate

pytestmark = pytest.mark.gpu


def rand_state(n, seed):
    rng = np.random.default_rng(seed)
    v = rng.normal(size=1 << n) + 1j * rng.normal(size=1 << n)
    return v / np.linalg.norm(v)


def infidelity(a, b):
    return 1.0 - abs(np.vdot(a, b)) ** 2 / (np.vdot(a, a).real * np.vdot(b, b).real)


def run_tc(n, gates, init, mode=qs.QS_TC_BF16X3, width=6):
    s = qs.State(n, qs.QS_C64)
    try:
        qs.qs_copy_from_host(s.h, init.astype(np.complex64))
        s.apply(gates, qs.options(tc=mode, dtype=qs.QS_C64, tc_width=width))
        st = qs.qs_stats(s.h)
        return s.amplitudes().astype(np.complex128), st
    finally:
        s.close()


@pytest.mark.parametrize("targets", [(0, 1, 2, 3, 4, 5), (13, 2, 9, 0, 7, 4), (15, 14, 12, 11, 10, 8)])
def test_single_six_qubit_unitary(targets):
    n = 16
    U = W.random_unitary(6, sum(targets))
    gates = [Gate("UNITARY", targets, (), (), U)]
    init = rand_state(n, 3)
    want = oracle.apply_circuit(n, gates, init.copy())
    got, st = run_tc(n, gates, init)
    assert st["tc_gates"] == 1
    assert infidelity(want, got) <= 1e-6
    assert np.max(np.abs(got - want)) <= 1e-5


@pytest.mark.parametrize("n,depth", [(14, 6), (17, 8)])
def test_layered_circuit_on_tensor_cores(n, depth):
    gates = W.layered(n, depth, 1003)
    init = oracle.basis_state(n, 0)
    want = oracle.apply_circuit(n, gates, init.copy())
    got, st = run_tc(n, gates, init)
    assert st["tc_gates"] > 0
    assert infidelity(want, got) <= 1e-6
    assert np.max(np.abs(got - want)) <= 1e-5


def test_mixed_circuit_tc_and_simt_steps():
    n = 15
    gates = W.random_circuit(n, 150, 77, ["H", "T", "RZ", "U3", "CX", "CZ", "SWAP", "RY"]) + W.qft(n)
    init = rand_state(n, 9)
    want = oracle.apply_circuit(n, gates, init.copy())
    got, st = run_tc(n, gates, init)
    assert st["tc_gates"] > 0
    assert infidelity(want, got) <= 1e-6
    assert np.max(np.abs(got - want)) <= 1e-5


def test_layered_24_qubits_on_tensor_cores():
    """A 24-qubit state (128 MiB complex64, larger than L2): many slabs per tensor-core launch,
    targets spread over all 24 qubits."""
    n = 24
    gates = W.layered(n, 6, 1003)
    init = oracle.basis_state(n, 0x5A5A5A)
    want = oracle.apply_circuit(n, gates, init.copy())
    got, st = run_tc(n, gates, init)
    assert st["tc_gates"] >= 4
    assert infidelity(want, got) <= 1e-6
    assert np.max(np.abs(got - want)) <= 1e-5


@pytest.mark.parametrize("targets", [(0, 1, 2, 3, 4, 5), (13, 2, 9, 0, 7, 4)])
def test_tf32x3_single_unitary(targets):
    """TF32 x 3 mode: two K halves per slab, E half-images loaded per half."""
    n = 16
    U = W.random_unitary(6, 7 + sum(targets))
    gates = [Gate("UNITARY", targets, (), (), U)]
    init = rand_state(n, 4)
    want = oracle.apply_circuit(n, gates, init.copy())
    s = qs.State(n, qs.QS_C64)
    try:
        qs.qs_copy_from_host(s.h, init.astype(np.complex64))
        s.apply(gates, qs.options(tc=qs.QS_TC_TF32X3, dtype=qs.QS_C64))
        assert qs.qs_stats(s.h)["tc_gates"] == 1
        got = s.amplitudes().astype(np.complex128)
    finally:
        s.close()
    assert infidelity(want, got) <= 1e-6
    # TF32 parts carry more bits than BF16 ones: the error is at the complex64 rounding level
    assert np.max(np.abs(got - want)) <= 2e-6


@pytest.mark.parametrize("n,depth", [(17, 8), (24, 4)])
def test_tf32x3_layered_against_oracle(n, depth):
    gates = W.layered(n, depth, 1003)
    init = oracle.basis_state(n, 0)
    want = oracle.apply_circuit(n, gates, init.copy())
    s = qs.State(n, qs.QS_C64)
    try:
        s.apply(gates, qs.options(tc=qs.QS_TC_TF32X3, dtype=qs.QS_C64))
        assert qs.qs_stats(s.h)["tc_gates"] > 0
        got = s.amplitudes().astype(np.complex128)
    finally:
        s.close()
    assert infidelity(want, got) <= 1e-6
    assert np.max(np.abs(got - want)) <= 1e-5


MODES = [qs.QS_TC_BF16X3, qs.QS_TC_TF32X3]


@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("targets", [(0, 1, 2, 3, 4, 5, 6), (13, 2, 9, 0, 7, 4, 11), (15, 14, 12, 11, 10, 8, 1),
                                     (6, 5, 4, 3, 2, 1, 0)])
def test_single_seven_qubit_unitary(targets, mode):
    """A 7-qubit gate: four 64x64 blocks (one per value pair of the 7th target bit) multiplied
    into four accumulators and combined; the 7th target is a low bit, a middle bit or the top."""
    n = 16
    U = W.random_unitary(7, 31 + sum(targets))
    gates = [Gate("UNITARY", targets, (), (), U)]
    init = rand_state(n, 5)
    want = oracle.apply_circuit(n, gates, init.copy())
    got, st = run_tc(n, gates, init, mode, 7)
    assert st["tc_gates"] == 1
    assert infidelity(want, got) <= 1e-6
    assert np.max(np.abs(got - want)) <= (1e-5 if mode == qs.QS_TC_BF16X3 else 2e-6)


@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("n,depth", [(17, 8), (24, 4)])
def test_layered_with_seven_qubit_blocks(n, depth, mode):
    gates = W.layered(n, depth, 1003)
    init = oracle.basis_state(n, 0x15A5A & ((1 << n) - 1))
    want = oracle.apply_circuit(n, gates, init.copy())
    got, st = run_tc(n, gates, init, mode, 7)
    assert st["tc_gates"] > 0
    assert infidelity(want, got) <= 1e-6
    assert np.max(np.abs(got - want)) <= 1e-5


def test_seven_and_six_qubit_steps_in_one_plan():
    """A circuit whose fusion leaves 7-qubit blocks, narrower blocks padded to 6 and SIMT steps."""
    n = 15
    gates = W.random_circuit(n, 150, 78, ["H", "T", "RZ", "U3", "CX", "CZ", "SWAP", "RY"]) + W.qft(n)
    gates += [Gate("UNITARY", (3, 9, 14, 0, 6), (), (), W.random_unitary(5, 5))]
    init = rand_state(n, 10)
    want = oracle.apply_circuit(n, gates, init.copy())
    p = qs.qs_fuse(gates, n, qs.options(tc=qs.QS_TC_BF16X3, dtype=qs.QS_C64, tc_width=7))
    try:
        widths = [int(l.split()[2]) for l in qs.qs_plan_dump(p).splitlines() if l.startswith("OP DENSE")]
    finally:
        qs.qs_plan_destroy(p)
    assert 7 in widths and 6 in widths
    got, st = run_tc(n, gates, init, qs.QS_TC_BF16X3, 7)
    assert infidelity(want, got) <= 1e-6
    assert np.max(np.abs(got - want)) <= 1e-5


@pytest.mark.parametrize("n", [20, 21, 22])
def test_pipelined_slab_counts(n):
    """BF16x3 6-qubit gates in the usual layout run a two-slab pipeline per CTA; 20, 21 and 22
    qubits give CTAs 0-1, 1-2 and 3-4 slabs (152 CTAs), the pipeline's short cases."""
    gates = W.layered(n, 4, 1005)
    init = rand_state(n, 11)
    want = oracle.apply_circuit(n, gates, init.copy())
    got, st = run_tc(n, gates, init)
    assert st["tc_gates"] > 0
    assert infidelity(want, got) <= 1e-6
    assert np.max(np.abs(got - want)) <= 1e-5
