"""Batched persistent launch: per-circuit <H> against the FP64 oracle.

H = sum_i Z_i + 0.5 sum_i Z_i Z_{i+1} (open chain), circuits = hardware-efficient ansatz
(RY layer, RZ layer, CX ladder) x L with uneven qubit counts and depths.  Tolerance on <H>:
1e-9 * n for complex128, 1e-4 * n for complex64.
"""
import numpy as np
import pytest

import oracle
from paper_2406_14084_gb300 import qs
from paper_2406_14084_gb300 import workloads as W

pytestmark = pytest.mark.gpu

NMAX = 24
H_TERMS = W.zz_chain_hamiltonian(NMAX)  # terms on qubits >= n are dropped per circuit


def oracle_expect(circuits):
    out = []
    for n, gates in circuits:
        a = oracle.apply_circuit(n, gates)
        out.append(oracle.expect_pauli(a, n, W.zz_chain_hamiltonian(n)).real)
    return np.array(out)


@pytest.mark.parametrize("dtype", [qs.QS_C64, qs.QS_C128])
@pytest.mark.parametrize("graph", [0, 1])
def test_batch_matches_oracle(dtype, graph):
    circuits = W.vqe_batch(24, 4004, nmin=10, nmax=17, lmin=1, lmax=4)
    want = oracle_expect(circuits)
    b = qs.qs_batch_create(circuits, qs.options(dtype=dtype, graph=graph))
    try:
        info = qs.qs_batch_info_get(b)
        assert info["circuits"] == len(circuits) and info["items"] >= len(circuits)
        for rep in range(2):  # second run replays the graph / relaunches from scratch
            got = qs.qs_apply_batch(b, H_TERMS, len(circuits))
            ns = np.array([c[0] for c in circuits])
            tol = (1e-9 if dtype == qs.QS_C128 else 1e-4) * ns
            assert np.all(np.abs(got - want) <= tol), np.max(np.abs(got - want))
    finally:
        qs.qs_batch_destroy(b)


@pytest.mark.parametrize("dtype", [qs.QS_C64, qs.QS_C128])
def test_batch_full_range_circuits_match_oracle(dtype):
    """The batch configuration's extremes: circuits of up to 24 qubits and 12 layers (slabs run
    multi-pass with the most items per pass) mixed with small ones, on the graph path."""
    shapes = [(24, 12, 71), (24, 7, 72), (22, 12, 73), (20, 2, 74), (17, 12, 75), (13, 9, 76),
              (11, 12, 77), (10, 2, 78)]
    circuits = [(n, W.vqe_circuit(n, L, seed)) for n, L, seed in shapes]
    want = oracle_expect(circuits)
    b = qs.qs_batch_create(circuits, qs.options(dtype=dtype, graph=1))
    try:
        info = qs.qs_batch_info_get(b)
        assert info["rounds"] >= 2
        for _ in range(2):
            got = qs.qs_apply_batch(b, H_TERMS, len(circuits))
            ns = np.array([c[0] for c in circuits])
            tol = (1e-9 if dtype == qs.QS_C128 else 1e-4) * ns
            assert np.all(np.abs(got - want) <= tol), np.max(np.abs(got - want))
    finally:
        qs.qs_batch_destroy(b)


def test_batch_small_slab_forces_multipass_and_tuner():
    circuits = W.vqe_batch(12, 99, nmin=12, nmax=16, lmin=2, lmax=3)
    want = oracle_expect(circuits)
    b = qs.qs_batch_create(circuits, qs.options(dtype=qs.QS_C64, slab_bits=11, graph=1))
    try:
        info = qs.qs_batch_info_get(b)
        assert info["rounds"] >= 2
        got = qs.qs_apply_batch(b, H_TERMS, len(circuits))
        assert np.max(np.abs(got - want)) <= 1e-4 * 16
        chosen = qs.qs_batch_tune(b, H_TERMS)
        assert chosen in (11, 12, 13)
        got = qs.qs_apply_batch(b, H_TERMS, len(circuits))
        assert np.max(np.abs(got - want)) <= 1e-4 * 16
    finally:
        qs.qs_batch_destroy(b)


def test_batch_rejects_x_terms_and_bad_input():
    circuits = W.vqe_batch(2, 5, nmin=10, nmax=11, lmin=1, lmax=1)
    b = qs.qs_batch_create(circuits, qs.options())
    try:
        with pytest.raises(qs.QsError) as e:
            qs.qs_apply_batch(b, [(1.0, 1, 0)], 2)
        assert e.value.status == qs.QS_EUNSUPPORTED
    finally:
        qs.qs_batch_destroy(b)
    with pytest.raises(qs.QsError):
        qs.qs_batch_create([(40, [])], qs.options())
