"""Complex128 register stages in double-float arithmetic (QS_ARITH_DF) against the FP64 oracle.

The state stays complex128 in HBM; each pass of register stages converts its slab to pairs of
FP32 numbers (about 48 significant bits) and back.  The bar is the complex128 tolerance of the
FP64 path, max |delta amp| <= 1e-12, on circuits with every gate kind, on deep layered circuits
and the QFT, and at full size (32 qubits, U then U^-1).
"""
import numpy as np
import pytest

import oracle
from paper_2406_14084_gb300 import qs
from paper_2406_14084_gb300 import workloads as W
from paper_2406_14084_gb300.workloads import Gate

pytestmark = pytest.mark.gpu

ALL = ["H", "X", "Y", "Z", "S", "SDG", "T", "TDG", "RX", "RY", "RZ", "P", "U3", "CX", "CZ",
       "CP", "SWAP", "RZZ"]


def run_df(n, gates, x0=0, **kw):
    with qs.State(n, qs.QS_C128) as s:
        s.set_basis(x0)
        s.apply(gates, qs.options(dtype=qs.QS_C128, arith=qs.QS_ARITH_DF, **kw))
        return s.amplitudes()


@pytest.mark.parametrize("n,seed", [(9, 1), (14, 2), (18, 3)])
def test_random_circuits_all_kinds(n, seed):
    gates = W.random_circuit(n, 300, 7000 + seed, ALL)
    want = oracle.apply_circuit(n, gates)
    got = run_df(n, gates)
    assert np.max(np.abs(got - want)) <= 1e-12


@pytest.mark.parametrize("fuse", [1, 2, 5])
def test_fused_and_controlled_gates(fuse):
    n = 16
    gates = W.random_circuit(n, 200, 7100 + fuse, ALL)
    gates += [Gate("U3", (3,), (7, 11), (0.3, 0.9, 1.7)), Gate("RY", (12,), (0,), (2.2,))]
    gates += W.layered(n, 3, 7200 + fuse)
    want = oracle.apply_circuit(n, gates)
    got = run_df(n, gates, fuse_width=fuse)
    assert np.max(np.abs(got - want)) <= 1e-12


def test_deep_layered_and_qft():
    n = 20
    gates = W.layered(n, 40, 1002) + W.qft(n)
    x0 = 0x5A5A5 & ((1 << n) - 1)
    want = oracle.apply_circuit(n, gates, oracle.basis_state(n, x0))
    got = run_df(n, gates, x0=x0)
    assert np.max(np.abs(got - want)) <= 1e-12
    assert abs(np.vdot(got, got).real - 1.0) <= 1e-12


def test_small_states_and_stage_widths():
    for n in (1, 2, 5, 12, 13):
        gates = W.random_circuit(n, 60, 7300 + n, ALL) if n > 1 else [Gate("U3", (0,), (), (0.4, 0.2, 0.1))]
        want = oracle.apply_circuit(n, gates)
        for rb in (3, 4):
            got = run_df(n, gates, stage_bits=rb)
            assert np.max(np.abs(got - want)) <= 1e-12, (n, rb)


def test_fp64_and_df_plans_agree_on_readouts():
    n = 19
    gates = W.layered(n, 12, 77)
    H = W.zz_chain_hamiltonian(n)
    with qs.State(n, qs.QS_C128) as a, qs.State(n, qs.QS_C128) as b:
        a.apply(gates, qs.options(dtype=qs.QS_C128))
        b.apply(gates, qs.options(dtype=qs.QS_C128, arith=qs.QS_ARITH_DF))
        assert abs(a.expect(H) - b.expect(H)) <= 1e-9 * n
        assert np.max(np.abs(a.probs([0, 7, 18]) - b.probs([0, 7, 18]))) <= 1e-12


def free_gib():
    import torch

    free, _ = torch.cuda.mem_get_info()
    return free / 2**30


def test_layered32_df_inverse_returns_basis_state():
    n = 32
    if free_gib() < 70:
        pytest.skip("needs 64 GiB of free device memory")
    g = W.layered(n, 40, 1002)
    inv = []
    for x in reversed(g):
        if x.kind == "U3":
            t, p, l = x.params
            inv.append(Gate("U3", x.targets, (), (-t, -l, -p)))
        else:
            inv.append(x)
    x0 = 0x9C3A5A17 & ((1 << n) - 1)
    opts = qs.options(dtype=qs.QS_C128, arith=qs.QS_ARITH_DF)
    with qs.State(n, qs.QS_C128) as s:
        s.set_basis(x0)
        s.apply(g, opts)
        assert abs(s.norm2() - 1.0) <= 1e-12
        s.apply(inv, opts)
        a = qs.qs_copy_to_host(s.h, n, qs.QS_C128, x0, 1)[0]
        assert abs(a - 1.0) <= 1e-10, a
