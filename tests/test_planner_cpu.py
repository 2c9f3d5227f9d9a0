"""Host-side tests of the C-ABI library that need no GPU: symbol exports, argument validation,
and the planner, whose listings (qs_plan_dump) are replayed on the FP64 oracle and compared
with the unfused circuit (fusion products, diagonal tables, slab residency, remaps, relabels).
"""
import os
import re

import numpy as np
import pytest

import oracle
from paper_2406_14084_gb300 import qs
from paper_2406_14084_gb300 import workloads as W
from paper_2406_14084_gb300.workloads import Gate

import plan_replay as PR
from plan_replay import replay, to_logical

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
GOLD = os.path.join(ROOT, "tests", "golden")


def header_functions():
    text = open(os.path.join(ROOT, "include", "qs.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(qs_[a-z0-9_]+)\s*\(", text)))


def test_library_exports_every_declared_symbol():
    L = qs.lib()
    names = header_functions()
    assert len(names) >= 20
    for name in names:
        assert hasattr(L, name), name
    # the binding mirrors every declared entry point
    assert set(names) <= set(qs.exported_symbols())


def test_version_and_defaults():
    assert "sm_103a" in qs.qs_version()
    o = qs.options()
    assert o.blocking == 1 and o.fuse_width >= 1


def rand_state(n, seed):
    rng = np.random.default_rng(seed)
    v = rng.normal(size=1 << n) + 1j * rng.normal(size=1 << n)
    return v / np.linalg.norm(v)


ALL = ["H", "X", "Y", "Z", "S", "SDG", "T", "TDG", "RX", "RY", "RZ", "P", "U3", "CX", "CZ",
       "CP", "SWAP", "RZZ"]


def mixed_circuit(n, ng, seed, with_matrices=True, with_controls=True):
    rng = W.SplitMix64(seed)
    gates = list(W.random_circuit(n, ng, seed, ALL))
    if with_controls:
        out = []
        for g in gates:
            free = [q for q in range(n) if q not in g.targets + g.controls]
            if free and rng.below(4) == 0 and g.kind != "SWAP":
                out.append(g._replace(controls=g.controls + (free[rng.below(len(free))],)))
            else:
                out.append(g)
        gates = out
    if with_matrices:
        for i in range(6):
            k = 1 + rng.below(3)
            qs_ = tuple(rng.distinct(n, k))
            gates.insert(rng.below(len(gates)), Gate("UNITARY", qs_, (), (), W.random_unitary(k, seed + i)))
            k = 1 + rng.below(4)
            qs_ = tuple(rng.distinct(n, k))
            gates.insert(rng.below(len(gates)), Gate("DIAG", qs_, (), (), W.random_diag(k, seed + 50 + i)))
        gates.insert(3, Gate("SWAP", (0, n - 1), (1,)))
    return gates


def check_plan(gates, n, opts, seed=0):
    plan = qs.qs_fuse(gates, n, opts)
    try:
        text = qs.qs_plan_dump(plan)
        info = qs.qs_plan_info_get(plan)
    finally:
        qs.qs_plan_destroy(plan)
    a0 = rand_state(n, seed)
    want = oracle.apply_circuit(n, gates, a0.copy())
    got = a0.copy()
    layout, stats = replay(text, got)
    got_log = to_logical(got, n, layout)
    err = np.max(np.abs(got_log - want))
    assert err < 1e-12, err
    return info, stats


@pytest.mark.parametrize("fuse", [0, 1, 2, 3, 5])
@pytest.mark.parametrize("dtype", [qs.QS_C64, qs.QS_C128])
def test_gather_plans_match_oracle(fuse, dtype):
    n = 9
    gates = mixed_circuit(n, 120, 4000 + fuse)
    info, stats = check_plan(gates, n, qs.options(fuse_width=fuse, slab_bits=6, seg_bits=2, dtype=dtype))
    assert stats["max_b"] <= 6
    assert info["input_gates"] == len(gates)


@pytest.mark.parametrize("slab,seg,narrow", [(5, 1, 0), (6, 3, 1), (8, 2, 0), (8, 5, 1), (9, 4, 0), (10, 6, 1)])
@pytest.mark.parametrize("dtype", [qs.QS_C64, qs.QS_C128])
def test_slab_segment_and_stage_width_grid(slab, seg, narrow, dtype):
    """Gather plans over a grid of slab sizes, contiguous segment bits and both register-stage
    widths the kernels are built for (5 / 4 bits for complex64, 4 / 3 for complex128)."""
    n = 10
    stage = (5 if dtype == qs.QS_C64 else 4) - narrow
    gates = mixed_circuit(n, 140, 6100 + 10 * slab + seg)
    info, stats = check_plan(gates, n, qs.options(fuse_width=3, slab_bits=slab, seg_bits=seg,
                                                  stage_bits=stage, dtype=dtype))
    assert stats["max_b"] <= slab
    assert info["stage_bits"] == stage and info["input_gates"] == len(gates)


@pytest.mark.parametrize("slab", [4, 5, 7])
def test_lowblock_remap_plans_match_oracle(slab):
    n = 10
    gates = mixed_circuit(n, 100, 77 + slab)
    info, stats = check_plan(gates, n, qs.options(fuse_width=2, slab_bits=slab, seg_bits=2,
                                                  slab_mode=qs.QS_SLAB_REMAP))
    assert stats["remaps"] > 0


def test_unblocked_plan_is_one_op_per_gate():
    n = 7
    gates = [g for g in mixed_circuit(n, 60, 5, with_matrices=False)
             if not (g.kind == "SWAP" and not g.controls)]
    info, stats = check_plan(gates, n, qs.options(fuse_width=0, blocking=0))
    assert stats["unblocked"] == len(gates) and stats["passes"] == 0


@pytest.mark.parametrize("n", [1, 2, 3, 4])
def test_tiny_states(n):
    gates = mixed_circuit(n, 30, 9 + n, with_matrices=False, with_controls=n > 2) if n > 1 else \
        [Gate("H", (0,)), Gate("T", (0,)), Gate("U3", (0,), (), (0.1, 0.2, 0.3)), Gate("X", (0,))]
    check_plan(gates, n, qs.options())


def test_diagonal_gates_need_no_slab_residence():
    """Diagonal gates on high qubits fuse into tables applied from outside the slab."""
    n = 12
    gates = [Gate("H", (q,)) for q in range(4)]
    gates += [Gate("CP", (q, 11), (), (0.1 * q,)) for q in range(11)]
    gates += [Gate("RZZ", (10, 11), (), (0.7,)), Gate("T", (9,))]
    info, stats = check_plan(gates, n, qs.options(slab_bits=6, seg_bits=2))
    assert stats["passes"] == 1


def test_uncontrolled_swaps_are_relabels():
    n = 8
    gates = [Gate("H", (0,)), Gate("SWAP", (0, 7)), Gate("RY", (7,), (), (0.3,)), Gate("SWAP", (3, 5))]
    info, stats = check_plan(gates, n, qs.options(slab_bits=5, seg_bits=2, factor=1))
    # the relabel renames RY's qubit onto H's, so both fuse into one 1-qubit op
    assert stats["ops"] == 1
    info, stats = check_plan(gates, n, qs.options(slab_bits=5, seg_bits=2, fuse_width=0, factor=1))
    assert stats["ops"] == 2


def test_qft_and_layered_plans():
    n = 12
    g = W.qft(n)
    info, _ = check_plan(g, n, qs.options(slab_bits=8, seg_bits=3), seed=1)
    g = W.layered(n, 6, 1002)
    info, _ = check_plan(g, n, qs.options(slab_bits=8, seg_bits=3, fuse_width=3), seed=2)


def read_listing(path):
    out = []
    for line in open(path):
        if line.strip() and not line.startswith("#"):
            out.append(line.split())
    return out


def test_worked_example_low_block_plan():
    """Appendix worked example (10 qubits, chunk size 4): the low-block planner with a 4-qubit
    block and remap passes reproduces the raw circuit, and never needs more remap passes than
    the paper's listing has swap lines (5 SQS + 1 CSQS)."""
    raw = []
    for f in read_listing(os.path.join(GOLD, "worked_example_raw.txt")):
        qs_ = tuple(int(v) for v in f[1:-1])
        raw.append(Gate("H", qs_) if f[0] == "H" else Gate("RZZ", qs_, (), (float(f[-1]),)))
    info, stats = check_plan(raw, 10, qs.options(fuse_width=0, slab_bits=4, seg_bits=1,
                                                 slab_mode=qs.QS_SLAB_REMAP))
    assert stats["remaps"] <= 6
    # gather slabs: RZZ is diagonal and needs no residence; the H gates touch 7 qubits, one of
    # them in the 1-bit segment, so 3 free slab positions take two passes and no remap
    info, stats = check_plan(raw, 10, qs.options(fuse_width=0, slab_bits=4, seg_bits=1))
    assert stats["passes"] == 2 and stats["remaps"] == 0


def test_invalid_inputs_rejected_on_host():
    with pytest.raises(qs.QsError) as e:
        qs.qs_fuse([Gate("H", (9,))], 5)
    assert e.value.status == qs.QS_EINVAL
    with pytest.raises(qs.QsError):
        qs.qs_fuse([Gate("CX", (1,), (1,))], 5)
    with pytest.raises(qs.QsError):
        qs.qs_fuse([Gate("CX", (1,))], 5)
    with pytest.raises(qs.QsError):
        qs.qs_fuse([Gate("UNITARY", (0,), (), (), None)], 5)
    with pytest.raises(qs.QsError):
        qs.qs_fuse([Gate("H", (0,))], 0)
    with pytest.raises(qs.QsError):
        qs.qs_fuse([Gate("RZ", (0,), (), (float("nan"),))], 3)
    with pytest.raises(qs.QsError) as e:
        qs.qs_fuse([Gate("UNITARY", tuple(range(6)), (), (), W.random_unitary(6, 1))], 8,
                   qs.options(fuse_width=0))
    assert e.value.status == qs.QS_EUNSUPPORTED
    assert "tensor-core" in qs.qs_last_error()


def test_fault_injection_on_host(monkeypatch):
    monkeypatch.setenv("QS_FAULT", "plan")
    with pytest.raises(qs.QsError) as e:
        qs.qs_fuse([Gate("H", (0,))], 3)
    assert "injected" in str(e.value)


@pytest.mark.parametrize("width", [6, 7])
@pytest.mark.parametrize("mode", [qs.QS_TC_BF16X3, qs.QS_TC_TF32X3])
@pytest.mark.parametrize("n", [13, 15])
def test_tensor_core_plans_match_oracle(n, mode, width):
    """Tensor-core mode fuses into dense blocks of at most 6 or 7 qubits (4+ qubit blocks run as
    tensor-core steps: 7-qubit blocks as such, narrower ones padded to 6); the listing carries
    the FP64 fused matrices, replayed on the oracle."""
    gates = W.layered(n, 4, 11) + W.random_circuit(n, 40, 12, ALL)
    opts = qs.options(tc=mode, dtype=qs.QS_C64, tc_width=width)
    info, stats = check_plan(gates, n, opts)
    assert info["tc_gates"] > 0
    p = qs.qs_fuse(gates, n, opts)
    try:
        widths = [int(l.split()[2]) for l in qs.qs_plan_dump(p).splitlines() if l.startswith("OP DENSE")]
    finally:
        qs.qs_plan_destroy(p)
    if width == 7:
        assert 7 in widths
    assert max(widths) == width


def test_tensor_core_mode_rejections():
    g = W.layered(14, 2, 1)
    with pytest.raises(qs.QsError) as e:
        qs.qs_fuse(g, 14, qs.options(tc=qs.QS_TC_BF16X3, dtype=qs.QS_C128))
    assert e.value.status == qs.QS_EUNSUPPORTED
    with pytest.raises(qs.QsError) as e:
        qs.qs_fuse(W.layered(10, 2, 1), 10, qs.options(tc=qs.QS_TC_BF16X3, dtype=qs.QS_C64))
    assert e.value.status == qs.QS_EUNSUPPORTED
    with pytest.raises(qs.QsError) as e:
        qs.qs_fuse(g, 14, qs.options(tc=qs.QS_TC_TF32X3, dtype=qs.QS_C64, tc_width=8))
    assert e.value.status == qs.QS_EUNSUPPORTED


@pytest.mark.parametrize("dtype,stage", [(qs.QS_C64, 5), (qs.QS_C64, 4), (qs.QS_C128, 4), (qs.QS_C128, 3)])
def test_euler_split_and_stage_diagonal_tables(dtype, stage):
    """Complex 1-qubit gates become a real rotation between two phases; the phases and CZ signs
    of a stage merge into register-bit tables.  The replayed plan still equals the oracle."""
    n = 12
    g = W.layered(n, 8, 2024)
    info, stats = check_plan(g, n, qs.options(slab_bits=9, seg_bits=3, dtype=dtype, stage_bits=stage, euler=2), seed=3)
    p = qs.qs_fuse(g, n, qs.options(slab_bits=9, seg_bits=3, dtype=dtype, stage_bits=stage, euler=2))
    try:
        X = qs.qs_plan_features(p)
    finally:
        qs.qs_plan_destroy(p)
    assert X[:, 16].sum() <= 1        # complex 2x2 in stages: at most the global-phase carrier
    assert X[:, 16].sum() + X[:, 17].sum() >= n * 8  # one rotation per U3 (one carries the phase)
    assert X[:, 20].sum() >= 1        # merged register-bit diagonal tables


def test_euler_split_of_generic_unitaries_and_rz():
    n = 10
    rng = W.SplitMix64(5)
    gates = []
    for i in range(60):
        q = rng.below(n)
        r = rng.below(4)
        if r == 0:
            gates.append(Gate("UNITARY", (q,), (), (), W.random_unitary(1, 900 + i)))
        elif r == 1:
            gates.append(Gate("RZ", (q,), (), (rng.angle(),)))
        elif r == 2:
            gates.append(Gate("RX", (q,), (), (rng.angle(),)))
        else:
            a, b = rng.distinct(n, 2)
            gates.append(Gate("CZ", (a, b)))
    for dtype in (qs.QS_C64, qs.QS_C128):
        check_plan(gates, n, qs.options(slab_bits=7, seg_bits=2, dtype=dtype, euler=2), seed=4)


def test_euler_split_is_the_default_and_can_be_turned_off():
    g = W.layered(12, 4, 7)
    counts = {}
    for dtype in (qs.QS_C64, qs.QS_C128):
        for eu in (0, 1, 2):
            p = qs.qs_fuse(g, 12, qs.options(dtype=dtype, euler=eu, slab_bits=9, seg_bits=3))
            counts[dtype, eu] = qs.qs_plan_features(p)[:, 17].sum()  # real 1-qubit rotations
            qs.qs_plan_destroy(p)
    for dtype in (qs.QS_C64, qs.QS_C128):
        assert counts[dtype, 0] == counts[dtype, 2] > 0 and counts[dtype, 1] == 0


@pytest.mark.parametrize("dtype", [qs.QS_C64, qs.QS_C128])
def test_factored_rotations_replay_against_oracle(dtype):
    """Register-stage real 2 x 2 gates written as D N (N with two unit entries, D folded into the
    stage tables): the listing holds such N matrices, and replaying it on the oracle gives the
    circuit's state.  Rotations with |cos| < |sin| take the anti-diagonal form."""
    n = 11
    gates = W.layered(n, 6, 31) + [Gate("H", (q,)) for q in range(n)]
    gates += [Gate("RY", (q,), (), (2.6 + 0.05 * q,)) for q in range(n)]  # |cos| < |sin|
    gates += W.qft(n)
    plan = qs.qs_fuse(gates, n, qs.options(dtype=dtype))
    text = qs.qs_plan_dump(plan)
    qs.qs_plan_destroy(plan)
    _, items, _ = PR.parse_dump(text)
    forms = {"N": 0, "NM": 0, "A": 0, "AM": 0}
    for it in items:
        if it[0] == "OP" and it[1] == "DENSE" and len(it[2]) == 1 and not it[3]:
            m = it[4]
            if m[0, 0] == 1:
                forms["N" if m[1, 1] == 1 else "NM" if m[1, 1] == -1 else "N?"] = 1 + forms.get("N", 0)
            elif m[0, 1] == 1:
                forms["A" if m[1, 0] == 1 else "AM" if m[1, 0] == -1 else "A?"] = 1 + forms.get("A", 0)
    # rotations give N / AM, reflections (H) NM, rotations with |cos| < |sin| A or AM
    assert forms["N"] and forms["NM"] and (forms["A"] or forms["AM"]), forms
    assert "N?" not in forms and "A?" not in forms
    check_plan(gates, n, qs.options(dtype=dtype))
    off, _ = check_plan(gates, n, qs.options(dtype=dtype, factor=1))


def test_arith_option_is_validated():
    g = W.layered(12, 2, 3)
    p = qs.qs_fuse(g, 12, qs.options(dtype=qs.QS_C128, arith=qs.QS_ARITH_DF))
    qs.qs_plan_destroy(p)
    with pytest.raises(qs.QsError) as e:
        qs.qs_fuse(g, 12, qs.options(dtype=qs.QS_C128, arith=2))
    assert e.value.status == qs.QS_EINVAL


def test_identity_products_are_dropped():
    """H H and RZ(t) RZ(-t) fuse to the identity and leave no op; a uniform phase stays."""
    n = 6
    gates = [Gate("H", (2,)), Gate("H", (2,)), Gate("RZ", (4,), (), (0.7,)), Gate("RZ", (4,), (), (-0.7,))]
    info, stats = check_plan(gates, n, qs.options(dtype=qs.QS_C128))
    assert stats["ops"] == 0
    phase = [Gate("DIAG", (1,), (), (), np.array([1j, 1j]))]
    info, stats = check_plan(phase, n, qs.options(dtype=qs.QS_C128))
    assert stats["ops"] == 1


@pytest.mark.parametrize("dtype,arith,widest", [(qs.QS_C128, qs.QS_ARITH_FP64, 4 + 10),
                                                (qs.QS_C128, qs.QS_ARITH_DF, 4 + 6),
                                                (qs.QS_C64, qs.QS_ARITH_FP64, 5 + 6)])
def test_stage_table_condition_bits_default_by_arithmetic(dtype, arith, widest):
    """merge_bits = 0: merged stage tables read up to 10 condition bits besides the register bits
    for complex128 stages in FP64 (whose time is FP64 multiplies), 6 otherwise; the replayed
    plan still equals the oracle, and an explicit merge_bits overrides the default."""
    n = 16
    g = W.qft(n)
    info, stats = check_plan(g, n, qs.options(dtype=dtype, arith=arith), seed=5)
    p = qs.qs_fuse(g, n, qs.options(dtype=dtype, arith=arith))
    q = qs.qs_fuse(g, n, qs.options(dtype=dtype, arith=arith, merge_bits=2))
    try:
        widths = [int(l.split()[2]) for l in qs.qs_plan_dump(p).splitlines() if l.startswith("OP DIAG")]
        narrow = [int(l.split()[2]) for l in qs.qs_plan_dump(q).splitlines() if l.startswith("OP DIAG")]
    finally:
        qs.qs_plan_destroy(p)
        qs.qs_plan_destroy(q)
    rb = 5 if dtype == qs.QS_C64 else 4  # register bits of a stage
    assert max(widths) == widest
    assert max(narrow) <= rb + 2
