"""GPU parity: the CUDA path through the C ABI against the FP64 oracle, element by element.

Tolerances (max |delta amplitude|): 1e-12 for complex128, 1e-5 for complex64.  Readouts:
|delta| <= 1e-9 * n (complex128) and 1e-4 * n (complex64) for expectations, 1e-12 / 1e-6 for
probabilities.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2406_14084_gb300 import qs
from paper_2406_14084_gb300 import workloads as W
from paper_2406_14084_gb300.workloads import Gate

pytestmark = pytest.mark.gpu

TOL = {qs.QS_C64: 1e-5, qs.QS_C128: 1e-12}
ALL = ["H", "X", "Y", "Z", "S", "SDG", "T", "TDG", "RX", "RY", "RZ", "P", "U3", "CX", "CZ",
       "CP", "SWAP", "RZZ"]


def run(n, gates, dtype, opts=None, x0=0, init=None):
    s = qs.State(n, dtype)
    try:
        if init is not None:
            s_init = init.astype(np.complex64 if dtype == qs.QS_C64 else np.complex128)
            qs.qs_copy_from_host(s.h, s_init)
        else:
            s.set_basis(x0)
        if opts is not None:
            opts.dtype = dtype
        s.apply(gates, opts)
        return s.amplitudes().astype(np.complex128)
    finally:
        s.close()


def ref(n, gates, x0=0, init=None):
    a = init.copy() if init is not None else oracle.basis_state(n, x0)
    return oracle.apply_circuit(n, gates, a)


def rand_state(n, seed):
    rng = np.random.default_rng(seed)
    v = rng.normal(size=1 << n) + 1j * rng.normal(size=1 << n)
    return v / np.linalg.norm(v)


def mixed(n, ng, seed):
    rng = W.SplitMix64(seed)
    gates = list(W.random_circuit(n, ng, seed, ALL))
    out = []
    for g in gates:
        free = [q for q in range(n) if q not in g.targets + g.controls]
        if free and rng.below(4) == 0:
            out.append(g._replace(controls=g.controls + (free[rng.below(len(free))],)))
        else:
            out.append(g)
    for i in range(8):
        k = 1 + rng.below(5)
        out.insert(rng.below(len(out)), Gate("UNITARY", tuple(rng.distinct(n, k)), (), (),
                                              W.random_unitary(k, seed + i)))
        k = 1 + rng.below(min(7, n))
        out.insert(rng.below(len(out)), Gate("DIAG", tuple(rng.distinct(n, k)), (), (),
                                              W.random_diag(k, seed + 99 + i)))
    return out


# ----------------------------------------------------------------------------- config 1

@pytest.mark.parametrize("blocking", [0, 1])
def test_config1_random_200_gates_complex128(blocking):
    """20 qubits, complex128, |0..0>, 200 gates from {H,X,S,T,RZ,U3,CX,CZ,SWAP}, no fusion."""
    n = 20
    gates = W.random_circuit(n, 200, 1001)
    want = ref(n, gates)
    got = run(n, gates, qs.QS_C128, qs.options(fuse_width=0, blocking=blocking))
    assert np.max(np.abs(got - want)) <= 1e-12


@pytest.mark.parametrize("dtype", [qs.QS_C64, qs.QS_C128])
@pytest.mark.parametrize("fuse", [1, 2, 3, 4, 5])
def test_config1_with_fusion_and_blocking(dtype, fuse):
    n = 20
    gates = W.random_circuit(n, 200, 1001)
    want = ref(n, gates)
    got = run(n, gates, dtype, qs.options(fuse_width=fuse))
    assert np.max(np.abs(got - want)) <= TOL[dtype]


# ----------------------------------------------------------------------------- all gate kinds

@pytest.mark.parametrize("dtype", [qs.QS_C64, qs.QS_C128])
@pytest.mark.parametrize("mode", ["gather", "lowblock", "unblocked", "nofuse"])
def test_mixed_kinds_controls_matrices(dtype, mode):
    n = 15
    gates = mixed(n, 150, 31)
    opts = {"gather": qs.options(fuse_width=3, slab_bits=9),
            "lowblock": qs.options(fuse_width=2, slab_bits=9, slab_mode=qs.QS_SLAB_REMAP),
            "unblocked": qs.options(fuse_width=0, blocking=0),
            "nofuse": qs.options(fuse_width=0)}[mode]
    init = rand_state(n, 5)
    want = ref(n, gates, init=init)
    got = run(n, gates, dtype, opts, init=init)
    assert np.max(np.abs(got - want)) <= TOL[dtype]


@pytest.mark.parametrize("n", [1, 2, 3, 4, 5, 6, 9])
@pytest.mark.parametrize("dtype", [qs.QS_C64, qs.QS_C128])
def test_small_and_ragged_sizes(n, dtype):
    if n == 1:
        gates = [Gate("H", (0,)), Gate("T", (0,)), Gate("U3", (0,), (), (0.4, 1.2, 2.2)), Gate("X", (0,))]
    else:
        gates = W.random_circuit(n, 40, 70 + n, ALL)
    init = rand_state(n, n)
    want = ref(n, gates, init=init)
    for opts in (qs.options(), qs.options(fuse_width=0, blocking=0)):
        got = run(n, gates, dtype, opts, init=init)
        assert np.max(np.abs(got - want)) <= TOL[dtype]


@pytest.mark.parametrize("dtype", [qs.QS_C64, qs.QS_C128])
def test_boundary_qubits_of_segment_and_slab(dtype):
    """Targets and controls at bit 0, the last segment bit, the first outside bit, n-1."""
    n = 18
    lo = 4 if dtype == qs.QS_C64 else 3
    qs_ = [0, lo - 1, lo, 12, 13, n - 1]
    gates = []
    for i, a in enumerate(qs_):
        gates.append(Gate("U3", (a,), (), (0.3 + i, 0.2 * i, 1.1)))
        for b in qs_:
            if b != a:
                gates.append(Gate("CX", (b,), (a,)))
                gates.append(Gate("CP", (a, b), (), (0.7 + 0.1 * i,)))
    gates.append(Gate("UNITARY", (n - 1, 0, lo), (), (), W.random_unitary(3, 4)))
    gates.append(Gate("DIAG", tuple(qs_), (), (), W.random_diag(len(qs_), 5)))
    init = rand_state(n, 8)
    want = ref(n, gates, init=init)
    for b in (8, 10, 12):
        got = run(n, gates, dtype, qs.options(slab_bits=b, fuse_width=2), init=init)
        assert np.max(np.abs(got - want)) <= TOL[dtype]


# ----------------------------------------------------------------------------- circuit shapes

@pytest.mark.parametrize("dtype", [qs.QS_C64, qs.QS_C128])
def test_qft_random_basis(dtype):
    n = 22
    x = W.random_basis(n, 1002)
    gates = W.qft(n)
    y = np.arange(1 << n)
    rev = np.zeros_like(y)
    for j in range(n):
        rev |= ((y >> j) & 1) << (n - 1 - j)
    closed = 2.0 ** (-n / 2) * np.exp(2j * np.pi * ((x * rev) % (1 << n)) / (1 << n))
    got = run(n, gates, dtype, qs.options(), x0=x)
    assert np.max(np.abs(got - closed)) <= TOL[dtype]


@pytest.mark.parametrize("dtype", [qs.QS_C64, qs.QS_C128])
@pytest.mark.parametrize("fuse", [1, 2, 4])
def test_layered_circuit(dtype, fuse):
    n = 20
    gates = W.layered(n, 8, 1003)
    want = ref(n, gates)
    got = run(n, gates, dtype, qs.options(fuse_width=fuse))
    assert np.max(np.abs(got - want)) <= TOL[dtype]


def test_vqe_and_qaoa_shapes():
    for n, gates in [(16, W.vqe_circuit(16, 4, 5)), (18, W.qaoa_like(18, 3, 6))]:
        want = ref(n, gates)
        for dtype in (qs.QS_C64, qs.QS_C128):
            got = run(n, gates, dtype, qs.options())
            assert np.max(np.abs(got - want)) <= TOL[dtype]


# ----------------------------------------------------------------------------- readouts

@pytest.mark.parametrize("dtype", [qs.QS_C64, qs.QS_C128])
def test_readouts_after_relabelling_plan(dtype):
    """probs / expectations / norm read logical qubits whatever layout the plan left."""
    n = 16
    gates = W.layered(n, 3, 9) + [Gate("SWAP", (0, 15)), Gate("SWAP", (3, 9))] + W.vqe_circuit(n, 2, 4)
    want = ref(n, gates)
    s = qs.State(n, dtype)
    try:
        s.apply(gates, qs.options(dtype=dtype))
        ptol = 1e-12 if dtype == qs.QS_C128 else 1e-6
        for q in ([0], [15, 3], [9, 0, 4, 1], list(range(n))):
            assert np.max(np.abs(s.probs(q) - oracle.probs(want, n, q))) <= ptol
        H = W.zz_chain_hamiltonian(n)
        terms = H + [(0.3, 0b1010, 0b0110), (-0.7, 1 << 15 | 1, 0), (0.2, 0, 0), (1.1, 0b11 << 7, 0b10 << 7)]
        e = s.expect(terms)
        etol = (1e-9 if dtype == qs.QS_C128 else 1e-4) * n
        w = oracle.expect_pauli(want, n, terms)
        assert abs(e.real - w.real) <= etol and abs(e.imag) <= etol
        assert abs(s.norm2() - 1.0) <= (1e-12 if dtype == qs.QS_C128 else 1e-5)
        got = s.amplitudes().astype(np.complex128)
        assert np.max(np.abs(got - want)) <= TOL[dtype]
    finally:
        s.close()


def test_expectation_closed_forms_on_gpu():
    n = 20
    H = W.zz_chain_hamiltonian(n)
    for dtype in (qs.QS_C64, qs.QS_C128):
        s = qs.State(n, dtype)
        try:
            assert abs(s.expect(H).real - (n + 0.5 * (n - 1))) <= 1e-6
            s.apply([Gate("H", (q,)) for q in range(n)])
            assert abs(s.expect(H).real) <= 1e-6
        finally:
            s.close()


def test_remap_canonicalize_and_copy_roundtrip():
    n = 17
    for dtype in (qs.QS_C64, qs.QS_C128):
        init = rand_state(n, 12)
        s = qs.State(n, dtype)
        try:
            qs.qs_copy_from_host(s.h, init.astype(np.complex64 if dtype == qs.QS_C64 else np.complex128))
            qs.qs_remap(s.h, [0, 2, 5], [16, 9, 11])
            # readouts are logical: unchanged by a remap
            got = s.amplitudes().astype(np.complex128)
            assert np.max(np.abs(got - init)) <= TOL[dtype]
            # raw buffer really is permuted
            qs.qs_remap(s.h, [1], [13])
            ptr, phys = qs.qs_get_buffer(s.h, n)
            assert phys[1] == 13 and phys[13] == 1
            qs.qs_canonicalize(s.h)
            ptr, phys = qs.qs_get_buffer(s.h, n)
            assert phys == list(range(n))
        finally:
            s.close()


def test_remap_physical_content_matches_oracle_remap():
    import torch
    n = 15
    init = rand_state(n, 3)
    buf = torch.empty(1 << n, dtype=torch.complex128, device="cuda")
    buf.copy_(torch.from_numpy(init))
    stream = torch.cuda.Stream()
    h = qs.qs_create_from_buffer(n, qs.QS_C128, buf.data_ptr(), stream.cuda_stream)
    try:
        qs.qs_remap(h, [0, 3, 4], [14, 7, 10])
        qs.qs_sync(h)
        want = oracle.remap(init.copy(), n, [0, 3, 4], [14, 7, 10])
        assert np.array_equal(buf.cpu().numpy(), want)  # a permutation: bit-exact
    finally:
        qs.qs_destroy(h)


def test_external_buffer_and_stream():
    import torch
    n = 18
    buf = torch.zeros(1 << n, dtype=torch.complex64, device="cuda")
    stream = torch.cuda.Stream()
    h = qs.qs_create_from_buffer(n, qs.QS_C64, buf.data_ptr(), stream.cuda_stream)
    try:
        qs.qs_set_basis(h, 5)
        gates = W.random_circuit(n, 60, 3)
        qs.qs_apply_circuit(h, gates, qs.options())
        qs.qs_canonicalize(h)
        qs.qs_sync(h)
        want = ref(n, gates, x0=5)
        got = buf.cpu().numpy().astype(np.complex128)
        assert np.max(np.abs(got - want)) <= 1e-5
    finally:
        qs.qs_destroy(h)


def test_plan_reuse_and_stats():
    n = 19
    gates = W.layered(n, 4, 77)
    plan = qs.qs_fuse(gates, n, qs.options(dtype=qs.QS_C128))
    s = qs.State(n, qs.QS_C128)
    try:
        for _ in range(2):
            s.set_basis(0)
            qs.qs_apply_plan(s.h, plan)
            got = s.amplitudes()
            assert np.max(np.abs(got - ref(n, gates))) <= 1e-12
        st = qs.qs_stats(s.h)
        info = qs.qs_plan_info_get(plan)
        assert st["plans_applied"] == 2 and st["passes"] >= 2 * info["passes"]
    finally:
        s.close()
        qs.qs_plan_destroy(plan)


def test_invalid_calls_leave_state_untouched():
    n = 10
    s = qs.State(n, qs.QS_C128)
    try:
        s.apply([Gate("H", (0,))])
        before = s.amplitudes()
        with pytest.raises(qs.QsError):
            s.apply([Gate("H", (0,)), Gate("CX", (12,), (0,))])
        with pytest.raises(qs.QsError):
            s.probs([0, 0])
        with pytest.raises(qs.QsError):
            s.expect([(1.0, 1 << 12, 0)])
        with pytest.raises(qs.QsError):
            qs.qs_set_basis(s.h, 1 << 10)
        assert np.array_equal(s.amplitudes(), before)
    finally:
        s.close()


def test_host_fault_injection_paths(monkeypatch):
    monkeypatch.setenv("QS_FAULT", "alloc")
    with pytest.raises(qs.QsError) as e:
        qs.State(10)
    assert e.value.status == qs.QS_ENOMEM
    monkeypatch.setenv("QS_FAULT", "launch")
    s = None
    monkeypatch.delenv("QS_FAULT")
    s = qs.State(8)
    try:
        monkeypatch.setenv("QS_FAULT", "launch")
        with pytest.raises(qs.QsError) as e:
            s.apply([Gate("H", (0,))])
        assert e.value.status == qs.QS_ECUDA
        monkeypatch.delenv("QS_FAULT")
        s.apply([Gate("H", (0,))])
        assert abs(s.amplitudes()[0] - 1 / math.sqrt(2)) < 1e-6
    finally:
        s.close()


@pytest.mark.parametrize("dtype", [qs.QS_C64, qs.QS_C128])
@pytest.mark.parametrize("n", [16, 19])
def test_expectation_many_terms_per_x_mask(dtype, n):
    """Groups of four or more Z strings per X mask take the Walsh-Hadamard tile kernel: X mask
    zero, inside the 1024-amplitude tile (even and odd), above it (paired tiles, with and
    without low bits); smaller groups take the per-term loop.  Against the oracle on a random
    (circuit-prepared) state."""
    rng = W.SplitMix64(300 + n)
    gates = W.layered(n, 3, 77) + W.vqe_circuit(n, 2, 78)
    want = ref(n, gates)
    terms, by_group = [], []
    groups = ((0, 40), (0b101 << 3, 9), (1 << (n - 1), 130), (0b11, 3), (0b1001, 12),
              ((1 << (n - 2)) | 0b1, 20), ((1 << 12) | (1 << 10) | 0b110, 7),
              (0b110 << 9, 300))  # 300 terms: split into groups of 256 and 44
    for xm, count in groups:
        grp = []
        for _ in range(count):
            zm = rng.next_u64() & ((1 << n) - 1)
            grp.append((rng.angle() - 3.0, xm, zm))
        by_group.append(grp)
        terms += grp
    s = qs.State(n, dtype)
    try:
        s.apply(gates, qs.options(dtype=dtype))
        e = s.expect(terms)
        w = oracle.expect_pauli(want, n, terms)
        tol = (1e-9 if dtype == qs.QS_C128 else 2e-4) * len(terms)
        assert abs(e.real - w.real) <= tol and abs(e.imag - w.imag) <= tol
        # each group alone, against the oracle on the device's own amplitudes (kernel arithmetic only)
        mine = s.amplitudes().astype(np.complex128)
        for grp in by_group:
            e = s.expect(grp)
            w = oracle.expect_pauli(mine, n, grp)
            tol = (1e-12 if dtype == qs.QS_C128 else 2e-6) * sum(abs(c) for c, _, _ in grp)
            assert abs(e.real - w.real) <= tol and abs(e.imag - w.imag) <= tol, grp[0][1]
    finally:
        s.close()
