"""Pins for the FP64 oracle: closed forms, the paper's printed worked example and values,
textbook identities, invariants, and brute force through an independent numpy route.

None of these re-types the oracle's own loops: the brute-force check builds each gate as a
tensor contraction (numpy.tensordot over the target axes), the rotation gates are compared
with matrix exponentials of Pauli matrices (scipy.linalg.expm), and the worked example and
fused-diagonal values are the numbers printed in arXiv 2406.14084's artifact appendix.
"""
import math
import os

import numpy as np
import pytest
import scipy.linalg

import oracle
from paper_2406_14084_gb300 import workloads as W
from paper_2406_14084_gb300.workloads import Gate

GOLD = os.path.join(os.path.dirname(__file__), "golden")

I2 = np.eye(2)
PX = np.array([[0, 1], [1, 0]], dtype=complex)
PY = np.array([[0, -1j], [1j, 0]], dtype=complex)
PZ = np.array([[1, 0], [0, -1]], dtype=complex)


def rand_state(n, seed):
    rng = np.random.default_rng(seed)
    v = rng.normal(size=1 << n) + 1j * rng.normal(size=1 << n)
    return (v / np.linalg.norm(v)).astype(np.complex128)


# ----------------------------------------------------------------------------- closed forms

@pytest.mark.parametrize("n", [1, 2, 5, 10])
def test_hadamard_layer_uniform(n):
    """H on every qubit of |0..0> gives every amplitude 2^{-n/2}."""
    a = oracle.apply_circuit(n, [Gate("H", (q,)) for q in range(n)])
    assert np.max(np.abs(a - 2.0 ** (-n / 2))) < 1e-14


@pytest.mark.parametrize("n", [2, 3, 7])
def test_ghz(n):
    g = [Gate("H", (0,))] + [Gate("CX", (q + 1,), (q,)) for q in range(n - 1)]
    a = oracle.apply_circuit(n, g)
    expect = np.zeros(1 << n, dtype=complex)
    expect[0] = expect[-1] = 1 / math.sqrt(2)
    assert np.max(np.abs(a - expect)) < 1e-15


def bitrev(y, n):
    return int(format(y, f"0{n}b")[::-1], 2)


@pytest.mark.parametrize("n", [1, 2, 3, 6, 8])
def test_qft_of_basis_state_closed_form(n):
    """No-swap QFT of |x>: amplitude at y is 2^{-n/2} exp(2 pi i x rev(y) / 2^n)."""
    for x in [0, 1, (1 << n) - 1, W.random_basis(n, 7)]:
        a = oracle.apply_circuit(n, W.qft(n), oracle.basis_state(n, x))
        y = np.arange(1 << n)
        rev = np.array([bitrev(int(v), n) for v in y])
        expect = 2.0 ** (-n / 2) * np.exp(2j * np.pi * x * rev / (1 << n))
        assert np.max(np.abs(a - expect)) < 1e-13


def test_qft_gate_count_matches_paper():
    """Table 2: the 31-qubit QFT has 496 gates (31 H + 465 CP, no final swaps)."""
    g = W.qft(31)
    assert len(g) == 496
    assert sum(1 for x in g if x.kind == "H") == 31


# ----------------------------------------------------------------------------- gate conventions

def U(kind, *params, k=1):
    return oracle.gate_matrix(Gate(kind, tuple(range(k)), (), tuple(params)))


def close(a, b, tol=1e-14):
    return np.max(np.abs(np.asarray(a) - np.asarray(b))) < tol


def test_clifford_identities():
    H, X, Y, Z, S, T = (U(k) for k in ("H", "X", "Y", "Z", "S", "T"))
    assert close(H @ Z @ H, X) and close(H @ X @ H, Z)
    assert close(S @ S, Z) and close(T @ T, S)
    assert close(U("SDG"), S.conj().T) and close(U("TDG"), T.conj().T)
    assert close(Y, 1j * X @ Z)
    assert close(X, PX) and close(Y, PY) and close(Z, PZ)
    assert close(H @ H, I2)


@pytest.mark.parametrize("theta", [0.3, 1.7, -2.9, 5.5])
def test_rotations_are_pauli_exponentials(theta):
    assert close(U("RX", theta), scipy.linalg.expm(-0.5j * theta * PX))
    assert close(U("RY", theta), scipy.linalg.expm(-0.5j * theta * PY))
    assert close(U("RZ", theta), scipy.linalg.expm(-0.5j * theta * PZ))
    assert close(U("P", theta), np.exp(0.5j * theta) * U("RZ", theta))
    zz = np.kron(PZ, PZ)
    assert close(U("RZZ", theta, k=2), scipy.linalg.expm(-0.5j * theta * zz))


@pytest.mark.parametrize("seed", range(4))
def test_u3_is_zyz_euler_product(seed):
    rng = W.SplitMix64(seed)
    th, ph, la = rng.angle(), rng.angle(), rng.angle()
    zyz = U("RZ", ph) @ U("RY", th) @ U("RZ", la)
    assert close(U("U3", th, ph, la), np.exp(0.5j * (ph + la)) * zyz)
    u = U("U3", th, ph, la)
    assert close(u.conj().T @ u, I2)


def read_matrix(path):
    rows = [r for r in open(path) if r.strip() and not r.startswith("#")]
    return np.array([[float(v) for v in r.split()] for r in rows])


def test_cnot_matches_eq3():
    """Eq. 3 orders the 4-tuple with the control i as the high bit and target j as the low bit."""
    M = read_matrix(os.path.join(GOLD, "eq3_cnot.txt"))
    # target = qubit 0 (low bit), control = qubit 1 (high bit)
    got = oracle.circuit_unitary([Gate("CX", (0,), (1,))], 2)
    assert close(got, M)


def test_two_qubit_gate_identities():
    cx01 = oracle.circuit_unitary([Gate("CX", (1,), (0,))], 2)
    cx10 = oracle.circuit_unitary([Gate("CX", (0,), (1,))], 2)
    swap = oracle.circuit_unitary([Gate("SWAP", (0, 1))], 2)
    assert close(swap, cx01 @ cx10 @ cx01)
    cz = oracle.circuit_unitary([Gate("CZ", (0, 1))], 2)
    assert close(cz, oracle.circuit_unitary([Gate("CZ", (1, 0))], 2))
    assert close(cz, oracle.circuit_unitary([Gate("CP", (0, 1), (), (math.pi,))], 2))
    # CZ = (I x H) CX (I x H) with H on the target
    h_t = [Gate("H", (0,))]
    assert close(cz, oracle.circuit_unitary(h_t + [Gate("CX", (0,), (1,))] + h_t, 2))
    # CP(l) = controlled-P(l)
    assert close(oracle.circuit_unitary([Gate("CP", (0, 1), (), (0.7,))], 2),
                 oracle.circuit_unitary([Gate("P", (1,), (0,), (0.7,))], 2))


def test_fused_rzz_diagonal_matches_paper_values():
    """Appendix, Fig. 5(c): the fused D4 gates print Re(diag[0]) = cos(sum of RZZ angles / 2)
    with each RZZ's angle equal to its ID."""
    for line in open(os.path.join(GOLD, "fused_diag_rzz.txt")):
        if not line.strip() or line.startswith("#"):
            continue
        val, *items = line.split()
        gates = []
        for it in items:
            qs, gid = it.split(":")
            a, b = (int(v) for v in qs.split(","))
            gates.append(Gate("RZZ", (a, b), (), (float(gid),)))
        Uf = oracle.circuit_unitary(gates, 4)
        assert np.allclose(Uf, np.diag(np.diag(Uf)), atol=0)  # still diagonal
        assert abs(Uf[0, 0].real - float(val)) < 1e-15


# ----------------------------------------------------------------------------- brute force

def apply_by_contraction(state, n, g):
    """Independent route: the gate as a tensor contraction over the target axes of the state
    tensor (axis 0 = qubit n-1), with controls as projectors."""
    Ug = oracle.gate_matrix(g)
    k = len(g.targets)
    psi = state.reshape((2,) * n)
    ax = lambda q: n - 1 - q  # noqa: E731
    # U's row/col index bit j is target t_j -> reshape (2,)*k has axis 0 = bit k-1 = t_{k-1}
    Ut = Ug.reshape((2,) * (2 * k))
    in_axes = [ax(g.targets[k - 1 - j]) for j in range(k)]
    moved = np.tensordot(Ut, psi, axes=(list(range(k, 2 * k)), in_axes))
    # tensordot puts the k output axes first; move them back into place
    out = np.moveaxis(moved, list(range(k)), in_axes)
    if g.controls:
        mask = np.ones((2,) * n, dtype=bool)
        idx = [slice(None)] * n
        for c in g.controls:
            sel = [slice(None)] * n
            sel[ax(c)] = 0
            mask[tuple(sel)] = False
        out = np.where(mask, out, psi)
    return out.reshape(-1)


ALL_KINDS = ["H", "X", "Y", "Z", "S", "SDG", "T", "TDG", "RX", "RY", "RZ", "P", "U3", "CX",
             "CZ", "CP", "SWAP", "RZZ", "UNITARY", "DIAG"]


def random_gate(rng, n, kind, seed):
    two = {"CZ", "CP", "SWAP", "RZZ"}
    nctl = rng.below(3) if n >= 5 else 0
    if kind == "UNITARY":
        k = 1 + rng.below(min(3, n - nctl))
    elif kind == "DIAG":
        k = 1 + rng.below(min(4, n - nctl))
    elif kind in two:
        k = 2
    else:
        k = 1
    qs = rng.distinct(n, k + nctl + (1 if kind == "CX" else 0))
    tg, ct = tuple(qs[:k]), tuple(qs[k:])
    par = (rng.angle(), rng.angle(), rng.angle())
    m = None
    if kind == "UNITARY":
        m = W.random_unitary(k, seed)
    elif kind == "DIAG":
        m = W.random_diag(k, seed)
    return Gate(kind, tg, ct, par, m)


@pytest.mark.parametrize("n", [1, 3, 5, 6])
def test_index_loop_matches_contraction(n):
    rng = W.SplitMix64(100 + n)
    a0 = rand_state(n, n)
    ref = a0.copy()
    gates = []
    for i in range(60):
        kind = ALL_KINDS[rng.below(len(ALL_KINDS))]
        if n < 2 and kind in ("CZ", "CP", "SWAP", "RZZ", "CX"):
            continue
        g = random_gate(rng, n, kind, 1000 + i)
        gates.append(g)
        ref = apply_by_contraction(ref, n, g)
    got = oracle.apply_circuit(n, gates, a0.copy())
    assert np.max(np.abs(got - ref)) < 1e-13


@pytest.mark.parametrize("n", [4, 6])
def test_full_matrix_product_brute_force(n):
    """The 2^n x 2^n matrix of a circuit (each gate embedded by contraction on every basis
    column, matrices multiplied) applied to a state equals the one-gate-at-a-time result."""
    rng = W.SplitMix64(55 + n)
    gates = [random_gate(rng, n, ALL_KINDS[rng.below(len(ALL_KINDS))], 3000 + i) for i in range(25)]
    M = np.eye(1 << n, dtype=complex)
    for g in gates:
        G = np.stack([apply_by_contraction(np.eye(1 << n, dtype=complex)[:, j].copy(), n, g)
                      for j in range(1 << n)], axis=1)
        M = G @ M
    a0 = rand_state(n, 9)
    got = oracle.apply_circuit(n, gates, a0.copy())
    assert np.max(np.abs(got - M @ a0)) < 1e-13
    assert np.max(np.abs(M.conj().T @ M - np.eye(1 << n))) < 1e-12


def test_circuit_unitary_is_kron_for_disjoint_gates():
    g1 = Gate("U3", (0,), (), (0.4, 1.1, 2.3))
    g2 = Gate("RY", (1,), (), (0.9,))
    Uf = oracle.circuit_unitary([g1, g2], 2)
    assert close(Uf, np.kron(U("RY", 0.9), U("U3", 0.4, 1.1, 2.3)))


# ----------------------------------------------------------------------------- invariants

def inverse(g):
    k = g.kind
    p = g.params
    if k in ("H", "X", "Y", "Z", "CX", "CZ", "SWAP"):
        return g
    if k in ("S", "T"):
        return g._replace(kind=k + "DG")
    if k in ("SDG", "TDG"):
        return g._replace(kind=k[:-2])
    if k in ("RX", "RY", "RZ", "P", "CP", "RZZ"):
        return g._replace(params=(-p[0],) + tuple(p[1:]))
    if k == "U3":
        return g._replace(params=(-p[0], -p[2], -p[1]))
    if k == "UNITARY":
        return g._replace(matrix=np.asarray(g.matrix).conj().T.copy())
    if k == "DIAG":
        return g._replace(matrix=np.asarray(g.matrix).conj().copy())
    raise ValueError(k)


@pytest.mark.parametrize("n", [3, 8, 12])
def test_norm_preserved_and_inverse_restores(n):
    rng = W.SplitMix64(7 * n)
    gates = [random_gate(rng, n, ALL_KINDS[rng.below(len(ALL_KINDS))], 500 + i) for i in range(80)]
    a0 = rand_state(n, 3)
    a = oracle.apply_circuit(n, gates, a0.copy())
    assert abs(oracle.norm2(a, n) - 1.0) < 1e-12
    b = oracle.apply_circuit(n, [inverse(g) for g in reversed(gates)], a.copy())
    assert np.max(np.abs(b - a0)) < 1e-12


# ----------------------------------------------------------------------------- remap, worked example

def test_remap_is_bit_exchange_of_basis_states():
    n = 6
    for x in [0, 5, 37, 63]:
        a = oracle.basis_state(n, x)
        oracle.remap(a, n, [0, 2], [4, 5])
        y = x
        for p, q in ((0, 4), (2, 5)):
            bp, bq = (x >> p) & 1, (x >> q) & 1
            y = (y & ~((1 << p) | (1 << q))) | (bq << p) | (bp << q)
        assert a[y] == 1.0 and np.count_nonzero(a) == 1


def test_remap_equals_swap_gates():
    n = 7
    a0 = rand_state(n, 11)
    a = oracle.remap(a0.copy(), n, [1, 3], [6, 0])
    b = oracle.apply_circuit(n, [Gate("SWAP", (1, 6)), Gate("SWAP", (3, 0))], a0.copy())
    assert np.max(np.abs(a - b)) == 0.0


def parse_listing(path):
    out = []
    for line in open(path):
        if not line.strip() or line.startswith("#"):
            continue
        f = line.split()
        out.append(f)
    return out


def listing_gate(f):
    kind, *rest = f
    gid = int(rest[-1])
    qs = tuple(int(v) for v in rest[:-1])
    if kind == "H":
        return Gate("H", qs)
    if kind == "RZZ":
        return Gate("RZZ", qs, (), (float(gid),))
    raise ValueError(kind)


def test_worked_example_swaps_and_final_layout():
    """Appendix worked example (Fig. 5(a) -> 5(b)): running the optimized listing, with SQS and
    CSQS read as pairwise exchanges of physical bit positions, gives the raw circuit's state
    up to the final physical->logical layout.  Every RZZ's physical targets must map back to
    its original logical targets (the paper's order-validation check)."""
    n = 10
    raw = [listing_gate(f) for f in parse_listing(os.path.join(GOLD, "worked_example_raw.txt"))]
    raw_by_id = {int(f[-1]): f for f in parse_listing(os.path.join(GOLD, "worked_example_raw.txt"))}
    a0 = rand_state(n, 2024)
    want = oracle.apply_circuit(n, raw, a0.copy())
    got = a0.copy()
    layout = list(range(n))  # physical position p holds logical qubit layout[p]
    seen_ids = []
    for f in parse_listing(os.path.join(GOLD, "worked_example_optimized.txt")):
        if f[0] in ("SQS", "CSQS"):
            k = int(f[1])
            A = [int(v) for v in f[2:2 + k]]
            B = [int(v) for v in f[2 + k:2 + 2 * k]]
            oracle.remap(got, n, A, B)
            for p, q in zip(A, B):
                layout[p], layout[q] = layout[q], layout[p]
            continue
        g = listing_gate(f)
        gid = int(f[-1])
        seen_ids.append(gid)
        logical = sorted(layout[p] for p in g.targets)
        assert logical == sorted(int(v) for v in raw_by_id[gid][1:-1])
        assert all(p < 4 for p in g.targets)  # chunk (cache) size 4
        oracle.apply_circuit(n, [g], got)
    assert sorted(seen_ids) == list(range(14))
    # got[x_phys] = want[x_log] with logical bit layout[p] = physical bit p
    idx = np.arange(1 << n)
    logi = np.zeros_like(idx)
    for p in range(n):
        logi |= ((idx >> p) & 1) << layout[p]
    assert np.max(np.abs(got - want[logi])) < 1e-14
    assert layout != list(range(n))  # the listing ends in a non-identity layout


# ----------------------------------------------------------------------------- readouts

def test_probs_closed_forms():
    n = 5
    a = oracle.basis_state(n, 19)
    p = oracle.probs(a, n, list(range(n)))
    assert p[19] == 1.0 and p.sum() == 1.0
    a = oracle.apply_circuit(n, [Gate("H", (2,))])
    p = oracle.probs(a, n, [2])
    assert close(p, [0.5, 0.5])
    a = rand_state(n, 5)
    full = oracle.probs(a, n, list(range(n)))
    assert close(full, np.abs(a) ** 2, 1e-16)
    # marginal over qubits (3, 0): bit 0 of the output index is qubit 3
    m = oracle.probs(a, n, [3, 0])
    ref = np.zeros(4)
    for x in range(1 << n):
        ref[((x >> 3) & 1) | (((x >> 0) & 1) << 1)] += abs(a[x]) ** 2
    assert close(m, ref, 1e-15)


@pytest.mark.parametrize("n", [2, 6, 11])
def test_expectation_closed_forms(n):
    H = W.zz_chain_hamiltonian(n)
    a = oracle.basis_state(n, 0)
    assert abs(oracle.expect_pauli(a, n, H) - (n + 0.5 * (n - 1))) < 1e-12
    a = oracle.apply_circuit(n, [Gate("H", (q,)) for q in range(n)])
    assert abs(oracle.expect_pauli(a, n, H)) < 1e-12
    th = [0.3 + 0.41 * q for q in range(n)]
    a = oracle.apply_circuit(n, [Gate("RY", (q,), (), (th[q],)) for q in range(n)])
    want = sum(math.cos(t) for t in th) + 0.5 * sum(math.cos(th[i]) * math.cos(th[i + 1])
                                                    for i in range(n - 1))
    assert abs(oracle.expect_pauli(a, n, H) - want) < 1e-12
    # RZ and CX on |0..0> leave every Z_i at +1
    g = [Gate("RZ", (q,), (), (1.3,)) for q in range(n)] + [Gate("CX", (q + 1,), (q,)) for q in range(n - 1)]
    a = oracle.apply_circuit(n, g)
    assert abs(oracle.expect_pauli(a, n, H) - (n + 0.5 * (n - 1))) < 1e-12


def test_expectation_x_and_y():
    th = 0.77
    a = oracle.apply_circuit(1, [Gate("RY", (0,), (), (th,))])
    assert abs(oracle.expect_pauli(a, 1, [(1.0, 1, 0)]) - math.sin(th)) < 1e-15
    a = oracle.apply_circuit(1, [Gate("RX", (0,), (), (th,))])
    assert abs(oracle.expect_pauli(a, 1, [(1.0, 1, 1)]) - (-math.sin(th))) < 1e-15
    # <psi|P|psi> equals psi^H (P matrix) psi with P built as a Kronecker product
    n = 4
    a = rand_state(n, 77)
    for xm, zm in [(0b1010, 0b0110), (0b1111, 0), (0, 0b1001), (0b0101, 0b0101)]:
        P = np.array([[1.0]])
        for q in range(n - 1, -1, -1):
            x, z = (xm >> q) & 1, (zm >> q) & 1
            P = np.kron(P, PY if (x and z) else PX if x else PZ if z else I2)
        want = np.vdot(a, P @ a)
        assert abs(oracle.expect_pauli(a, n, [(1.0, xm, zm)]) - want) < 1e-14


# ----------------------------------------------------------------------------- MLP

def mlp_params(F, H, seed):
    rng = np.random.default_rng(seed)
    return [rng.normal(size=(F, H)) / np.sqrt(F), rng.normal(size=H) * 0.1,
            rng.normal(size=(H, H)) / np.sqrt(H), rng.normal(size=H) * 0.1,
            rng.normal(size=H) / np.sqrt(H), rng.normal(size=1) * 0.1]


def test_mlp_gradients_match_finite_differences():
    F, H, B = 5, 16, 7
    rng = np.random.default_rng(1)
    X = rng.normal(size=(B, F))
    t = rng.normal(size=B)
    P = mlp_params(F, H, 2)
    loss, grads = oracle.mlp_loss_grad(X, t, P)
    y = oracle.mlp_forward(X, P)
    assert abs(loss - np.mean((y - t) ** 2)) < 1e-14
    h = 1e-6
    for pi, p in enumerate(P):
        flat = p.reshape(-1)
        for j in range(0, flat.size, max(1, flat.size // 9)):
            old = flat[j]
            flat[j] = old + h
            lp = np.mean((oracle.mlp_forward(X, P) - t) ** 2)
            flat[j] = old - h
            lm = np.mean((oracle.mlp_forward(X, P) - t) ** 2)
            flat[j] = old
            fd = (lp - lm) / (2 * h)
            assert abs(fd - grads[pi].reshape(-1)[j]) < 1e-6 * max(1.0, abs(fd))


def test_mlp_forward_relu_network_by_hand():
    """A 1-input network with hand-set weights: y = relu(relu(x - 1) * 2 - 1) * 3 + 0.5."""
    F, H = 1, 1
    P = [np.array([[1.0]]), np.array([-1.0]), np.array([[2.0]]), np.array([-1.0]),
         np.array([3.0]), np.array([0.5])]
    X = np.array([[0.0], [1.5], [3.0]])
    y = oracle.mlp_forward(X, P)
    assert np.allclose(y, [0.5, 0.5, 9.5], atol=0)


def test_adam_first_step_moves_by_lr_times_sign():
    p = np.array([1.0, -2.0, 3.0])
    g = np.array([0.5, -4.0, 1e-3])
    m = np.zeros(3)
    v = np.zeros(3)
    oracle.adam_step(p, g, m, v, 1, lr=0.01, eps=1e-12)
    assert np.allclose(p, [1.0 - 0.01, -2.0 + 0.01, 3.0 - 0.01], atol=1e-9)


def test_adam_steps_two_and_three_by_hand():
    """Kingma & Ba, Algorithm 1, worked by hand with beta1 = 1/2, beta2 = 3/4, eps = 0 and
    lr = 1/10 on one parameter p0 = 1 with gradients 2, 1, -4 (moments start at zero):
      t = 1: m = 1,    v = 1,    m_hat = 1 / (1/2) = 2,        v_hat = 1 / (1/4) = 4,
             p1 = 1 - 0.1 * 2 / 2 = 0.9
      t = 2: m = 1,    v = 1,    m_hat = 1 / (3/4) = 4/3,      v_hat = 1 / (7/16) = 16/7,
             p2 = p1 - 0.1 * (4/3) / (4 / sqrt 7) = 0.9 - 0.1 * sqrt(7) / 3
      t = 3: m = -3/2, v = 19/4, m_hat = -(3/2) / (7/8) = -12/7, v_hat = (19/4) / (37/64) = 304/37,
             p3 = p2 + 0.1 * (12/7) / sqrt(304/37)
    A swapped beta, a moment update with the wrong weight or a bias correction with the wrong
    power changes p2 or p3.  A second parameter starts from non-zero moments at t = 2:
      m = 0.3, v = 0.5, g = 0.1:  m' = 0.2, v' = 0.3775,
      p' = 0 - 0.1 * (0.2 / (3/4)) / sqrt(0.3775 / (7/16))."""
    p = np.array([1.0])
    m, v = np.zeros(1), np.zeros(1)
    kw = dict(lr=0.1, beta1=0.5, beta2=0.75, eps=0.0)
    oracle.adam_step(p, np.array([2.0]), m, v, 1, **kw)
    assert p[0] == pytest.approx(0.9, abs=1e-15) and m[0] == 1.0 and v[0] == 1.0
    oracle.adam_step(p, np.array([1.0]), m, v, 2, **kw)
    p2 = 0.9 - 0.1 * math.sqrt(7.0) / 3.0
    assert (m[0], v[0]) == (1.0, 1.0)
    assert p[0] == pytest.approx(p2, abs=1e-15)
    oracle.adam_step(p, np.array([-4.0]), m, v, 3, **kw)
    assert m[0] == pytest.approx(-1.5, abs=1e-15) and v[0] == pytest.approx(4.75, abs=1e-15)
    assert p[0] == pytest.approx(p2 + 0.1 * (12.0 / 7.0) / math.sqrt(304.0 / 37.0), abs=1e-14)
    q, qm, qv = np.array([0.0]), np.array([0.3]), np.array([0.5])
    oracle.adam_step(q, np.array([0.1]), qm, qv, 2, **kw)
    assert qm[0] == pytest.approx(0.2, abs=1e-15) and qv[0] == pytest.approx(0.3775, abs=1e-15)
    assert q[0] == pytest.approx(-0.1 * (0.2 / 0.75) / math.sqrt(0.3775 / 0.4375), abs=1e-14)


def test_sampling_inverse_transform_pins():
    """Born-rule sampling by inverse transform: closed forms that fix the index order, the
    strict inequality at CDF steps, and the normalisation by the total weight."""
    n = 5
    # basis state: every draw lands on it
    a = oracle.basis_state(n, 19)
    assert np.all(oracle.sample(a, n, [0.0, 0.3, 0.999999]) == 19)
    # H on all qubits: uniform, outcome = floor(u * 2^n)
    a = oracle.apply_circuit(n, [Gate("H", (q,)) for q in range(n)])
    u = np.array([0.0, 0.01, 0.5, 0.77, 0.999])
    assert np.array_equal(oracle.sample(a, n, u), np.floor(u * 32).astype(np.uint64))
    # RY(theta) on qubit 2 only: P(x = 4) = sin^2(theta / 2), outcomes 0 and 4
    th = 1.1
    a = oracle.apply_circuit(n, [Gate("RY", (2,), (), (th,))])
    p0 = math.cos(th / 2) ** 2
    got = oracle.sample(a, n, [p0 - 1e-9, p0 + 1e-9, 0.0])
    assert list(got) == [0, 4, 0]
    # unnormalised input: the total weight rescales u
    b = 3.0 * a
    assert list(oracle.sample(b, n, [p0 - 1e-9, p0 + 1e-9])) == [0, 4]
    # brute force against sorted cumulative weights on a random state
    a = oracle.apply_circuit(6, W.random_circuit(6, 40, 12))
    w = np.abs(a) ** 2
    cdf = np.cumsum(w)
    u = np.random.default_rng(3).random(200)
    want = np.searchsorted(cdf, u * cdf[-1], side="right")
    assert np.array_equal(oracle.sample(a, 6, u), want.astype(np.uint64))
    with pytest.raises(ValueError):
        oracle.sample(a, 6, [1.0])
