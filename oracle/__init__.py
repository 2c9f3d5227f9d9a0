"""FP64 CPU oracle for the state-vector simulator (test infrastructure only).

Only the tests, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline leg may import
this package.  The product library never imports, links or calls it, and it imports nothing
from the product package: gates arrive as plain objects with the attributes
``kind, targets, controls, params, matrix`` (the seeded generators produce those).

The arithmetic lives in ``qs_oracle.c`` (plain loops, one gate at a time, no fusion; see the
header comment there for the paper passages each function follows).  This module compiles it
with gcc on first use and wraps it with ctypes.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "libqs_oracle.so")
_lock = threading.Lock()
_lib = None

MAX_TARGETS = 12
MAX_CONTROLS = 8

KINDS = {
    "H": 0, "X": 1, "Y": 2, "Z": 3, "S": 4, "SDG": 5, "T": 6, "TDG": 7, "RX": 8, "RY": 9,
    "RZ": 10, "P": 11, "U3": 12, "CX": 13, "CZ": 14, "CP": 15, "SWAP": 16, "RZZ": 17,
    "UNITARY": 18, "DIAG": 19,
}


class _Gate(ctypes.Structure):
    _fields_ = [
        ("kind", ctypes.c_int32),
        ("nt", ctypes.c_int32),
        ("nc", ctypes.c_int32),
        ("t", ctypes.c_int32 * MAX_TARGETS),
        ("c", ctypes.c_int32 * MAX_CONTROLS),
        ("p", ctypes.c_double * 3),
        ("m", ctypes.POINTER(ctypes.c_double)),
    ]


def build(force: bool = False) -> str:
    """Compile qs_oracle.c into a shared library (OpenMP when the compiler has it)."""
    src = os.path.join(_HERE, "qs_oracle.c")
    if (not force and os.path.exists(_SO)
            and os.path.getmtime(_SO) >= os.path.getmtime(src)
            and os.path.getmtime(_SO) >= os.path.getmtime(os.path.join(_HERE, "qs_oracle.h"))):
        return _SO
    os.makedirs(_BUILD, exist_ok=True)
    tmp = _SO + f".tmp{os.getpid()}"
    base = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", src, "-o", tmp, "-lm"]
    try:
        subprocess.run(base[:4] + ["-fopenmp"] + base[4:], check=True, capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True, capture_output=True)
    os.replace(tmp, _SO)
    return _SO


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = ctypes.CDLL(build())
            dp = ctypes.POINTER(ctypes.c_double)
            L.or_apply_circuit.argtypes = [dp, ctypes.c_int, ctypes.POINTER(_Gate), ctypes.c_int]
            L.or_apply_gate.argtypes = [dp, ctypes.c_int, ctypes.POINTER(_Gate)]
            L.or_gate_matrix.argtypes = [ctypes.POINTER(_Gate), dp]
            L.or_init_basis.argtypes = [dp, ctypes.c_int, ctypes.c_uint64]
            L.or_init_basis.restype = None
            L.or_set_threads.argtypes = [ctypes.c_int]
            L.or_set_threads.restype = None
            L.or_get_threads.argtypes = []
            L.or_remap.argtypes = [dp, ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_int),
                                   ctypes.POINTER(ctypes.c_int)]
            L.or_norm2.argtypes = [dp, ctypes.c_int]
            L.or_norm2.restype = ctypes.c_double
            L.or_probs.argtypes = [dp, ctypes.c_int, ctypes.POINTER(ctypes.c_int), ctypes.c_int, dp]
            L.or_sample.argtypes = [dp, ctypes.c_int, dp, ctypes.c_int64, ctypes.c_void_p]
            u64p = ctypes.POINTER(ctypes.c_uint64)
            L.or_expect_pauli.argtypes = [dp, ctypes.c_int, dp, u64p, u64p, ctypes.c_int, dp]
            L.or_circuit_unitary.argtypes = [ctypes.POINTER(_Gate), ctypes.c_int, ctypes.c_int, dp]
            L.or_mlp_forward.argtypes = [dp, ctypes.c_int, ctypes.c_int, ctypes.c_int] + [dp] * 7
            L.or_mlp_loss_grad.argtypes = [dp, dp, ctypes.c_int, ctypes.c_int, ctypes.c_int] + [dp] * 13
            L.or_adam_step.argtypes = [dp, dp, dp, dp, ctypes.c_int64, ctypes.c_int, ctypes.c_double,
                                       ctypes.c_double, ctypes.c_double, ctypes.c_double]
            L.or_adam_step.restype = None
            _lib = L
    return _lib


def _dptr(a: np.ndarray):
    assert a.dtype == np.float64 or a.dtype == np.complex128
    assert a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _marshal(gates):
    """Gate objects -> ctypes array (keeps matrix buffers alive in the returned tuple)."""
    arr = (_Gate * max(1, len(gates)))()
    keep = []
    for i, g in enumerate(gates):
        s = arr[i]
        s.kind = KINDS[g.kind]
        tg = list(g.targets)
        ct = list(g.controls)
        if not (1 <= len(tg) <= MAX_TARGETS) or len(ct) > MAX_CONTROLS:
            raise ValueError(f"gate {g.kind}: bad qubit counts")
        s.nt, s.nc = len(tg), len(ct)
        for j, q in enumerate(tg):
            s.t[j] = q
        for j, q in enumerate(ct):
            s.c[j] = q
        p = list(g.params) + [0.0] * (3 - len(g.params))
        for j in range(3):
            s.p[j] = float(p[j])
        if g.matrix is not None:
            m = np.ascontiguousarray(np.asarray(g.matrix, dtype=np.complex128))
            keep.append(m)
            s.m = _dptr(m)
        else:
            s.m = ctypes.POINTER(ctypes.c_double)()
    return arr, keep


def basis_state(n: int, x: int = 0) -> np.ndarray:
    a = np.empty(1 << n, dtype=np.complex128)
    lib().or_init_basis(_dptr(a), n, x)
    return a


def set_basis(state: np.ndarray, n: int, x: int = 0) -> np.ndarray:
    """Overwrite ``state`` (2^n complex128) with the basis state |x>, in place."""
    assert state.dtype == np.complex128 and state.shape == (1 << n,)
    lib().or_init_basis(_dptr(state), n, x)
    return state


def apply_circuit(n: int, gates, state: np.ndarray | None = None) -> np.ndarray:
    """Apply the gates one at a time (no fusion) to ``state`` (default |0..0>), in place."""
    if state is None:
        state = basis_state(n, 0)
    assert state.dtype == np.complex128 and state.shape == (1 << n,)
    if len(gates) == 0:
        return state
    arr, keep = _marshal(gates)
    rc = lib().or_apply_circuit(_dptr(state), n, arr, len(gates))
    if rc:
        raise ValueError(f"oracle rejected the circuit (code {rc})")
    return state


def gate_matrix(g) -> np.ndarray:
    k = len(g.targets)
    U = np.empty((1 << k, 1 << k), dtype=np.complex128)
    arr, keep = _marshal([g])
    rc = lib().or_gate_matrix(arr, _dptr(U))
    if rc:
        raise ValueError(f"oracle rejected the gate (code {rc})")
    return U


def circuit_unitary(gates, k: int) -> np.ndarray:
    """Unitary of a gate sequence on qubits 0..k-1 (column j = sequence applied to |j>)."""
    U = np.empty((1 << k, 1 << k), dtype=np.complex128)
    arr, keep = _marshal(gates)
    rc = lib().or_circuit_unitary(arr, len(gates), k, _dptr(U))
    if rc:
        raise ValueError(f"oracle rejected the circuit (code {rc})")
    return U


def remap(state: np.ndarray, n: int, A, B) -> np.ndarray:
    """Exchange index bits A[j] <-> B[j] pairwise, in place (Eq. 4)."""
    k = len(A)
    a = (ctypes.c_int * max(1, k))(*A)
    b = (ctypes.c_int * max(1, k))(*B)
    rc = lib().or_remap(_dptr(state), n, k, a, b)
    if rc:
        raise ValueError("bad remap")
    return state


def norm2(state: np.ndarray, n: int) -> float:
    return lib().or_norm2(_dptr(state), n)


def probs(state: np.ndarray, n: int, qubits) -> np.ndarray:
    nq = len(qubits)
    out = np.empty(1 << nq, dtype=np.float64)
    q = (ctypes.c_int * max(1, nq))(*qubits)
    rc = lib().or_probs(_dptr(state), n, q, nq, _dptr(out))
    if rc:
        raise ValueError("bad probs request")
    return out


def sample(state: np.ndarray, n: int, u) -> np.ndarray:
    """Outcome per uniform u[k] in [0, 1): smallest x whose running sum of |a_y|^2 (y <= x)
    exceeds u[k] times the total (inverse transform sampling of the Born distribution)."""
    u = np.ascontiguousarray(u, dtype=np.float64)
    out = np.empty(u.size, dtype=np.uint64)
    rc = lib().or_sample(_dptr(state), n, _dptr(u), u.size, out.ctypes.data_as(ctypes.c_void_p))
    if rc:
        raise ValueError("bad sample request")
    return out


def expect_pauli(state: np.ndarray, n: int, terms) -> complex:
    """sum_t c_t <psi|P_t|psi>; terms = [(coeff, xmask, zmask)], Y sets both masks."""
    nt = len(terms)
    c = np.array([t[0] for t in terms], dtype=np.float64)
    xm = np.array([t[1] for t in terms], dtype=np.uint64)
    zm = np.array([t[2] for t in terms], dtype=np.uint64)
    out = np.zeros(2, dtype=np.float64)
    u64p = ctypes.POINTER(ctypes.c_uint64)
    rc = lib().or_expect_pauli(_dptr(state), n, _dptr(c), xm.ctypes.data_as(u64p),
                               zm.ctypes.data_as(u64p), nt, _dptr(out))
    if rc:
        raise ValueError("bad Pauli term")
    return complex(out[0], out[1])


# ----------------------------------------------------------------------------- MLP (FP64)

def mlp_forward(X, params):
    W1, b1, W2, b2, W3, b3 = [np.ascontiguousarray(p, dtype=np.float64) for p in params]
    X = np.ascontiguousarray(X, dtype=np.float64)
    B, F = X.shape
    H = W1.shape[1]
    y = np.empty(B, dtype=np.float64)
    rc = lib().or_mlp_forward(_dptr(X), B, F, H, _dptr(W1), _dptr(b1), _dptr(W2), _dptr(b2),
                              _dptr(W3), _dptr(b3), _dptr(y))
    assert rc == 0
    return y


def mlp_loss_grad(X, target, params):
    W1, b1, W2, b2, W3, b3 = [np.ascontiguousarray(p, dtype=np.float64) for p in params]
    X = np.ascontiguousarray(X, dtype=np.float64)
    t = np.ascontiguousarray(target, dtype=np.float64)
    B, F = X.shape
    H = W1.shape[1]
    grads = [np.empty_like(p) for p in (W1, b1, W2, b2, W3, b3)]
    loss = np.zeros(1)
    rc = lib().or_mlp_loss_grad(_dptr(X), _dptr(t), B, F, H, _dptr(W1), _dptr(b1), _dptr(W2),
                                _dptr(b2), _dptr(W3), _dptr(b3), *[_dptr(g) for g in grads],
                                _dptr(loss))
    assert rc == 0
    return float(loss[0]), grads


def adam_step(p, g, m, v, t, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8):
    """In-place Adam update of flat FP64 arrays p, m, v with gradient g (step t >= 1)."""
    for a in (p, g, m, v):
        assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    lib().or_adam_step(_dptr(p), _dptr(g), _dptr(m), _dptr(v), p.size, t, lr, beta1, beta2, eps)


def set_threads(t: int) -> None:
    """Thread count of the oracle's OpenMP loops (results are identical at any count)."""
    lib().or_set_threads(int(t))


def get_threads() -> int:
    return int(lib().or_get_threads())
