"""ctypes binding of libqs.so (include/qs.h).  Argument marshalling only: every step of the
simulation runs in the library's CUDA kernels.  If the library cannot be built or loaded,
every call raises; there is no CPU fallback.

Function names match the C ABI.  Gates are objects with attributes
``kind, targets, controls, params, matrix`` (see ``workloads.Gate``).
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_lock = threading.Lock()
_lib = None

QS_C64, QS_C128 = 0, 1
QS_OK, QS_EINVAL, QS_ENOMEM, QS_ECUDA, QS_ETIMEOUT, QS_EUNSUPPORTED = range(6)
QS_PLANNER_GREEDY, QS_PLANNER_LEARNED = 0, 1
QS_TC_OFF, QS_TC_TF32X3, QS_TC_BF16X3 = 0, 1, 2
QS_ARITH_FP64, QS_ARITH_DF = 0, 1
QS_SLAB_GATHER, QS_SLAB_REMAP = 0, 1
MAX_TARGETS, MAX_CONTROLS = 7, 8

KINDS = {
    "H": 0, "X": 1, "Y": 2, "Z": 3, "S": 4, "SDG": 5, "T": 6, "TDG": 7, "RX": 8, "RY": 9,
    "RZ": 10, "P": 11, "U3": 12, "CX": 13, "CZ": 14, "CP": 15, "SWAP": 16, "RZZ": 17,
    "UNITARY": 18, "DIAG": 19,
}


class QsError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"qs status {status}: {msg}")
        self.status = status


class QsGate(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("nt", ctypes.c_int32), ("nc", ctypes.c_int32),
                ("t", ctypes.c_int32 * MAX_TARGETS), ("c", ctypes.c_int32 * MAX_CONTROLS),
                ("p", ctypes.c_double * 3), ("m", ctypes.POINTER(ctypes.c_double))]


class QsPauliTerm(ctypes.Structure):
    _fields_ = [("coeff", ctypes.c_double), ("xmask", ctypes.c_uint64), ("zmask", ctypes.c_uint64)]


class QsOptions(ctypes.Structure):
    _fields_ = [("fuse_width", ctypes.c_int32), ("blocking", ctypes.c_int32),
                ("slab_bits", ctypes.c_int32), ("seg_bits", ctypes.c_int32),
                ("slab_mode", ctypes.c_int32), ("planner", ctypes.c_int32), ("tc", ctypes.c_int32),
                ("tc_width", ctypes.c_int32), ("graph", ctypes.c_int32),
                ("diag_bits", ctypes.c_int32), ("dtype", ctypes.c_int32),
                ("stage_bits", ctypes.c_int32), ("fuse_force", ctypes.c_int32),
                ("euler", ctypes.c_int32), ("factor", ctypes.c_int32),
                ("merge_bits", ctypes.c_int32), ("arith", ctypes.c_int32), ("reserved", ctypes.c_int32 * 3)]


class QsPlanInfo(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32), ("passes", ctypes.c_int32), ("remaps", ctypes.c_int32),
                ("unblocked", ctypes.c_int32), ("tc_gates", ctypes.c_int32), ("ops", ctypes.c_int32),
                ("input_gates", ctypes.c_int32), ("slab_bits", ctypes.c_int32),
                ("seg_bits", ctypes.c_int32), ("flops_per_amp", ctypes.c_double),
                ("device_bytes", ctypes.c_int64), ("stages", ctypes.c_int32),
                ("stage_ops", ctypes.c_int32), ("smem_ops", ctypes.c_int32),
                ("stage_bits", ctypes.c_int32), ("learned", ctypes.c_int32),
                ("candidates", ctypes.c_int32), ("chosen", ctypes.c_int32),
                ("judge_state", ctypes.c_int32), ("predicted_ms", ctypes.c_double),
                ("greedy_predicted_ms", ctypes.c_double), ("judge_ms_learned", ctypes.c_double),
                ("judge_ms_greedy", ctypes.c_double), ("using_greedy", ctypes.c_int32),
                ("pad_", ctypes.c_int32)]


QS_PLAN_FEATURES = 28


class QsModelInfo(ctypes.Structure):
    _fields_ = [("nfeat", ctypes.c_int32), ("hidden", ctypes.c_int32), ("nparams", ctypes.c_int32),
                ("steps", ctypes.c_int32), ("ym", ctypes.c_float), ("ys", ctypes.c_float),
                ("last_loss", ctypes.c_float), ("pad_", ctypes.c_int32)]


class QsTrainOptions(ctypes.Structure):
    _fields_ = [("epochs", ctypes.c_int32), ("batch", ctypes.c_int32), ("lr", ctypes.c_float),
                ("fit_norm", ctypes.c_int32), ("seed", ctypes.c_uint64), ("graph", ctypes.c_int32),
                ("reserved", ctypes.c_int32 * 3)]


class QsBatchInfo(ctypes.Structure):
    _fields_ = [("circuits", ctypes.c_int32), ("items", ctypes.c_int32), ("rounds", ctypes.c_int32),
                ("slab_bits", ctypes.c_int32), ("stage_bits", ctypes.c_int32), ("graph", ctypes.c_int32),
                ("state_bytes", ctypes.c_int64), ("last_run_ms", ctypes.c_double),
                ("plan_bytes", ctypes.c_int64)]


class QsStats(ctypes.Structure):
    _fields_ = [("passes", ctypes.c_int64), ("remaps", ctypes.c_int64), ("unblocked", ctypes.c_int64),
                ("tc_gates", ctypes.c_int64), ("plans_applied", ctypes.c_int64),
                ("bytes_moved", ctypes.c_int64), ("pass_ms", ctypes.c_double),
                ("remap_ms", ctypes.c_double), ("unblocked_ms", ctypes.c_double),
                ("tc_ms", ctypes.c_double), ("timed_launches", ctypes.c_int64)]


_vp = ctypes.c_void_p
_i = ctypes.c_int
_u64 = ctypes.c_uint64
_dp = ctypes.POINTER(ctypes.c_double)
_fp = ctypes.POINTER(ctypes.c_float)

# name -> (argtypes); restype is qs_status (int) unless listed in _RESTYPE
_SIGS = {
    "qs_create": [_i, _i, ctypes.POINTER(_vp)],
    "qs_create_from_buffer": [_i, _i, _vp, _vp, ctypes.POINTER(_vp)],
    "qs_destroy": [_vp],
    "qs_set_stream": [_vp, _vp],
    "qs_set_basis": [_vp, _u64],
    "qs_copy_to_host": [_vp, _u64, _u64, _vp],
    "qs_copy_from_host": [_vp, _u64, _u64, _vp],
    "qs_get_buffer": [_vp, ctypes.POINTER(_vp), ctypes.POINTER(_i)],
    "qs_canonicalize": [_vp],
    "qs_sync": [_vp],
    "qs_options_default": [ctypes.POINTER(QsOptions)],
    "qs_fuse": [ctypes.POINTER(QsGate), ctypes.c_size_t, _i, ctypes.POINTER(QsOptions), ctypes.POINTER(_vp)],
    "qs_plan_destroy": [_vp],
    "qs_plan_info_get": [_vp, ctypes.POINTER(QsPlanInfo)],
    "qs_plan_dump": [_vp, ctypes.c_char_p, ctypes.c_size_t, ctypes.POINTER(ctypes.c_size_t)],
    "qs_apply_plan": [_vp, _vp],
    "qs_apply_circuit": [_vp, ctypes.POINTER(QsGate), ctypes.c_size_t, ctypes.POINTER(QsOptions)],
    "qs_remap": [_vp, _i, ctypes.POINTER(_i), ctypes.POINTER(_i)],
    "qs_norm2": [_vp, _dp],
    "qs_probs": [_vp, ctypes.POINTER(_i), _i, _dp],
    "qs_probs_noalloc": [_vp, _i, _i, ctypes.POINTER(_i), _i, _vp, _dp],
    "qs_expect_pauli_sum": [_vp, ctypes.POINTER(QsPauliTerm), ctypes.c_size_t, _dp],
    "qs_sample": [_vp, _dp, ctypes.c_size_t, ctypes.c_void_p],
    "qs_stats": [_vp, ctypes.POINTER(QsStats)],
    "qs_stats_reset": [_vp],
    "qs_set_profiling": [_vp, _i],
    "qs_batch_create": [_i, ctypes.POINTER(_i), ctypes.POINTER(ctypes.POINTER(QsGate)),
                        ctypes.POINTER(ctypes.c_size_t), ctypes.POINTER(QsOptions), ctypes.POINTER(_vp)],
    "qs_apply_batch": [_vp, ctypes.POINTER(QsPauliTerm), ctypes.c_size_t, _dp],
    "qs_batch_tune": [_vp, ctypes.POINTER(QsPauliTerm), ctypes.c_size_t, ctypes.POINTER(_i)],
    "qs_batch_info_get": [_vp, ctypes.POINTER(QsBatchInfo)],
    "qs_batch_destroy": [_vp],
    "qs_train_options_default": [ctypes.POINTER(QsTrainOptions)],
    "qs_model_create": [_i, _u64, ctypes.POINTER(_vp)],
    "qs_model_destroy": [_vp],
    "qs_model_info_get": [_vp, ctypes.POINTER(QsModelInfo)],
    "qs_model_get_params": [_vp, _fp, ctypes.c_size_t],
    "qs_model_set_params": [_vp, _fp, ctypes.c_size_t],
    "qs_model_get_moments": [_vp, _fp, _fp, ctypes.c_size_t],
    "qs_model_get_norm": [_vp, _fp, _fp, _fp, _fp],
    "qs_model_set_norm": [_vp, _fp, _fp, ctypes.c_float, ctypes.c_float],
    "qs_model_predict": [_vp, _fp, ctypes.c_size_t, _fp],
    "qs_model_loss_grad": [_vp, _fp, _fp, ctypes.c_size_t, _fp, _fp],
    "qs_model_train": [_vp, _fp, _fp, ctypes.c_size_t, ctypes.POINTER(QsTrainOptions), _fp],
    "qs_plan_features": [_vp, _fp, ctypes.c_size_t, ctypes.POINTER(ctypes.c_size_t)],
    "qs_plan_profile": [_vp, _vp, _fp, ctypes.c_size_t],
    "qs_fuse_learned": [ctypes.POINTER(QsGate), ctypes.c_size_t, _i, ctypes.POINTER(QsOptions), _vp,
                        ctypes.POINTER(_vp)],
    "qs_set_cost_model": [_vp],
    "qs_last_error": [],
    "qs_version": [],
}
_RESTYPE = {"qs_last_error": ctypes.c_char_p, "qs_version": ctypes.c_char_p, "qs_options_default": None,
            "qs_train_options_default": None}


def library_path() -> str:
    return os.path.join(_HERE, "_build", "libqs.so")


def exported_symbols() -> list:
    return sorted(_SIGS)


def lib(build_if_missing: bool = True):
    """Load libqs.so (building it first when nvcc is available).  Raises if impossible."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = library_path()
        if build_if_missing:
            from . import build as _build
            try:
                path = _build.build()
            except Exception as e:  # no silent fallback: the CUDA library is the product
                if not os.path.exists(path):
                    raise RuntimeError(f"libqs.so is missing and could not be built: {e}") from e
        if not os.path.exists(path):
            raise RuntimeError(f"libqs.so not found at {path}")
        L = ctypes.CDLL(path)
        for name, args in _SIGS.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = _RESTYPE.get(name, ctypes.c_int)
        _lib = L
        return L


def _check(rc: int):
    if rc != QS_OK:
        raise QsError(rc, lib().qs_last_error().decode())


# ----------------------------------------------------------------------------- marshalling

def marshal_gates(gates):
    arr = (QsGate * max(1, len(gates)))()
    keep = []
    for i, g in enumerate(gates):
        s = arr[i]
        s.kind = KINDS[g.kind]
        tg, ct = list(g.targets), list(g.controls)
        if not (1 <= len(tg) <= MAX_TARGETS) or len(ct) > MAX_CONTROLS:
            raise ValueError(f"gate {i}: bad qubit counts")
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
            s.m = m.ctypes.data_as(_dp)
        else:
            s.m = _dp()
    return arr, keep


def options(**kw) -> QsOptions:
    o = QsOptions()
    lib().qs_options_default(ctypes.byref(o))
    for k, v in kw.items():
        if not hasattr(o, k):
            raise KeyError(k)
        setattr(o, k, v)
    return o


# ----------------------------------------------------------------------------- C-ABI mirrors

def qs_version() -> str:
    return lib().qs_version().decode()


def qs_create(n: int, dtype: int = QS_C64):
    h = _vp()
    _check(lib().qs_create(n, dtype, ctypes.byref(h)))
    return h


def qs_create_from_buffer(n: int, dtype: int, dev_ptr: int, stream: int = 0):
    h = _vp()
    _check(lib().qs_create_from_buffer(n, dtype, _vp(dev_ptr), _vp(stream), ctypes.byref(h)))
    return h


def qs_destroy(state):
    _check(lib().qs_destroy(state))


def qs_set_stream(state, stream: int):
    _check(lib().qs_set_stream(state, _vp(stream)))


def qs_set_basis(state, x: int):
    _check(lib().qs_set_basis(state, x))


def qs_copy_to_host(state, n: int, dtype: int, first: int = 0, count: int | None = None, out=None):
    N = 1 << n
    if count is None:
        count = N - first
    npdt = np.complex64 if dtype == QS_C64 else np.complex128
    if out is None:
        out = np.empty(count, dtype=npdt)
    assert out.dtype == npdt and out.flags["C_CONTIGUOUS"] and out.size >= count
    _check(lib().qs_copy_to_host(state, first, count, out.ctypes.data_as(_vp)))
    return out


def qs_copy_from_host(state, host: np.ndarray, first: int = 0):
    assert host.flags["C_CONTIGUOUS"]
    _check(lib().qs_copy_from_host(state, first, host.size, host.ctypes.data_as(_vp)))


def qs_get_buffer(state, n: int):
    p = _vp()
    phys = (_i * n)()
    _check(lib().qs_get_buffer(state, ctypes.byref(p), phys))
    return p.value, list(phys)


def qs_canonicalize(state):
    _check(lib().qs_canonicalize(state))


def qs_sync(state):
    _check(lib().qs_sync(state))


def qs_fuse(gates, n: int, opts: QsOptions | None = None):
    arr, keep = marshal_gates(gates)
    h = _vp()
    _check(lib().qs_fuse(arr, len(gates), n, ctypes.byref(opts) if opts is not None else None,
                         ctypes.byref(h)))
    return h


def qs_plan_destroy(plan):
    _check(lib().qs_plan_destroy(plan))


def qs_fuse_learned(gates, n: int, opts: QsOptions | None, model):
    arr, keep = marshal_gates(gates)
    h = _vp()
    _check(lib().qs_fuse_learned(arr, len(gates), n, ctypes.byref(opts) if opts is not None else None,
                                 model, ctypes.byref(h)))
    return h


def qs_plan_features(plan) -> np.ndarray:
    """Per-step feature rows of a plan, shape (steps, QS_PLAN_FEATURES), float32."""
    nrows = ctypes.c_size_t()
    rc = lib().qs_plan_features(plan, None, 0, ctypes.byref(nrows))  # size query
    if rc not in (QS_OK, QS_EINVAL):
        _check(rc)
    out = np.zeros((nrows.value, QS_PLAN_FEATURES), dtype=np.float32)
    _check(lib().qs_plan_features(plan, _f32(out), nrows.value, ctypes.byref(nrows)))
    return out


def qs_plan_profile(state, plan, steps: int) -> np.ndarray:
    """Apply a plan, returning each step's device time in ms."""
    out = np.zeros(max(1, steps), dtype=np.float32)
    _check(lib().qs_plan_profile(state, plan, _f32(out), out.size))
    return out[:steps]


def _f32(a: np.ndarray):
    assert a.dtype == np.float32 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(_fp)


def qs_train_options(**kw) -> QsTrainOptions:
    o = QsTrainOptions()
    lib().qs_train_options_default(ctypes.byref(o))
    for k, v in kw.items():
        if not hasattr(o, k):
            raise AttributeError(k)
        setattr(o, k, v)
    return o


def qs_model_create(nfeat: int = QS_PLAN_FEATURES, seed: int = 1):
    h = _vp()
    _check(lib().qs_model_create(nfeat, seed, ctypes.byref(h)))
    return h


def qs_model_destroy(model):
    _check(lib().qs_model_destroy(model))


def qs_model_info_get(model) -> dict:
    info = QsModelInfo()
    _check(lib().qs_model_info_get(model, ctypes.byref(info)))
    return {f: getattr(info, f) for f, _ in QsModelInfo._fields_}


def qs_model_get_params(model) -> np.ndarray:
    out = np.zeros(qs_model_info_get(model)["nparams"], dtype=np.float32)
    _check(lib().qs_model_get_params(model, _f32(out), out.size))
    return out


def qs_model_get_moments(model):
    """Adam's first and second moment estimates (m, v), one entry per parameter."""
    k = qs_model_info_get(model)["nparams"]
    m, v = np.zeros(k, dtype=np.float32), np.zeros(k, dtype=np.float32)
    _check(lib().qs_model_get_moments(model, _f32(m), _f32(v), k))
    return m, v


def qs_model_set_params(model, params):
    p = np.ascontiguousarray(params, dtype=np.float32)
    _check(lib().qs_model_set_params(model, _f32(p), p.size))


def qs_model_get_norm(model):
    F = qs_model_info_get(model)["nfeat"]
    mu, sd = np.zeros(F, dtype=np.float32), np.zeros(F, dtype=np.float32)
    ym, ys = ctypes.c_float(), ctypes.c_float()
    _check(lib().qs_model_get_norm(model, _f32(mu), _f32(sd), ctypes.byref(ym), ctypes.byref(ys)))
    return mu, sd, ym.value, ys.value


def qs_model_set_norm(model, mu, sd, ym: float, ys: float):
    mu = np.ascontiguousarray(mu, dtype=np.float32)
    sd = np.ascontiguousarray(sd, dtype=np.float32)
    _check(lib().qs_model_set_norm(model, _f32(mu), _f32(sd), float(ym), float(ys)))


def qs_model_predict(model, X) -> np.ndarray:
    X = np.ascontiguousarray(X, dtype=np.float32)
    y = np.zeros(X.shape[0], dtype=np.float32)
    _check(lib().qs_model_predict(model, _f32(X), X.shape[0], _f32(y)))
    return y


def qs_model_loss_grad(model, X, T):
    X = np.ascontiguousarray(X, dtype=np.float32)
    T = np.ascontiguousarray(T, dtype=np.float32)
    g = np.zeros(qs_model_info_get(model)["nparams"], dtype=np.float32)
    loss = ctypes.c_float()
    _check(lib().qs_model_loss_grad(model, _f32(X), _f32(T), X.shape[0], _f32(g), ctypes.byref(loss)))
    return loss.value, g


def qs_model_train(model, X, T, opts: QsTrainOptions | None = None) -> float:
    X = np.ascontiguousarray(X, dtype=np.float32)
    T = np.ascontiguousarray(T, dtype=np.float32)
    loss = ctypes.c_float()
    _check(lib().qs_model_train(model, _f32(X), _f32(T), X.shape[0],
                                ctypes.byref(opts) if opts is not None else None, ctypes.byref(loss)))
    return loss.value


def qs_set_cost_model(model):
    _check(lib().qs_set_cost_model(model))


def qs_plan_info_get(plan) -> dict:
    info = QsPlanInfo()
    _check(lib().qs_plan_info_get(plan, ctypes.byref(info)))
    return {f: getattr(info, f) for f, _ in QsPlanInfo._fields_}


def qs_plan_dump(plan) -> str:
    need = ctypes.c_size_t()
    _check(lib().qs_plan_dump(plan, None, 0, ctypes.byref(need)))
    buf = ctypes.create_string_buffer(need.value)
    _check(lib().qs_plan_dump(plan, buf, need.value, ctypes.byref(need)))
    return buf.value.decode()


def qs_apply_plan(state, plan):
    _check(lib().qs_apply_plan(state, plan))


def qs_apply_circuit(state, gates, opts: QsOptions | None = None):
    arr, keep = marshal_gates(gates)
    _check(lib().qs_apply_circuit(state, arr, len(gates),
                                  ctypes.byref(opts) if opts is not None else None))


def qs_remap(state, A, B):
    k = len(A)
    a = (_i * max(1, k))(*A)
    b = (_i * max(1, k))(*B)
    _check(lib().qs_remap(state, k, a, b))


def qs_norm2(state) -> float:
    out = ctypes.c_double()
    _check(lib().qs_norm2(state, ctypes.byref(out)))
    return out.value


def qs_probs(state, qubits) -> np.ndarray:
    nq = len(qubits)
    out = np.empty(1 << nq, dtype=np.float64)
    q = (_i * max(1, nq))(*qubits)
    _check(lib().qs_probs(state, q, nq, out.ctypes.data_as(_dp)))
    return out


def qs_probs_noalloc(dev_ptr: int, n: int, dtype: int, qubits, stream: int = 0,
                     out: np.ndarray | None = None) -> np.ndarray:
    """Marginal probabilities of a raw device buffer (physical bit positions) without any
    allocation inside the library; `out` may be a preallocated float64 host array."""
    nq = len(qubits)
    if out is None:
        out = np.empty(1 << nq, dtype=np.float64)
    assert out.dtype == np.float64 and out.flags["C_CONTIGUOUS"] and out.size >= (1 << nq)
    q = (_i * max(1, nq))(*qubits)
    _check(lib().qs_probs_noalloc(_vp(dev_ptr), n, dtype, q, nq, _vp(stream), out.ctypes.data_as(_dp)))
    return out


def qs_sample(state, u) -> np.ndarray:
    """Outcome (logical index) for each uniform u[k] in [0, 1)."""
    u = np.ascontiguousarray(u, dtype=np.float64)
    out = np.zeros(u.size, dtype=np.uint64)
    _check(lib().qs_sample(state, u.ctypes.data_as(_dp), u.size, out.ctypes.data_as(_vp)))
    return out


def qs_expect_pauli_sum(state, terms) -> complex:
    nt = len(terms)
    arr = (QsPauliTerm * max(1, nt))()
    for i, (c, x, z) in enumerate(terms):
        arr[i].coeff, arr[i].xmask, arr[i].zmask = float(c), int(x), int(z)
    out = (ctypes.c_double * 2)()
    _check(lib().qs_expect_pauli_sum(state, arr, nt, out))
    return complex(out[0], out[1])


def _terms_array(terms):
    nt = len(terms)
    arr = (QsPauliTerm * max(1, nt))()
    for i, (c, x, z) in enumerate(terms):
        arr[i].coeff, arr[i].xmask, arr[i].zmask = float(c), int(x), int(z)
    return arr, nt


def qs_batch_create(circuits, opts: QsOptions | None = None):
    """circuits: list of (n, gates).  Returns a batch handle."""
    nc = len(circuits)
    ns = (_i * nc)(*[c[0] for c in circuits])
    keep = []
    ptrs = (ctypes.POINTER(QsGate) * nc)()
    counts = (ctypes.c_size_t * nc)()
    for i, (n, gates) in enumerate(circuits):
        arr, k = marshal_gates(gates)
        keep.append((arr, k))
        ptrs[i] = ctypes.cast(arr, ctypes.POINTER(QsGate))
        counts[i] = len(gates)
    h = _vp()
    _check(lib().qs_batch_create(nc, ns, ptrs, counts, ctypes.byref(opts) if opts is not None else None,
                                 ctypes.byref(h)))
    return h


def qs_apply_batch(batch, terms, ncirc: int) -> np.ndarray:
    arr, nt = _terms_array(terms)
    out = np.empty(ncirc, dtype=np.float64)
    _check(lib().qs_apply_batch(batch, arr, nt, out.ctypes.data_as(_dp)))
    return out


def qs_batch_tune(batch, terms) -> int:
    arr, nt = _terms_array(terms)
    chosen = _i()
    _check(lib().qs_batch_tune(batch, arr, nt, ctypes.byref(chosen)))
    return chosen.value


def qs_batch_info_get(batch) -> dict:
    info = QsBatchInfo()
    _check(lib().qs_batch_info_get(batch, ctypes.byref(info)))
    return {f: getattr(info, f) for f, _ in QsBatchInfo._fields_}


def qs_batch_destroy(batch):
    _check(lib().qs_batch_destroy(batch))


def qs_stats(state) -> dict:
    s = QsStats()
    _check(lib().qs_stats(state, ctypes.byref(s)))
    return {f: getattr(s, f) for f, _ in QsStats._fields_}


def qs_stats_reset(state):
    _check(lib().qs_stats_reset(state))


def qs_set_profiling(state, on: bool):
    _check(lib().qs_set_profiling(state, 1 if on else 0))


def qs_last_error() -> str:
    return lib().qs_last_error().decode()


# ----------------------------------------------------------------------------- convenience

class State:
    """Owning wrapper around a qs_state handle."""

    def __init__(self, n: int, dtype: int = QS_C64):
        self.n, self.dtype = n, dtype
        self.h = qs_create(n, dtype)

    def close(self):
        if self.h:
            qs_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def apply(self, gates, opts=None):
        qs_apply_circuit(self.h, gates, opts)
        return self

    def amplitudes(self) -> np.ndarray:
        return qs_copy_to_host(self.h, self.n, self.dtype)

    def probs(self, qubits):
        return qs_probs(self.h, qubits)

    def expect(self, terms):
        return qs_expect_pauli_sum(self.h, terms)

    def sample(self, u):
        return qs_sample(self.h, u)

    def norm2(self):
        return qs_norm2(self.h)

    def set_basis(self, x: int):
        qs_set_basis(self.h, x)
