"""The allocation-free readout qs_probs_noalloc, called through the C ABI, against the FP64
oracle's marginal probabilities of the same amplitudes.

qs_probs_noalloc exists for callers that cannot allocate device memory when they read results
(a framework's caching allocator already holds the device memory, a fixed arena was budgeted
up front, or the code path must not call cudaMalloc/cudaFree).  It keeps its histogram in one
fixed device array, so this test also checks that back-to-back calls with different qubit sets
do not see each other's bins.  The amplitudes are copied to the host once and the oracle sums
their squared moduli itself, so a fault shared by the library's two probability entry points
(the bit gather, the shared-memory or global-atomic histogram) shows up here.  The file is
named so that pytest collects it last.
"""
import numpy as np
import pytest

import oracle
from paper_2406_14084_gb300 import qs
from paper_2406_14084_gb300 import workloads as W

pytestmark = pytest.mark.gpu

FOURTEEN = [3, 0, 17, 9, 12, 4, 1, 15, 7, 11, 2, 13, 6, 16]  # the maximum: global-atomic bins


@pytest.mark.parametrize("dtype,tol", [(qs.QS_C128, 1e-12), (qs.QS_C64, 1e-6)])
def test_probs_noalloc_matches_oracle_on_consecutive_calls(dtype, tol):
    n = 18
    s = qs.State(n, dtype)
    try:
        s.apply(W.layered(n, 3, 5) + W.vqe_circuit(n, 2, 6), qs.options(dtype=dtype))
        qs.qs_canonicalize(s.h)  # physical order == logical order for the raw-buffer call
        ptr, phys = qs.qs_get_buffer(s.h, n)
        assert phys == list(range(n))
        qs.qs_sync(s.h)
        amps = s.amplitudes().astype(np.complex128)  # what the device buffer holds
        # 14 bins-bits (global atomics), fewer bins than the call before, none (the norm), and
        # 12 / 13 qubits, the first sizes past the shared-memory histogram
        sets = [FOURTEEN, [5, 2], [], list(range(12)), [17, 0, 8, 3, 14, 1, 10, 5, 12, 6, 2, 15, 9]]
        for qubits in sets + [FOURTEEN]:
            got = qs.qs_probs_noalloc(ptr, n, dtype, qubits)
            want = oracle.probs(amps, n, qubits)
            assert got.shape == want.shape == (1 << len(qubits),)
            assert np.max(np.abs(got - want)) <= tol, qubits
            assert abs(got.sum() - 1.0) <= 1e-5
    finally:
        s.close()


def test_probs_noalloc_rejects_too_many_qubits():
    n = 16
    s = qs.State(n, qs.QS_C64)
    try:
        ptr, _ = qs.qs_get_buffer(s.h, n)
        qs.qs_sync(s.h)
        with pytest.raises(qs.QsError) as e:
            qs.qs_probs_noalloc(ptr, n, qs.QS_C64, list(range(15)))
        assert e.value.status == qs.QS_EINVAL
        assert "2^14" in qs.qs_last_error()
        # still usable afterwards
        got = qs.qs_probs_noalloc(ptr, n, qs.QS_C64, [0])
        assert abs(got[0] - 1.0) <= 1e-6 and abs(got[1]) <= 1e-6
    finally:
        s.close()


def test_probs_noalloc_rejects_host_memory_before_any_launch():
    n = 10
    host = np.zeros(1 << n, dtype=np.complex128)
    host[0] = 1.0
    with pytest.raises(qs.QsError) as e:
        qs.qs_probs_noalloc(host.ctypes.data, n, qs.QS_C128, [0, 1])
    assert e.value.status == qs.QS_EINVAL
    assert "device memory" in qs.qs_last_error() or "device pointer" in qs.qs_last_error()
    # the context is intact: a device buffer still reads correctly
    s = qs.State(n, qs.QS_C128)
    try:
        ptr, _ = qs.qs_get_buffer(s.h, n)
        qs.qs_sync(s.h)
        got = qs.qs_probs_noalloc(ptr, n, qs.QS_C128, [0, 1])
        assert np.array_equal(got, [1.0, 0.0, 0.0, 0.0])
    finally:
        s.close()
