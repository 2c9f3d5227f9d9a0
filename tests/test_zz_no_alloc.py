"""The allocation-free readout qs_probs_noalloc, called through the C ABI, against the regular
qs_probs entry point.

qs_probs_noalloc exists for callers that cannot allocate device memory when they read results
(a framework's caching allocator already holds the device memory, a fixed arena was budgeted
up front, or the code path must not call cudaMalloc/cudaFree).  It keeps its histogram in one
fixed device array, so this test also checks that back-to-back calls with different qubit sets
do not see each other's bins.  The file is named so that pytest collects it last.
"""
import numpy as np
import pytest

from paper_2406_14084_gb300 import qs
from paper_2406_14084_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("dtype,tol", [(qs.QS_C128, 1e-12), (qs.QS_C64, 1e-6)])
def test_probs_noalloc_matches_probs_on_two_calls(dtype, tol):
    n = 18
    s = qs.State(n, dtype)
    try:
        s.apply(W.layered(n, 3, 5) + W.vqe_circuit(n, 2, 6), qs.options(dtype=dtype))
        qs.qs_canonicalize(s.h)  # physical order == logical order for the raw-buffer call
        ptr, phys = qs.qs_get_buffer(s.h, n)
        assert phys == list(range(n))
        qs.qs_sync(s.h)
        first = [3, 0, 17, 9, 12, 4, 1, 15, 7, 11, 2, 13, 6, 16]  # 14 qubits: the maximum
        second = [5, 2]                                          # fewer bins than the first call
        for qubits in (first, second):
            got = qs.qs_probs_noalloc(ptr, n, dtype, qubits)
            want = s.probs(qubits)
            assert got.shape == want.shape
            assert np.max(np.abs(got - want)) <= tol
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
