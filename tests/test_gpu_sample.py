"""Measurement sampling (qs_sample) against the oracle's inverse transform.

The GPU result is compared with oracle.sample applied to the same amplitudes (copied back from
the device), so only the summation order of the running weights differs; uniforms whose target
lies within a relative 1e-12 of a step of the cumulative weights are left out (either outcome
is correct there).  Exact cases: a basis state, the uniform state, the logical order after a
plan that leaves a relabelled layout."""
import numpy as np
import pytest

import oracle
from paper_2406_14084_gb300 import qs
from paper_2406_14084_gb300 import workloads as W
from paper_2406_14084_gb300.workloads import Gate

pytestmark = pytest.mark.gpu


def away_from_steps(a, u, rel=1e-12):
    w = np.abs(a.astype(np.complex128)) ** 2
    cdf = np.cumsum(w)
    t = u * cdf[-1]
    i = np.searchsorted(cdf, t, side="right")
    hi = np.abs(cdf[np.minimum(i, cdf.size - 1)] - t)
    lo = np.abs(t - np.where(i > 0, cdf[np.maximum(i - 1, 0)], -1.0))
    return (np.minimum(hi, lo) > rel * cdf[-1])


@pytest.mark.parametrize("dtype", [qs.QS_C64, qs.QS_C128])
@pytest.mark.parametrize("n", [1, 3, 7, 8, 9, 10, 14, 17])  # 8 = one 256-amplitude block
def test_sample_matches_oracle_inverse_transform(dtype, n):
    gates = W.random_circuit(n, 60, 900 + n) if n > 1 else [Gate("U3", (0,), (), (0.4, 0.2, 0.1))]
    u = np.random.default_rng(n).random(3000)
    with qs.State(n, dtype) as s:
        s.apply(gates, qs.options(dtype=dtype))
        got = s.sample(u)
        amps = s.amplitudes().astype(np.complex128)
    want = oracle.sample(amps, n, u)
    ok = away_from_steps(amps, u)
    assert ok.mean() > 0.99
    assert np.array_equal(got[ok], want[ok])
    assert np.all(got < (1 << n))


@pytest.mark.parametrize("dtype", [qs.QS_C64, qs.QS_C128])
def test_sample_exact_cases(dtype):
    n = 20
    with qs.State(n, dtype) as s:
        s.set_basis(0xBEEF)
        assert np.all(s.sample([0.0, 0.5, 0.999999]) == 0xBEEF)
        s.set_basis(0)
        s.apply([Gate("H", (q,)) for q in range(n)], qs.options(dtype=dtype))
        u = np.array([0.0, 0.123, 0.5, 0.9999])
        u = (np.floor(u * (1 << n)) + 0.5) / (1 << n)  # midway inside each outcome's step
        assert np.array_equal(s.sample(u), np.floor(u * (1 << n)).astype(np.uint64))
        assert s.sample([]).size == 0
        with pytest.raises(qs.QsError):
            s.sample([1.0])
        with pytest.raises(qs.QsError):
            s.sample([-0.1])


def test_sample_reads_logical_order_after_relabelling_plan():
    n = 12
    gates = [Gate("X", (0,)), Gate("SWAP", (0, 11)), Gate("H", (3,))]  # |x> = bit 11 set, qubit 3 in +
    with qs.State(n, qs.QS_C128) as s:
        s.apply(gates, qs.options(dtype=qs.QS_C128))
        got = s.sample([0.25, 0.75])
        assert list(got) == [1 << 11, (1 << 11) | (1 << 3)]


def test_sample_rejects_zero_state():
    n = 6
    with qs.State(n, qs.QS_C64) as s:
        qs.qs_copy_from_host(s.h, np.zeros(1 << n, dtype=np.complex64))
        with pytest.raises(qs.QsError):
            s.sample([0.5])


@pytest.mark.parametrize("dtype", [qs.QS_C64, qs.QS_C128])
@pytest.mark.parametrize("n", [9, 13, 18])
def test_sample_top_uniform_skips_trailing_zero_weight(dtype, n):
    """u just below 1 on a state whose upper half has zero weight (Born rule, Eq. 1: an outcome
    of zero probability is never drawn): the draw is the last outcome of positive weight."""
    u = np.array([np.nextafter(1.0, 0.0), 1.0 - 1e-12, 0.25 + 0.5 / (1 << (n - 1))])  # last: mid-step
    with qs.State(n, dtype) as s:
        s.apply([Gate("H", (q,)) for q in range(n - 1)], qs.options(dtype=dtype))
        got = s.sample(u)
        amps = s.amplitudes().astype(np.complex128)
    top = (1 << (n - 1)) - 1
    assert got[0] == top and got[1] == top
    assert np.array_equal(got, oracle.sample(amps, n, u))
