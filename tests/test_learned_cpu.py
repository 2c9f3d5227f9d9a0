"""Host-side parts of the learned planner: plan features, forced fusion, candidate grid.

No device work: qs_fuse and qs_plan_features run on the host."""
import numpy as np
import pytest

from paper_2406_14084_gb300 import costmodel
from paper_2406_14084_gb300 import qs
from paper_2406_14084_gb300 import workloads as W
from paper_2406_14084_gb300.workloads import Gate

F = qs.QS_PLAN_FEATURES


def features(gates, n, **kw):
    p = qs.qs_fuse(gates, n, qs.options(**kw))
    try:
        return qs.qs_plan_features(p), qs.qs_plan_info_get(p)
    finally:
        qs.qs_plan_destroy(p)


def test_one_row_per_step_and_kind_one_hot():
    g = W.layered(20, 6, 11)
    X, info = features(g, 20, dtype=qs.QS_C128)
    assert X.shape == (info["passes"] + info["remaps"] + info["unblocked"] + info["tc_gates"], F)
    assert np.all(X[:, 0] == 20) and np.all(X[:, 1] == 1)
    assert np.all(X[:, 2:6].sum(axis=1) == 1)
    assert np.all(X[:, 12] == info["stage_bits"])


def test_single_hadamard_is_one_real_one_qubit_op():
    X, _ = features([Gate("H", (3,))], 16, dtype=qs.QS_C64)
    assert X.shape == (1, F)
    row = X[0]
    assert row[2] == 1                           # slab pass
    assert row[17] == 1 and row[16] == 0         # real 2x2 (H) in a register stage
    assert row[26] == pytest.approx(4.0)         # 4 real FMAs per amplitude
    assert row[27] == 1


def test_controlled_phase_counts_quarter_of_amplitudes():
    X, _ = features([Gate("CP", (0, 1), (), (0.3,))], 16, dtype=qs.QS_C64, fuse_width=0)
    assert X.shape[0] == 1
    assert X[0, 19] + X[0, 20] + X[0, 24] >= 1   # a phase / diagonal op
    assert X[0, 26] <= 4.0


def test_unblocked_step_features():
    X, info = features([Gate("U3", (5,), (), (0.1, 0.2, 0.3))], 12, dtype=qs.QS_C128, blocking=0, fuse_width=0)
    assert info["unblocked"] == 1
    assert X[0, 4] == 1 and X[0, 6] == 1
    assert X[0, 22] == 1 and X[0, 23] == 2 and X[0, 26] == pytest.approx(8.0)


def test_forced_fusion_builds_wider_gates():
    g = W.layered(16, 8, 5)
    base = qs.qs_plan_info_get(p := qs.qs_fuse(g, 16, qs.options(dtype=qs.QS_C128, fuse_width=4)))
    qs.qs_plan_destroy(p)
    X, forced = features(g, 16, dtype=qs.QS_C128, fuse_width=4, fuse_force=1)
    assert forced["ops"] < base["ops"]
    assert X[:, 27].max() >= 3


def test_candidate_grid_matches_planner_limits():
    for dt, bmax, rb in ((qs.QS_C64, 13, 5), (qs.QS_C128, 12, 4)):
        grid = costmodel.candidate_options(dt, 30)
        assert len(grid) == 2 * 5 * 3 * 2 * 3
        assert {o["slab_bits"] for o in grid} == {bmax - 2, bmax - 1, bmax}
        assert {o["stage_bits"] for o in grid} == {rb - 1, rb}
        assert {o["merge_bits"] for o in grid} == {6, 8, 10}
        for o in grid:
            p = qs.qs_fuse(W.qft(18), 18, qs.options(dtype=dt, **o))
            assert qs.qs_plan_info_get(p)["slab_bits"] <= o["slab_bits"]
            qs.qs_plan_destroy(p)


def test_learned_fuse_without_model_is_greedy():
    g = W.qft(18)
    p = qs.qs_fuse_learned(g, 18, qs.options(dtype=qs.QS_C128), None)
    q = qs.qs_fuse(g, 18, qs.options(dtype=qs.QS_C128))
    try:
        a, b = qs.qs_plan_info_get(p), qs.qs_plan_info_get(q)
        assert a["learned"] == 0 and a["chosen"] == -1 and a["judge_state"] == 2
        assert a["passes"] == b["passes"] and a["ops"] == b["ops"]
        assert np.array_equal(qs.qs_plan_features(p), qs.qs_plan_features(q))
    finally:
        qs.qs_plan_destroy(p)
        qs.qs_plan_destroy(q)


def test_planner_learned_option_without_model_falls_back():
    qs.qs_set_cost_model(None)
    p = qs.qs_fuse(W.qft(14), 14, qs.options(dtype=qs.QS_C64, planner=qs.QS_PLANNER_LEARNED))
    try:
        assert qs.qs_plan_info_get(p)["chosen"] == -1
    finally:
        qs.qs_plan_destroy(p)


def test_train_options_defaults():
    o = qs.qs_train_options()
    assert o.epochs > 0 and o.batch > 0 and o.lr > 0 and o.fit_norm == 1
