"""Cost-model network kernels against the FP64 oracle MLP.

Forward to 1e-5 (relative to the output scale), gradients to 1e-4 relative (norm-wise and for
every entry above 1% of the largest), one and three Adam steps (parameters and moments) against
the oracle's Adam steps, and a training run that fits a known function."""
import numpy as np
import pytest

import oracle
from paper_2406_14084_gb300 import qs

pytestmark = pytest.mark.gpu

H = 128


def split(flat, F):
    o = 0
    out = []
    for shape in ((F, H), (H,), (H, H), (H,), (H,), (1,)):
        size = int(np.prod(shape))
        out.append(flat[o:o + size].reshape(shape).astype(np.float64))
        o += size
    assert o == flat.size
    return out


def random_model(F, seed):
    m = qs.qs_model_create(F, seed)
    rng = np.random.default_rng(seed)
    p = qs.qs_model_get_params(m)
    # non-zero biases so every bias path is exercised
    p = p + rng.normal(0, 0.05, p.size).astype(np.float32)
    qs.qs_model_set_params(m, p)
    return m, p


@pytest.mark.parametrize("F,B", [(qs.QS_PLAN_FEATURES, 100), (5, 31), (32, 64)])
def test_forward_matches_oracle(F, B):
    m, p = random_model(F, 3 + F)
    try:
        X = np.random.default_rng(F).normal(0, 1, (B, F)).astype(np.float32)
        got = qs.qs_model_predict(m, X)
        want = oracle.mlp_forward(X.astype(np.float64), split(p, F))
        scale = max(1.0, float(np.max(np.abs(want))))
        assert np.max(np.abs(got - want)) <= 1e-5 * scale
    finally:
        qs.qs_model_destroy(m)


@pytest.mark.parametrize("F,B", [(qs.QS_PLAN_FEATURES, 96), (7, 45)])
def test_gradients_match_oracle(F, B):
    m, p = random_model(F, 11 + F)
    try:
        rng = np.random.default_rng(B)
        X = rng.normal(0, 1, (B, F)).astype(np.float32)
        T = rng.normal(0, 1, B).astype(np.float32)
        loss, g = qs.qs_model_loss_grad(m, X, T)
        wl, wg = oracle.mlp_loss_grad(X.astype(np.float64), T.astype(np.float64), split(p, F))
        wg = np.concatenate([a.ravel() for a in wg])
        assert abs(loss - wl) <= 1e-5 * max(1.0, abs(wl))
        assert np.linalg.norm(g - wg) <= 1e-4 * np.linalg.norm(wg)
        big = np.abs(wg) > 0.01 * np.max(np.abs(wg))
        assert np.all(np.abs(g[big] - wg[big]) <= 1e-4 * np.abs(wg[big]) + 1e-6 * np.max(np.abs(wg)))
    finally:
        qs.qs_model_destroy(m)


def test_one_adam_step_matches_oracle():
    F, B, lr = 9, 64, 1e-2
    m, p = random_model(F, 5)
    try:
        rng = np.random.default_rng(9)
        X = rng.normal(0, 1, (B, F)).astype(np.float32)
        T = rng.normal(0, 1, B).astype(np.float32)
        _, g = oracle.mlp_loss_grad(X.astype(np.float64), T.astype(np.float64), split(p, F))
        g = np.concatenate([a.ravel() for a in g])
        want = p.astype(np.float64).copy()
        mom, vel = np.zeros_like(want), np.zeros_like(want)
        oracle.adam_step(want, g, mom, vel, 1, lr=lr)
        # one epoch of one full batch: one Adam step; rows are shuffled but the batch is all of them
        qs.qs_model_train(m, X, T, qs.qs_train_options(epochs=1, batch=B, lr=lr, fit_norm=0, graph=0))
        got = qs.qs_model_get_params(m)
        # Adam's first step moves a parameter by lr * g / (|g| + eps), about lr * sign(g); where
        # |g| is near eps the FP32 sum order decides, so compare the clearly determined moves
        sure = np.abs(g) > 1e-4 * np.max(np.abs(g))
        assert np.max(np.abs((got - p) - (want - p))[sure]) <= 2e-4 * lr + 1e-6
        assert np.max(np.abs(got - p)) <= lr * (1 + 1e-3)
        assert qs.qs_model_info_get(m)["steps"] == 1
    finally:
        qs.qs_model_destroy(m)


def test_three_adam_steps_match_oracle():
    """Three full-batch Adam steps (Kingma & Ba, Algorithm 1): parameters and both moment
    estimates against the oracle's FP64 steps, each taken at the oracle's own gradient of the
    current parameters.  From the second step on the update depends on beta1, beta2 and both
    bias corrections, which the first step does not."""
    F, B, lr = 9, 64, 1e-2
    m, p = random_model(F, 17)
    try:
        rng = np.random.default_rng(19)
        X = rng.normal(0, 1, (B, F)).astype(np.float32)
        T = rng.normal(0, 1, B).astype(np.float32)
        want = p.astype(np.float64).copy()
        mom, vel = np.zeros_like(want), np.zeros_like(want)
        grads = []
        for t in (1, 2, 3):
            _, g = oracle.mlp_loss_grad(X.astype(np.float64), T.astype(np.float64), split(want, F))
            g = np.concatenate([a.ravel() for a in g])
            grads.append(g)
            oracle.adam_step(want, g, mom, vel, t, lr=lr, beta1=0.9, beta2=0.999, eps=1e-8)
        qs.qs_model_train(m, X, T, qs.qs_train_options(epochs=3, batch=B, lr=lr, fit_norm=0, graph=0))
        assert qs.qs_model_info_get(m)["steps"] == 3
        got = qs.qs_model_get_params(m).astype(np.float64)
        gm, gv = (a.astype(np.float64) for a in qs.qs_model_get_moments(m))
        gmax = max(float(np.max(np.abs(g))) for g in grads)
        # moments are sums of FP32 gradients: compare against the gradient scale
        assert np.max(np.abs(gm - mom)) <= 1e-4 * gmax
        assert np.max(np.abs(gv - vel)) <= 1e-4 * gmax * gmax + 1e-3 * np.max(np.abs(vel))
        # parameter moves where every step's gradient is clearly above the FP32 sum noise (units
        # whose ReLU is off for every row have exactly zero gradients and do not move)
        sure = np.all([np.abs(g) > 1e-3 * gmax for g in grads], axis=0)
        zero = np.all([g == 0 for g in grads], axis=0)
        assert sure.sum() > 0.25 * sure.size
        assert np.max(np.abs((got - p) - (want - p))[sure]) <= 1e-3 * lr
        assert np.max(np.abs(got - p)[zero], initial=0.0) <= 1e-3 * lr
        # Adam moves each parameter by at most about lr per step
        assert np.max(np.abs(got - p)) <= 3 * lr * (1 + 1e-3)
    finally:
        qs.qs_model_destroy(m)


def test_training_fits_a_smooth_function():
    F, N = 6, 4096
    rng = np.random.default_rng(1)
    X = rng.uniform(-1, 1, (N, F)).astype(np.float32)
    y = (np.sin(2 * X[:, 0]) + X[:, 1] * X[:, 2] + 0.5 * np.abs(X[:, 3]) + 3.0).astype(np.float32)
    m = qs.qs_model_create(F, 2)
    try:
        before = float(np.mean((qs.qs_model_predict(m, X) - y) ** 2))
        loss = qs.qs_model_train(m, X, y, qs.qs_train_options(epochs=80, batch=128, lr=2e-3, seed=4))
        after = float(np.mean((qs.qs_model_predict(m, X) - y) ** 2))
        assert after < 0.05 * float(np.var(y)) and after < 0.01 * before
        assert loss < 0.05  # standardised space
        info = qs.qs_model_info_get(m)
        assert info["steps"] == 80 * (N // 128)
        # graph replay and eager epochs give the same parameters
        m2 = qs.qs_model_create(F, 2)
        qs.qs_model_train(m2, X, y, qs.qs_train_options(epochs=3, batch=128, lr=2e-3, seed=4, graph=0))
        m3 = qs.qs_model_create(F, 2)
        qs.qs_model_train(m3, X, y, qs.qs_train_options(epochs=3, batch=128, lr=2e-3, seed=4, graph=1))
        assert np.array_equal(qs.qs_model_get_params(m2), qs.qs_model_get_params(m3))
        qs.qs_model_destroy(m2)
        qs.qs_model_destroy(m3)
    finally:
        qs.qs_model_destroy(m)


def test_standardisation_is_applied():
    F, B = 4, 40
    m, p = random_model(F, 21)
    try:
        rng = np.random.default_rng(2)
        X = rng.normal(3, 2, (B, F)).astype(np.float32)
        mu = np.array([3, 3, 3, 3], np.float32)
        sd = np.array([2, 2, 2, 2], np.float32)
        qs.qs_model_set_norm(m, mu, sd, 1.5, 4.0)
        got = qs.qs_model_predict(m, X)
        want = oracle.mlp_forward(((X - mu) / sd).astype(np.float64), split(p, F)) * 4.0 + 1.5
        assert np.max(np.abs(got - want)) <= 1e-5 * max(1.0, float(np.max(np.abs(want))))
    finally:
        qs.qs_model_destroy(m)


def test_bad_arguments():
    with pytest.raises(qs.QsError):
        qs.qs_model_create(33, 1)
    m = qs.qs_model_create(4, 1)
    try:
        with pytest.raises(qs.QsError):
            qs.qs_model_set_params(m, np.zeros(3, np.float32))
        with pytest.raises(qs.QsError):
            qs.qs_model_set_norm(m, np.zeros(4, np.float32), np.zeros(4, np.float32), 0.0, 1.0)
        with pytest.raises(qs.QsError):
            qs.qs_model_train(m, np.full((8, 4), np.nan, np.float32), np.zeros(8, np.float32))
    finally:
        qs.qs_model_destroy(m)
