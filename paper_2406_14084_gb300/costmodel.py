"""Training data and training for the learned planner's cost model.

The data are timings the simulator generates itself: random circuits of the shapes the planner
meets (layered U3 + CZ brickwork, QFT, uniform random gate lists, hardware-efficient ansatz)
are planned with options drawn from the learned planner's candidate grid; every step of every
plan is described by ``qs_plan_features`` and timed on the device by ``qs_plan_profile``
(CUDA events around each launch, best of ``repeats`` applies).  The target of a step is
``ln(ms) - (n - 20) ln 2``.  Training runs the library's own forward / backward / Adam kernels
(``qs_model_train``).  This module only orchestrates library calls.
"""
from __future__ import annotations

import math
import time

import numpy as np

from . import qs
from . import workloads as W

FUSES = [(1, 0), (2, 0), (3, 1), (4, 1), (5, 1)]


def max_slab_bits(dtype: int) -> int:
    return 13 if dtype == qs.QS_C64 else 12


def candidate_options(dtype: int, n: int):
    """The learned planner's grid (Euler split x fusion width / forced fusion x slab bits x stage
    bits x stage-table condition bits)."""
    bmax = min(max_slab_bits(dtype), n)
    rbmax = 5 if dtype == qs.QS_C64 else 4
    out = []
    for eu in (1, 2):
        for fw, force in FUSES:
            for sb in range(max(bmax - 2, 6), bmax + 1):
                for rb in (rbmax - 1, rbmax):
                    for mb in (6, 8, 10):
                        out.append(dict(fuse_width=fw, fuse_force=force, slab_bits=sb, stage_bits=rb, euler=eu,
                                        merge_bits=mb))
    return out


def random_circuit_family(rng: W.SplitMix64, n: int):
    """One circuit of a random family and size, as (name, gates)."""
    kind = rng.below(4)
    if kind == 0:
        depth = 2 + rng.below(14)
        return f"layered{depth}", W.layered(n, depth, rng.next_u64())
    if kind == 1:
        return "qft", W.qft(n)
    if kind == 2:
        ng = 40 + rng.below(400)
        return f"random{ng}", W.random_circuit(n, ng, rng.next_u64())
    layers = 1 + rng.below(6)
    return f"ansatz{layers}", W.vqe_circuit(n, layers, rng.next_u64())


def collect(target_rows: int, seed: int, nmin: int, nmax: int, dtypes=(qs.QS_C64, qs.QS_C128),
            repeats: int = 2, time_budget_s: float | None = None, log=None):
    """Time plan steps until ``target_rows`` rows (or the time budget) are reached.

    Returns (X float32 [rows, QS_PLAN_FEATURES], y float32 [rows], meta list)."""
    rng = W.SplitMix64(seed)
    X, Y, meta = [], [], []
    rows = 0
    states = {}
    t0 = time.perf_counter()
    try:
        while rows < target_rows:
            if time_budget_s is not None and time.perf_counter() - t0 > time_budget_s:
                break
            dtype = dtypes[rng.below(len(dtypes))]
            lo = max(nmin, 25) if dtype == qs.QS_C64 else nmin  # keep states above L2 size
            n = lo + rng.below(nmax - lo + 1)
            name, gates = random_circuit_family(rng, n)
            grid = candidate_options(dtype, n)
            # a quarter of the plans with the greedy planner's own options, the rest from the grid
            o = {} if rng.below(4) == 0 else grid[rng.below(len(grid))]
            plan = qs.qs_fuse(gates, n, qs.options(dtype=dtype, **o))
            try:
                feats = qs.qs_plan_features(plan)
                if feats.shape[0] == 0:
                    continue
                key = (n, dtype)
                if key not in states:
                    # one live state at a time keeps device memory small
                    for st in states.values():
                        st.close()
                    states.clear()
                    states[key] = qs.State(n, dtype)
                st = states[key]
                best = None
                for _ in range(repeats):
                    ms = qs.qs_plan_profile(st.h, plan, feats.shape[0])
                    best = ms if best is None else np.minimum(best, ms)
            finally:
                qs.qs_plan_destroy(plan)
            ok = best > 0
            y = np.log(best[ok].astype(np.float64)) - (n - 20) * math.log(2.0)
            X.append(feats[ok])
            Y.append(y.astype(np.float32))
            meta.append((name, n, dtype, o, int(ok.sum())))
            rows += int(ok.sum())
            if log is not None:
                log(f"{rows:6d} rows  {name:>12s} n={n} {'c64' if dtype == 0 else 'c128'} {o}")
    finally:
        for st in states.values():
            st.close()
    if not X:
        return np.zeros((0, qs.QS_PLAN_FEATURES), np.float32), np.zeros(0, np.float32), meta
    return np.concatenate(X), np.concatenate(Y), meta


def train(X, y, seed: int = 7, epochs: int = 60, batch: int = 256, lr: float = 1e-3):
    """A new model trained on (X, y) with the library's kernels; returns (model, final loss)."""
    model = qs.qs_model_create(X.shape[1], seed)
    loss = qs.qs_model_train(model, X, y, qs.qs_train_options(epochs=epochs, batch=batch, lr=lr, seed=seed))
    return model, loss


def save(model, path: str):
    mu, sd, ym, ys = qs.qs_model_get_norm(model)
    np.savez(path, params=qs.qs_model_get_params(model), mu=mu, sd=sd, ym=ym, ys=ys)


def load(path: str):
    z = np.load(path)
    model = qs.qs_model_create(int(z["mu"].size), 1)
    qs.qs_model_set_params(model, z["params"])
    qs.qs_model_set_norm(model, z["mu"], z["sd"], float(z["ym"]), float(z["ys"]))
    return model


def main(argv=None):
    import argparse

    ap = argparse.ArgumentParser(description="collect step timings and train the cost model")
    ap.add_argument("--rows", type=int, default=50000)
    ap.add_argument("--nmin", type=int, default=24)
    ap.add_argument("--nmax", type=int, default=29)
    ap.add_argument("--seed", type=int, default=2024)
    ap.add_argument("--budget", type=float, default=None, help="seconds of data collection at most")
    ap.add_argument("--epochs", type=int, default=60)
    ap.add_argument("--out", required=True, help=".npz for the trained model")
    ap.add_argument("--data", default=None, help="also save the timing data (.npz)")
    ap.add_argument("--extra-data", default=None, help="earlier timing data (.npz) to train on too")
    a = ap.parse_args(argv)
    t0 = time.perf_counter()
    X, y, meta = collect(a.rows, a.seed, a.nmin, a.nmax, time_budget_s=a.budget)
    if a.extra_data:
        z = np.load(a.extra_data)
        X = np.concatenate([X, z["X"].astype(np.float32)])
        y = np.concatenate([y, z["y"].astype(np.float32)])
    t1 = time.perf_counter()
    if a.data:
        np.savez(a.data, X=X, y=y)
    model, loss = train(X, y, epochs=a.epochs)
    t2 = time.perf_counter()
    pred = qs.qs_model_predict(model, X)
    rmse = float(np.sqrt(np.mean((pred - y) ** 2)))
    save(model, a.out)
    qs.qs_model_destroy(model)
    print(f"rows {X.shape[0]} circuits {len(meta)} collect {t1 - t0:.1f}s train {t2 - t1:.1f}s "
          f"loss(std) {loss:.4f} rmse(ln) {rmse:.4f}")


if __name__ == "__main__":
    main()
