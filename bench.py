"""Benchmark: apply a fused, slab-blocked circuit to a full state vector on one GB300.

Default workload (the plain method at scale, at the paper's FP64 precision): the quantum Fourier
transform of a seeded random basis state on 32 qubits, complex128 (64 GiB state; 32 H + 496 CP
gates), seeded synthetic input standing in for the paper's generated benchmark circuits.  Other
workloads: --workload layered32_c128 | layered34_c64 | precision33_c64 | batch1024_c64 | ...

One step = qs_apply_plan of the whole circuit on the resident state (every plan step: slab
passes, remaps).  `value` = input gates / device time of the timed steps (CUDA events on the
state's stream, W warm-up steps first, barrier + synchronize on both sides, max over ranks).
`e2e` = the same metric through the public API with host inputs: qs_set_basis +
qs_apply_circuit (host gate list: planning and upload inside the timed region) +
qs_expect_pauli_sum read back to the host.

`forms` (default workload, one rank): the other configurations measured once each in the same
run on the same GPU -- the 32-qubit complex128 layered circuit; tensor-core against plain form
(33-qubit complex64, depth 60) with each mode's fidelity against the FP64 path; batched against
per-circuit form (1024 ansatz circuits); learned against greedy planner.

`cpu_baseline`: the FP64 CPU oracle on the machine's host cores, single-thread and OpenMP, on the
first gates of the same circuit at the bench's qubit count when host memory allows it.
--impl reference runs the same oracle as the reference arm.

Multi-GPU: replicas only (the path has no exchange step on one-GPU machines); each rank runs the
full workload and value = ranks x gates / max time.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

HBM_NOMINAL_GBS = 8000.0
DEFAULT_WORKLOAD = "qft32_c128"
WORKLOADS = {
    "layered34_c64": dict(n=34, dtype="c64", kind="layered", depth=40, seed=1002),
    "layered32_c128": dict(n=32, dtype="c128", kind="layered", depth=40, seed=1002),
    "qft32_c128": dict(n=32, dtype="c128", kind="qft", seed=1002),
    "layered30_c64": dict(n=30, dtype="c64", kind="layered", depth=40, seed=1002),
    "layered28_c64": dict(n=28, dtype="c64", kind="layered", depth=40, seed=1002),
    "precision33_c64": dict(n=33, dtype="c64", kind="layered", depth=60, seed=1003, tc=True),
    "precision30_c64": dict(n=30, dtype="c64", kind="layered", depth=60, seed=1003, tc=True),
    "precision28_c64": dict(n=28, dtype="c64", kind="layered", depth=60, seed=1003, tc=True),
    "config1": dict(n=20, dtype="c128", kind="random", ngates=200, seed=1001),
    "batch1024_c64": dict(n=24, dtype="c64", kind="batch", count=1024, seed=1004),
    "batch1024_c128": dict(n=24, dtype="c128", kind="batch", count=1024, seed=1004),
    "batch64_c64": dict(n=20, dtype="c64", kind="batch", count=64, seed=1004, nmax=20),
    "readout28_c64": dict(n=28, dtype="c64", kind="readout", seed=1009),
    "qaoa31_c128": dict(n=31, dtype="c128", kind="qaoa", p=5, seed=1006),
    "qft31_c128": dict(n=31, dtype="c128", kind="qft", seed=1006),
    "gatesweep30_c128": dict(n=30, dtype="c128", kind="gatesweep", reps=2, seed=1007),
    "gatesweep30_c64": dict(n=30, dtype="c64", kind="gatesweep", reps=2, seed=1007),
    "hsweep_c128": dict(n=33, dtype="c128", kind="hsweep", seed=1008),
    "hsweep_c64": dict(n=33, dtype="c64", kind="hsweep", seed=1008),
    "learned32_c128": dict(n=32, dtype="c128", kind="learned", depth=80, seed=1005),
    "learned28_c128": dict(n=28, dtype="c128", kind="learned", depth=80, seed=1005),
}


def make_circuit(w, n=None):
    from paper_2406_14084_gb300 import workloads as W

    n = n or w["n"]
    if w["kind"] in ("layered", "learned"):
        return W.layered(n, w["depth"], w["seed"]), 0
    if w["kind"] == "qaoa":
        return W.qaoa_complete(n, w["p"], w["seed"]), 0
    if w["kind"] == "qft":
        return W.qft(n), W.random_basis(n, w["seed"])
    return W.random_circuit(n, w["ngates"], w["seed"]), 0


# The paper's own figures for exactly these workloads (31-qubit complex128, wall time on its
# DGX-A100 setup converted to gates/s): QAOA p = 5, 2,511 gates in 17.5 s; QFT, 496 gates in 3.6 s.
# Context only -- another machine.
PAPER_GATES_PER_S = {"qaoa31_c128": 2511 / 17.5, "qft31_c128": 496 / 3.6}

# Non-tensor ALU peaks from unit counts and the maximum SM clock: 152 SMs x 2.07 GHz x FMA lanes
# per SM per clock (128 FP32, 2 FP64) x 2 flops per FMA.
ALU_PEAK_TFLOPS = {"c64": 152 * 2.07e9 * 128 * 2 / 1e12, "c128": 152 * 2.07e9 * 2 * 2 / 1e12}

TRAFFIC_SOURCES = ("k_slab.cu", "slab_common.cuh", "dev_common.cuh", "df_arith.cuh", "qs_internal.h")


def slab_kernel_hash() -> str:
    import hashlib

    h = hashlib.sha256()
    for f in TRAFFIC_SOURCES:
        with open(os.path.join(ROOT, "paper_2406_14084_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def circuit_flops_per_amp(gates) -> float:
    """Algorithmic flops per amplitude of the unfused circuit: a dense k-qubit gate is a 2^k x 2^k
    complex matrix-vector product (8 * 2^k flops per amplitude, over the 2^-c of amplitudes its c
    controls select); a diagonal costs 6 flops on the amplitudes it changes; X / CX / SWAP none."""
    f = 0.0
    for g in gates:
        k, c = len(g.targets), len(g.controls)
        sel = 2.0 ** -c
        if g.kind in ("X", "CX", "SWAP"):
            continue
        if g.kind in ("Z", "S", "SDG", "T", "TDG", "P"):
            f += 6.0 * 0.5 * sel
        elif g.kind in ("CZ", "CP"):
            f += 6.0 * 0.25 * sel
        elif g.kind in ("RZ", "RZZ", "DIAG"):
            f += 6.0 * sel
        else:
            f += 8.0 * 2 ** k * sel
    return f


def measured_traffic(n: int, dtype: str):
    """DRAM bytes per slab-pass launch from the committed ncu summary of that precision, scaled
    by 2^(n - n_capture) (every pass streams the whole state once); None if the kernel sources
    changed since."""
    p = os.path.join(ROOT, "profiles", "slab_pass_traffic.json")
    if not os.path.exists(p):
        return None
    with open(p) as f:
        doc = json.load(f)
    for t in doc.get("captures", [doc]):
        if t.get("dtype") == dtype and t.get("source_hash") == slab_kernel_hash():
            return t["dram_bytes_per_launch"] * 2.0 ** (n - t["n"])
    return None


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return {"hbm_gbs": d.get("hbm_gbs"), "bf16_tflops": d.get("bf16_tflops"), "source": "of measured"}
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "source": "of fallback"}


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []
        self.t = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 8:
                continue
            try:
                sm.append(float(f[0]))
                smax.append(float(f[1]))
            except ValueError:
                continue
            for nm, v in zip(names, f[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def max_over_ranks(value: float, dist=None, device: str = "cpu") -> float:
    """The slowest rank's time: every replica's timed region is over only when all are."""
    if dist is None:
        return value
    import torch

    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_throughput(units_per_rank: int, steps: int, ms_max: float, world: int) -> float:
    """Whole-job rate of `world` independent replicas: all units over the slowest rank's time."""
    return world * units_per_rank * steps / (ms_max / 1e3)


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


# ----------------------------------------------------------------------------- CPU oracle leg

def host_info():
    """CPU model, usable cores and host memory of this machine (read from /proc and lscpu)."""
    info = {"nproc": len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()}
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.startswith("Model name:"):
                model = ln.split(":", 1)[1].strip()
                break
    except Exception:
        pass
    if model is None:
        try:
            with open("/proc/cpuinfo") as f:
                for ln in f:
                    if ln.lower().startswith(("model name", "cpu part")):
                        model = ln.split(":", 1)[1].strip()
                        break
        except OSError:
            pass
    info["cpu_model"] = model
    try:
        mem = {}
        with open("/proc/meminfo") as f:
            for ln in f:
                k, v = ln.split(":", 1)
                mem[k] = int(v.split()[0]) * 1024
        info["host_ram_gb"] = mem.get("MemTotal", 0) / 1e9
        info["mem_available_gb"] = mem.get("MemAvailable", 0) / 1e9
    except OSError:
        info["host_ram_gb"] = info["mem_available_gb"] = None
    return info


def oracle_qubits(n_full: int, hi: dict) -> int:
    """Largest state (<= n_full qubits, complex128) the oracle may hold: at most 40 % of the
    host's available memory, so the GPU process and the box keep ample headroom."""
    avail = (hi.get("mem_available_gb") or 8.0) * 1e9
    n = n_full
    while n > 20 and (1 << n) * 16 > 0.4 * avail:
        n -= 1
    return n


def oracle_timed_gates(n_s, gates, state, budget_s, max_gates):
    """Apply gates one at a time from the start of the circuit until max_gates or the budget
    is spent (at least one); returns (gates done, seconds)."""
    import oracle

    done, t0 = 0, time.perf_counter()
    while done < min(max_gates, len(gates)):
        oracle.apply_circuit(n_s, gates[done:done + 1], state)
        done += 1
        if time.perf_counter() - t0 >= budget_s:
            break
    return done, time.perf_counter() - t0


def oracle_sample(w, budget_s: float = 15.0):
    """The FP64 oracle on the host cores, on the first gates of the same circuit (the whole
    circuit's first 50 gates at most): single-thread, then OpenMP over every usable core, each
    within half the budget.  The state has the bench's qubit count when host memory allows it;
    otherwise the largest that fits, and gates/s is scaled by the state-size ratio (the work per
    gate is proportional to 2^n).  Host GB/s counts one read and one write of the state per gate."""
    import oracle

    if w["kind"] == "batch":
        return oracle_sample_batch(w, budget_s)

    hi = host_info()
    n_full = w["n"]
    n_s = oracle_qubits(n_full, hi)
    gates, x0 = make_circuit(w, n_s)
    state = oracle.basis_state(n_s, x0 & ((1 << n_s) - 1))
    scale = 2.0 ** (n_s - n_full)
    gate_bytes = 2.0 * (1 << n_s) * 16
    threads_all = int(hi["nproc"] or 1)
    modes = {}
    for name, threads, cap in (("single_thread", 1, 50), ("openmp", threads_all, 50)):
        oracle.set_threads(threads)
        done, dt = oracle_timed_gates(n_s, gates, state, budget_s / 2, cap)
        per_gate = dt / done
        modes[name] = {"threads": threads, "gates": done, "seconds": dt, "s_per_gate": per_gate,
                       "gates_per_s": scale / per_gate, "host_gbs": gate_bytes / per_gate / 1e9}
    oracle.set_threads(threads_all)
    del state
    omp = modes["openmp"]
    return {"value": omp["gates_per_s"], "unit": "gates/s", "cores": threads_all, "kind": "oracle",
            "sample": (f"first {omp['gates']} gates (OpenMP, {threads_all} threads) and first "
                       f"{modes['single_thread']['gates']} (1 thread) of the same circuit on a "
                       f"{n_s}-qubit complex128 state"
                       + ("" if n_s == n_full else f", gates/s scaled by 2^({n_s}-{n_full})")),
            "qubits": n_s, "dtype": "c128", "modes": modes, "host": hi}


def oracle_sample_batch(w, budget_s: float):
    """Oracle amplitude-gate rate on the batch's smallest circuits, scaled to the whole batch."""
    import oracle
    from paper_2406_14084_gb300 import workloads as W

    circuits = W.vqe_batch(w["count"], w["seed"], nmax=w.get("nmax", 24))
    total_gates = sum(len(g) for _, g in circuits)
    total_work = sum(len(g) * (1 << n) for n, g in circuits)
    done_work, done_c, t0 = 0, 0, time.perf_counter()
    for n, g in sorted(circuits, key=lambda c: c[0]):
        a = oracle.apply_circuit(n, g)
        oracle.expect_pauli(a, n, W.zz_chain_hamiltonian(n))
        done_work += len(g) * (1 << n)
        done_c += 1
        if time.perf_counter() - t0 > budget_s:
            break
    dt = time.perf_counter() - t0
    est = total_work / (done_work / dt)
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    return {"value": total_gates / est, "unit": "gates/s", "cores": cores, "kind": "oracle",
            "sample": f"{done_c} smallest circuits of the batch (with <H>) in {dt:.1f} s; rate of "
                      f"amplitude-gate updates scaled to all {len(circuits)} circuits"}


def run_reference(args, w):
    """The reference arm: the FP64 CPU oracle as it stands, on every usable host core.  Each
    step is a bounded sample of the workload (the next gates of the circuit, continuing where
    the previous step stopped, on one resident state), sized so that the K + W steps take a few
    minutes in all; value = gates per second scaled to the workload's state size, ms_per_step =
    the whole circuit's gate count at that rate."""
    import oracle

    if w["kind"] == "batch":
        cpu = oracle_sample_batch(w, args.cpu_budget)
        v = cpu["value"]
        gates_full = sum(len(g) for _, g in __import__("paper_2406_14084_gb300.workloads",
                                                         fromlist=["vqe_batch"]).vqe_batch(
            w["count"], w["seed"], nmax=w.get("nmax", 24)))
        ms = 1e3 * gates_full / v
        return {"impl": "reference", "metric": "gates/s", "value": v, "unit": "gates/s", "n_gpus": args.gpus,
                "steps": 1, "warmup": 0, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "c128", "data": "synthetic (seeded generator)",
                "config": {"workload": args.workload}, "cpu_baseline": cpu,
                "e2e": {"value": v, "unit": "gates/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    hi = host_info()
    n_full = w["n"]
    n_s = oracle_qubits(n_full, hi)
    gates, x0 = make_circuit(w, n_s)
    full_gates = len(make_circuit(w)[0]) if n_s != n_full else len(gates)
    threads = int(hi["nproc"] or 1)
    oracle.set_threads(threads)
    state = oracle.basis_state(n_s, x0 & ((1 << n_s) - 1))
    scale = 2.0 ** (n_s - n_full)
    per_step = max(1.0, min(args.cpu_budget, 150.0 / max(1, args.steps)))
    pos = [0]

    def step(budget, cap):
        if pos[0] >= len(gates):
            oracle.set_basis(state, n_s, x0 & ((1 << n_s) - 1))
            pos[0] = 0
        done, dt = oracle_timed_gates(n_s, gates[pos[0]:], state, budget, cap)
        pos[0] += done
        return done, dt

    for _ in range(args.warmup):
        step(0.0, 1)
    tot_g, tot_s, step_s = 0, 0.0, []
    for _ in range(args.steps):
        d, dt = step(per_step, 10 ** 9)
        tot_g += d
        tot_s += dt
        step_s.append(dt)
    rate = tot_g / tot_s * scale
    sample = (f"{args.steps} steps of about {per_step:.1f} s, each the next gates of the circuit "
              f"({tot_g} gates in all) on a {n_s}-qubit complex128 state with {threads} OpenMP threads"
              + ("" if n_s == n_full else f", gates/s scaled by 2^({n_s}-{n_full})"))
    cpu = {"value": rate, "unit": "gates/s", "cores": threads, "kind": "oracle", "sample": sample,
           "qubits": n_s, "dtype": "c128", "host": hi,
           "host_gbs": 2.0 * (1 << n_s) * 16 * tot_g / tot_s / 1e9}
    return {"impl": "reference", "metric": "gates/s", "value": rate, "unit": "gates/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * full_gates / rate,
            "ms_per_step_basis": "the whole circuit's gates at the measured per-gate time",
            "sample_ms_per_step": 1e3 * statistics.mean(step_s), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "c128", "data": "synthetic (seeded generator)",
            "config": {"workload": args.workload, "qubits": n_full, "gates": full_gates},
            "cpu_baseline": cpu,
            "e2e": {"value": rate, "unit": "gates/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def run_batch(args, w):
    """Batched persistent launch over the whole circuit list (one graph replay per step)."""
    import torch

    from paper_2406_14084_gb300 import qs
    from paper_2406_14084_gb300 import workloads as W

    torch.cuda.set_device(0)
    dtype = qs.QS_C64 if w["dtype"] == "c64" else qs.QS_C128
    circuits = W.vqe_batch(w["count"], w["seed"], nmax=w.get("nmax", 24))
    H = W.zz_chain_hamiltonian(24)
    ngates = sum(len(g) for _, g in circuits)
    t_plan0 = time.perf_counter()
    b = qs.qs_batch_create(circuits, qs.options(dtype=dtype, graph=1))
    t_plan = time.perf_counter() - t_plan0
    chosen = qs.qs_batch_tune(b, H)
    for _ in range(args.warmup):
        qs.qs_apply_batch(b, H, len(circuits))
    clocks = ClockSampler(0)
    clocks.start()
    dev_ms, t0 = 0.0, time.perf_counter()
    for _ in range(args.steps):
        res = qs.qs_apply_batch(b, H, len(circuits))
        dev_ms += qs.qs_batch_info_get(b)["last_run_ms"]
    wall = time.perf_counter() - t0
    clk = clocks.stop()
    info = qs.qs_batch_info_get(b)
    qs.qs_batch_destroy(b)
    # e2e: the user's whole call sequence -- create (planning, plan upload), run, read back <H>
    e2e_t0 = time.perf_counter()
    b2 = qs.qs_batch_create(circuits, qs.options(dtype=dtype, graph=0, slab_bits=chosen))
    qs.qs_apply_batch(b2, H, len(circuits))
    e2e_s = time.perf_counter() - e2e_t0
    kept_terms = sum(sum(1 for t in H if t[2] < (1 << n)) for n, _ in circuits)
    e2e_h2d = qs.qs_batch_info_get(b2)["plan_bytes"] + 16 * kept_terms + 40 * len(circuits)
    qs.qs_batch_destroy(b2)
    # the per-circuit form on the same GPU: plans built and states allocated beforehand; per
    # circuit the start state, qs_apply_plan and qs_expect_pauli_sum (host result)
    plans = [qs.qs_fuse(g, m, qs.options(dtype=dtype)) for m, g in circuits]
    states = {m: qs.State(m, dtype) for m in sorted({m for m, _ in circuits})}
    Hs = {m: W.zz_chain_hamiltonian(m) for m in states}
    torch.cuda.synchronize()
    p0 = time.perf_counter()
    plain = []
    for (m, _), p in zip(circuits, plans):
        st = states[m]
        qs.qs_set_basis(st.h, 0)
        qs.qs_apply_plan(st.h, p)
        plain.append(qs.qs_expect_pauli_sum(st.h, Hs[m]).real)
    plain_s = time.perf_counter() - p0
    for p in plans:
        qs.qs_plan_destroy(p)
    for st in states.values():
        st.close()
    import numpy as np
    agree = float(np.max(np.abs(np.array(plain) - res)))
    ms_step = dev_ms / args.steps
    return {
        "metric": "gates/s", "value": ngates / (ms_step / 1e3), "unit": "gates/s", "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": w["dtype"],
        "data": "synthetic (seeded hardware-efficient ansatz batch)",
        "config": {"workload": args.workload, "circuits": len(circuits), "gates": ngates,
                   "qubits": "10..24", "layers": "2..12", "items": info["items"], "rounds": info["rounds"],
                   "slab_bits": chosen, "stage_bits": info["stage_bits"], "graph": True,
                   "state_bytes": info["state_bytes"], "l2": "states larger than L2"},
        "wall_ms_per_step": 1e3 * wall / args.steps, "plan_s": t_plan,
        "per_circuit_form": {"gates_per_s": ngates / plain_s, "seconds": plain_s,
                             "speedup_of_batched": plain_s / (ms_step / 1e3),
                             "max_abs_diff_vs_batched": agree},
        "clocks": clk, "gpu_launches": args.steps,
        "e2e": {"value": ngates / e2e_s, "unit": "gates/s", "h2d_bytes_per_step": int(e2e_h2d),
                "d2h_bytes_per_step": 8 * len(circuits)},
    }

def run_learned(args, w):
    """Learned planner against greedy on the same GPU: layered depth-80 and QFT circuits.

    Each circuit is planned twice (greedy = the caller's options; learned = the shipped cost
    model), both plans run on the same resident state, and each step is the sum over the two
    circuits of the plan's device time (CUDA events around every launch)."""
    import numpy as np
    import torch

    from paper_2406_14084_gb300 import costmodel
    from paper_2406_14084_gb300 import qs
    from paper_2406_14084_gb300 import workloads as W

    torch.cuda.set_device(0)
    dtype = qs.QS_C64 if w["dtype"] == "c64" else qs.QS_C128
    n = w["n"]
    circuits = [("layered", W.layered(n, w["depth"], w["seed"])), ("qft", W.qft(n))]
    model = costmodel.load(os.path.join(ROOT, "paper_2406_14084_gb300", "data", "cost_model.npz"))
    st = qs.State(n, dtype)
    rows, ms = {}, {"greedy": 0.0, "learned": 0.0}
    launches = 0
    clocks = ClockSampler(0)
    for name, g in circuits:
        t0 = time.perf_counter()
        pg = qs.qs_fuse(g, n, qs.options(dtype=dtype))
        tg = time.perf_counter() - t0
        t0 = time.perf_counter()
        pl = qs.qs_fuse_learned(g, n, qs.options(dtype=dtype), model)
        tl = time.perf_counter() - t0
        info = qs.qs_plan_info_get(pl)
        res = {"gates": len(g), "plan_s_greedy": tg, "plan_s_learned": tl, "candidates": info["candidates"],
               "chosen": info["chosen"], "predicted_ms": info["predicted_ms"],
               "greedy_predicted_ms": info["greedy_predicted_ms"]}
        for tag, p in (("greedy", pg), ("learned", pl)):
            steps = qs.qs_plan_features(p).shape[0]
            for _ in range(args.warmup):
                qs.qs_plan_profile(st.h, p, steps)
            clocks.start()
            t = [float(qs.qs_plan_profile(st.h, p, steps).sum()) for _ in range(args.steps)]
            clk = clocks.stop()
            launches += steps * args.steps
            res[tag + "_ms"] = float(np.median(t))
            res[tag + "_passes"] = qs.qs_plan_info_get(p)["passes"]
            ms[tag] += res[tag + "_ms"]
        res["gain"] = res["greedy_ms"] / res["learned_ms"]
        rows[name] = res
        qs.qs_plan_destroy(pg)
        qs.qs_plan_destroy(pl)
    st.close()
    qs.qs_model_destroy(model)
    ngates = sum(len(g) for _, g in circuits)
    return {
        "metric": "gates/s", "value": ngates / (ms["learned"] / 1e3), "unit": "gates/s", "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms["learned"], "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": w["dtype"],
        "data": "synthetic (seeded layered depth-80 + QFT)",
        "config": {"workload": args.workload, "qubits": n, "gates": ngates, "planner": "learned",
                   "l2": "state larger than L2"},
        "greedy": {"gates_per_s": ngates / (ms["greedy"] / 1e3), "ms_per_step": ms["greedy"]},
        "gain_vs_greedy": ms["greedy"] / ms["learned"], "circuits": rows, "clocks": clk,
        "gpu_launches": launches,
    }

def run_readouts(args, w):
    """The readout step (norm, marginal probabilities, Pauli-sum expectation, sampling) on an
    n-qubit state: each is one read of the state, so the roofline is 2^n * s bytes per call over
    its wall time (each call synchronises and returns host data)."""
    import numpy as np
    import torch

    from paper_2406_14084_gb300 import qs
    from paper_2406_14084_gb300 import workloads as W

    torch.cuda.set_device(0)
    dtype = qs.QS_C64 if w["dtype"] == "c64" else qs.QS_C128
    n = w["n"]
    s_amp = 8 if dtype == qs.QS_C64 else 16
    H = W.zz_chain_hamiltonian(n)
    u = np.random.default_rng(w["seed"]).random(100000)
    calls = {"norm2": lambda st: st.norm2(), "probs_3q": lambda st: st.probs([0, n // 2, n - 1]),
             "expect_zz_chain": lambda st: st.expect(H), "sample_100k": lambda st: st.sample(u)}
    rows = {}
    peaks = measured_peaks()
    clocks = ClockSampler(0)
    with qs.State(n, dtype) as st:
        st.apply(W.layered(n, 2, w["seed"]), qs.options(dtype=dtype))
        clocks.start()
        for name, f in calls.items():
            for _ in range(args.warmup):
                f(st)
            ts = []
            for _ in range(args.steps):
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                f(st)
                ts.append(time.perf_counter() - t0)
            best = min(ts)
            gbs = (1 << n) * s_amp / best / 1e9
            rows[name] = {"ms": 1e3 * best, "gbs": gbs, "frac_of_hbm": gbs / peaks["hbm_gbs"]}
        clk = clocks.stop()
    ms_total = sum(r["ms"] for r in rows.values())
    return {
        "metric": "readouts/s", "value": len(rows) / (ms_total / 1e3), "unit": "readouts/s", "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_total, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": w["dtype"], "data": "synthetic (seeded layered state)",
        "config": {"workload": args.workload, "qubits": n, "terms": len(H), "shots": int(u.size),
                   "l2": "state larger than L2"},
        "readouts": rows, "hbm_peak_gbs": peaks["hbm_gbs"], "peak_source": peaks["source"], "clocks": clk,
        "gpu_launches": None,
    }


TABLE1_KINDS = ["H", "X", "Y", "Z", "S", "T", "RX", "RY", "RZ", "U3", "CX", "CZ", "CP", "SWAP", "RZZ"]


def _plan_device_ms(qs, st, plan, warmup, steps):
    nst = qs.qs_plan_features(plan).shape[0]
    if nst == 0:
        return 0.0
    for _ in range(warmup):
        qs.qs_plan_profile(st.h, plan, nst)
    return min(float(qs.qs_plan_profile(st.h, plan, nst).sum()) for _ in range(max(1, steps)))


def run_gate_sweeps(args, w):
    """Gate benchmarks shaped like the paper's (Sec. VI-D): per gate kind of Table 1, every
    qubit `reps` times, applied gate by gate (one pass per gate) and through the blocked plan;
    or (hsweep) ten H gates on states of 24..n qubits.  Device time from CUDA events per launch."""
    import numpy as np
    import torch

    from paper_2406_14084_gb300 import qs
    from paper_2406_14084_gb300 import workloads as W

    torch.cuda.set_device(0)
    dtype = qs.QS_C64 if w["dtype"] == "c64" else qs.QS_C128
    s_amp = 8 if dtype == qs.QS_C64 else 16
    rows, tot_g, tot_ms, launches = {}, 0, 0.0, 0
    clocks = ClockSampler(0)
    clocks.start()
    if w["kind"] == "gatesweep":
        n = w["n"]
        with qs.State(n, dtype) as st:
            st.apply([W.Gate("H", (q,)) for q in range(n)], qs.options(dtype=dtype))
            for kind in TABLE1_KINDS:
                g = W.gate_sweep(n, kind, w["reps"], w["seed"])
                row = {"gates": len(g)}
                for mode, o in (("gate_by_gate", dict(fuse_width=0, blocking=0)), ("blocked", {})):
                    p = qs.qs_fuse(g, n, qs.options(dtype=dtype, **o))
                    ms = _plan_device_ms(qs, st, p, args.warmup, args.steps)
                    launches += qs.qs_plan_features(p).shape[0] * (args.warmup + max(1, args.steps))
                    qs.qs_plan_destroy(p)
                    # uncontrolled SWAPs are relabellings: a plan of them does no device work
                    row[mode + "_gates_per_s"] = len(g) / (ms / 1e3) if ms > 0 else None
                    if mode == "gate_by_gate" and ms > 0:
                        row["gate_by_gate_gbs"] = len(g) * 2.0 * (1 << n) * s_amp / (ms / 1e3) / 1e9
                        row["gate_by_gate_frac_of_hbm"] = row["gate_by_gate_gbs"] / measured_peaks()["hbm_gbs"]
                    elif mode == "blocked" and ms > 0:
                        tot_g += len(g)
                        tot_ms += ms
                rows[kind] = row
    else:
        for n in range(24, w["n"] + 1):
            rng = W.SplitMix64(w["seed"] + n)
            g = [W.Gate("H", (rng.below(n),)) for _ in range(10)]
            with qs.State(n, dtype) as st:
                row = {"gates": len(g)}
                for mode, o in (("gate_by_gate", dict(fuse_width=0, blocking=0)), ("blocked", {})):
                    p = qs.qs_fuse(g, n, qs.options(dtype=dtype, **o))
                    nst = qs.qs_plan_features(p).shape[0]
                    ms = _plan_device_ms(qs, st, p, args.warmup, args.steps)
                    launches += nst * (args.warmup + max(1, args.steps))
                    qs.qs_plan_destroy(p)
                    row[mode + "_ms"] = ms
                    row[mode + "_passes"] = nst
                    row[mode + "_gbs"] = nst * 2.0 * (1 << n) * s_amp / (ms / 1e3) / 1e9
                    row[mode + "_frac_of_hbm"] = row[mode + "_gbs"] / measured_peaks()["hbm_gbs"]
                    if mode == "blocked" and n == w["n"]:
                        tot_g, tot_ms = len(g), ms
                rows[str(n)] = row
    clk = clocks.stop()
    peaks = measured_peaks()
    return {
        "metric": "gates/s", "value": tot_g / (tot_ms / 1e3), "unit": "gates/s", "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": tot_ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": w["dtype"], "data": "synthetic (seeded gate sweeps)",
        "config": {"workload": args.workload, "qubits": w["n"], "l2": "states larger than L2 from 24 qubits"},
        "sweep": rows, "hbm_peak_gbs": peaks["hbm_gbs"], "clocks": clk, "gpu_launches": launches,
    }

# ----------------------------------------------------------------------------- GPU leg

def fidelity_check(w, opts, dtype, n_small=22):
    """Same circuit family and options on an n_small-qubit state: GPU path vs the FP64 oracle."""
    import numpy as np

    import oracle
    from paper_2406_14084_gb300 import qs

    gates, x0 = make_circuit(w, n_small)
    x0 &= (1 << n_small) - 1
    want = oracle.apply_circuit(n_small, gates, oracle.basis_state(n_small, x0))
    s = qs.State(n_small, dtype)
    try:
        s.set_basis(x0)
        s.apply(gates, opts)
        got = s.amplitudes().astype(np.complex128)
    finally:
        s.close()
    ov = abs(np.vdot(want, got)) ** 2 / (np.vdot(want, want).real * np.vdot(got, got).real)
    return {"qubits": n_small, "gates": len(gates), "infidelity": float(1.0 - ov),
            "max_abs_err": float(np.max(np.abs(got - want))), "reference": "FP64 CPU oracle, same circuit family"}


def fidelity_vs_fp64_path(w, opts, n_copy=26):
    """Tensor-core form against the library's complex128 path (itself checked against the FP64
    oracle by the parity tests) on an n_copy-qubit copy of the same circuit: infidelity, max
    |delta amp| and the norm drift of the complex64 result."""
    import numpy as np

    from paper_2406_14084_gb300 import qs

    gates, x0 = make_circuit(w, n_copy)
    x0 &= (1 << n_copy) - 1
    with qs.State(n_copy, qs.QS_C128) as ref:
        ref.set_basis(x0)
        ref.apply(gates, qs.options(dtype=qs.QS_C128))
        want = ref.amplitudes()
    with qs.State(n_copy, qs.QS_C64) as s:
        s.set_basis(x0)
        s.apply(gates, opts)
        got = s.amplitudes().astype(np.complex128)
    nw, ng = np.vdot(want, want).real, np.vdot(got, got).real
    ov = abs(np.vdot(want, got)) ** 2 / (nw * ng)
    return {"qubits": n_copy, "gates": len(gates), "infidelity": float(1.0 - ov),
            "max_abs_err": float(np.max(np.abs(got - want))), "norm_drift": float(ng - nw),
            "reference": "complex128 path of this library (FP64), same circuit"}

# ----------------------------------------------------------------------------- forms

def _timed_apply_ms(qs, torch, st, plan, stream, x0=0):
    """One qs_apply_plan on a fresh start state, device time by CUDA events on the state's stream."""
    qs.qs_set_basis(st.h, x0)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    qs.qs_apply_plan(st.h, plan)
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1)


def _plan_alu(qs, plan, n, ms, dtype):
    flops = 2.0 * float(qs.qs_plan_features(plan)[:, 26].sum()) * (1 << n)
    peak = ALU_PEAK_TFLOPS["c64" if dtype == qs.QS_C64 else "c128"]
    return {"tflops": flops / (ms / 1e3) / 1e12, "frac_of_alu_peak": flops / (ms / 1e3) / 1e12 / peak}


def form_layered32_c128(qs, torch):
    """Config 2(ii): 32-qubit complex128 layered circuit of depth 40, greedy plan, one apply."""
    w = WORKLOADS["layered32_c128"]
    n, dtype = w["n"], qs.QS_C128
    gates, x0 = make_circuit(w)
    opts = qs.options(dtype=dtype)
    plan = qs.qs_fuse(gates, n, opts)
    info = qs.qs_plan_info_get(plan)
    stream = torch.cuda.Stream()
    with qs.State(n, dtype) as st:
        qs.qs_set_stream(st.h, stream.cuda_stream)
        ms = _timed_apply_ms(qs, torch, st, plan, stream, x0)
        norm = qs.qs_norm2(st.h)
    passes = info["passes"] + info["remaps"] + info["unblocked"]
    gbs = passes * 2.0 * (1 << n) * 16 / (ms / 1e3) / 1e9
    out = {"workload": "layered32_c128", "qubits": n, "gates": len(gates), "dtype": "c128",
           "ms": ms, "gates_per_s": len(gates) / (ms / 1e3), "passes": passes,
           "effective_hbm_gbs": gbs, "frac_of_hbm": gbs / measured_peaks()["hbm_gbs"],
           "alu": _plan_alu(qs, plan, n, ms, dtype), "norm_after": norm,
           "fidelity": fidelity_check(w, opts, dtype, n_small=20)}
    qs.qs_plan_destroy(plan)
    return out


def form_df_c128(qs, torch, name):
    """Complex128 in double-float form (qs_options.arith = QS_ARITH_DF): the register stages run on
    the FP32 pipe with pairs of FP32 numbers, the state stays complex128.  One apply of the
    32-qubit circuit against one apply with FP64 arithmetic, and max |delta amp| against the
    FP64 oracle on the 20-qubit copy of the same circuit."""
    w = WORKLOADS[name]
    n, dtype = w["n"], qs.QS_C128
    gates, x0 = make_circuit(w)
    o_df = qs.options(dtype=dtype, arith=qs.QS_ARITH_DF)
    p_df = qs.qs_fuse(gates, n, o_df)
    stream = torch.cuda.Stream()
    with qs.State(n, dtype) as st:
        qs.qs_set_stream(st.h, stream.cuda_stream)
        _timed_apply_ms(qs, torch, st, p_df, stream, x0)  # warm-up (kernel set-up)
        ms = _timed_apply_ms(qs, torch, st, p_df, stream, x0)
        norm = qs.qs_norm2(st.h)
    qs.qs_plan_destroy(p_df)
    return {"workload": name, "qubits": n, "gates": len(gates), "dtype": "c128 (double-float stages)",
            "ms": ms, "gates_per_s": len(gates) / (ms / 1e3), "norm_after": norm,
            "fidelity": fidelity_check(w, o_df, dtype, n_small=20)}


def form_tensor_cores(qs, torch):
    """Config 3: 33-qubit complex64 layered depth 60; tensor-core plans (6- and 7-qubit blocks,
    BF16 x 3 and TF32 x 3 split products) against the plain SIMT plan, one apply each; each
    mode's fidelity and max |delta amp| against the FP64 path on the 26-qubit copy, and against
    the oracle at 20 qubits."""
    w = WORKLOADS["precision33_c64"]
    n, dtype = w["n"], qs.QS_C64
    gates, x0 = make_circuit(w)
    o_plain = qs.options(dtype=dtype)
    modes = {"bf16x3": (qs.QS_TC_BF16X3, 6), "tf32x3": (qs.QS_TC_TF32X3, 6),
             "bf16x3_7q": (qs.QS_TC_BF16X3, 7), "tf32x3_7q": (qs.QS_TC_TF32X3, 7)}
    res = {"workload": "precision33_c64", "qubits": n, "gates": len(gates), "dtype": "c64", "modes": {}}
    stream = torch.cuda.Stream()
    p_plain = qs.qs_fuse(gates, n, o_plain)
    with qs.State(n, dtype) as st:
        qs.qs_set_stream(st.h, stream.cuda_stream)
        ms_plain = _timed_apply_ms(qs, torch, st, p_plain, stream, x0)
        res["plain"] = {"ms": ms_plain, "gates_per_s": len(gates) / (ms_plain / 1e3),
                        "passes": qs.qs_plan_info_get(p_plain)["passes"]}
        qs.qs_plan_destroy(p_plain)
        for name, (mode, width) in modes.items():
            o = qs.options(dtype=dtype, tc=mode, tc_width=width)
            try:
                p = qs.qs_fuse(gates, n, o)
            except qs.QsError as e:
                res["modes"][name] = {"unsupported": str(e)}
                continue
            info = qs.qs_plan_info_get(p)
            qs.qs_stats_reset(st.h)
            qs.qs_set_profiling(st.h, True)
            ms = _timed_apply_ms(qs, torch, st, p, stream, x0)
            qs.qs_set_profiling(st.h, False)
            stt = qs.qs_stats(st.h)
            qs.qs_plan_destroy(p)
            r = {"ms": ms, "gates_per_s": len(gates) / (ms / 1e3), "speedup_vs_plain": ms_plain / ms,
                 "tc_gates": info["tc_gates"], "passes": info["passes"]}
            if stt["tc_gates"]:
                r["tc_launch_ms"] = stt["tc_ms"] / stt["tc_gates"]
            r["fidelity_vs_fp64_path"] = fidelity_vs_fp64_path(w, o)
            r["fidelity_vs_oracle"] = fidelity_check(w, o, dtype, n_small=20)
            res["modes"][name] = r
    return res


def form_batch(qs, torch, dtype_name):
    """Config 4: 1024 ansatz circuits in one persistent launch (autotuned, graph replay) against
    the per-circuit form (plans built beforehand; per circuit: start state, qs_apply_plan,
    qs_expect_pauli_sum), same GPU; max |delta <H>| between the two."""
    import numpy as np

    from paper_2406_14084_gb300 import workloads as W

    w = WORKLOADS["batch1024_" + dtype_name]
    dtype = qs.QS_C64 if dtype_name == "c64" else qs.QS_C128
    circuits = W.vqe_batch(w["count"], w["seed"], nmax=w.get("nmax", 24))
    H = W.zz_chain_hamiltonian(24)
    ngates = sum(len(g) for _, g in circuits)
    b = qs.qs_batch_create(circuits, qs.options(dtype=dtype, graph=1))
    try:
        chosen = qs.qs_batch_tune(b, H)
        qs.qs_apply_batch(b, H, len(circuits))
        res = qs.qs_apply_batch(b, H, len(circuits))
        batch_ms = qs.qs_batch_info_get(b)["last_run_ms"]
    finally:
        qs.qs_batch_destroy(b)
    plans = [qs.qs_fuse(g, m, qs.options(dtype=dtype)) for m, g in circuits]
    states = {m: qs.State(m, dtype) for m in sorted({m for m, _ in circuits})}
    Hs = {m: W.zz_chain_hamiltonian(m) for m in states}
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    plain = []
    for (m, _), p in zip(circuits, plans):
        st = states[m]
        qs.qs_set_basis(st.h, 0)
        qs.qs_apply_plan(st.h, p)
        plain.append(qs.qs_expect_pauli_sum(st.h, Hs[m]).real)
    plain_s = time.perf_counter() - t0
    for p in plans:
        qs.qs_plan_destroy(p)
    for st in states.values():
        st.close()
    return {"workload": "batch1024_" + dtype_name, "circuits": len(circuits), "gates": ngates,
            "dtype": dtype_name, "slab_bits": chosen,
            "batched": {"ms": batch_ms, "gates_per_s": ngates / (batch_ms / 1e3)},
            "per_circuit": {"ms": 1e3 * plain_s, "gates_per_s": ngates / plain_s},
            "speedup_vs_per_circuit": 1e3 * plain_s / batch_ms,
            "max_abs_diff_expect_H": float(np.max(np.abs(np.array(plain) - res)))}


def form_learned(qs, torch, n):
    """Config 5: learned planner against greedy on layered depth 80 and QFT, complex128.  Each
    circuit: the greedy plan once; the learned plan three times (the first apply times the
    model's pick, the second its greedy twin, the third runs what the judge kept).  Outputs of
    the two plans compared on sampled amplitudes, and the learned plan against the oracle at
    20 qubits."""
    import numpy as np

    import oracle
    from paper_2406_14084_gb300 import costmodel
    from paper_2406_14084_gb300 import workloads as W

    dtype = qs.QS_C128
    model = costmodel.load(os.path.join(ROOT, "paper_2406_14084_gb300", "data", "cost_model.npz"))
    circuits = [("layered80", W.layered(n, 80, 1005)), ("qft", W.qft(n))]
    stream = torch.cuda.Stream()
    out = {"qubits": n, "dtype": "c128", "circuits": {}}
    tot = {"greedy": 0.0, "judged": 0.0}
    try:
        with qs.State(n, dtype) as sg, qs.State(n, dtype) as sl:
            for st in (sg, sl):
                qs.qs_set_stream(st.h, stream.cuda_stream)
            for name, g in circuits:
                pg = qs.qs_fuse(g, n, qs.options(dtype=dtype))
                pl = qs.qs_fuse_learned(g, n, qs.options(dtype=dtype), model)
                info = qs.qs_plan_info_get(pl)
                ms_g = _timed_apply_ms(qs, torch, sg, pg, stream)
                ms_pick = _timed_apply_ms(qs, torch, sl, pl, stream)
                ms_twin = _timed_apply_ms(qs, torch, sl, pl, stream)
                ms_j = _timed_apply_ms(qs, torch, sl, pl, stream)
                rng = np.random.default_rng(7)
                worst = 0.0
                for first in [0] + [int(v) * 4096 for v in rng.integers(0, (1 << n) // 4096, size=7)]:
                    a = qs.qs_copy_to_host(sg.h, n, dtype, first, 4096)
                    b = qs.qs_copy_to_host(sl.h, n, dtype, first, 4096)
                    worst = max(worst, float(np.max(np.abs(a - b))))
                small = W.layered(20, 80, 1005) if name == "layered80" else W.qft(20)
                want = oracle.apply_circuit(20, small)
                p22 = qs.qs_fuse_learned(small, 20, qs.options(dtype=dtype), model)
                with qs.State(20, dtype) as s22:
                    qs.qs_apply_plan(s22.h, p22)
                    err22 = float(np.max(np.abs(s22.amplitudes() - want)))
                qs.qs_plan_destroy(p22)
                out["circuits"][name] = {
                    "gates": len(g), "greedy_ms": ms_g, "model_pick_ms": ms_pick, "greedy_twin_ms": ms_twin,
                    "judged_ms": ms_j, "gain_judged": ms_g / ms_j, "gain_model_pick": ms_g / ms_pick,
                    "chosen": info["chosen"], "candidates": info["candidates"],
                    "predicted_ms": info["predicted_ms"], "greedy_predicted_ms": info["greedy_predicted_ms"],
                    "max_abs_diff_vs_greedy_sampled": worst, "max_abs_err_vs_oracle_20q": err22}
                tot["greedy"] += ms_g
                tot["judged"] += ms_j
                qs.qs_plan_destroy(pg)
                qs.qs_plan_destroy(pl)
    finally:
        qs.qs_model_destroy(model)
    out["gain_judged_total"] = tot["greedy"] / tot["judged"]
    return out


def run_forms(args):
    """Every other configuration, measured once on the same GPU in the same run."""
    import torch

    from paper_2406_14084_gb300 import qs

    forms, t0 = {}, time.perf_counter()
    jobs = [("layered32_c128", lambda: form_layered32_c128(qs, torch)),
            ("tensor_cores_vs_plain", lambda: form_tensor_cores(qs, torch)),
            ("batched_vs_per_circuit_c64", lambda: form_batch(qs, torch, "c64")),
            ("learned_vs_greedy", lambda: form_learned(qs, torch, args.learned_n)),
            ("layered32_c128_double_float", lambda: form_df_c128(qs, torch, "layered32_c128")),
            ("qft32_c128_double_float", lambda: form_df_c128(qs, torch, "qft32_c128")),
            ("batched_vs_per_circuit_c128", lambda: form_batch(qs, torch, "c128"))]
    for name, job in jobs:
        if time.perf_counter() - t0 > args.forms_budget:
            forms[name] = {"skipped": f"forms time budget of {args.forms_budget:.0f} s spent"}
            continue
        t1 = time.perf_counter()
        try:
            forms[name] = job()
        except Exception as e:  # a form that fails is reported, not fatal to the bench line
            forms[name] = {"error": f"{type(e).__name__}: {e}"}
        forms[name]["wall_s"] = time.perf_counter() - t1
        torch.cuda.synchronize()
    return forms


def run_gpu(args, w, ws, rank, local):
    import torch

    from paper_2406_14084_gb300 import qs
    from paper_2406_14084_gb300 import workloads as W

    torch.cuda.set_device(local)
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    n = w["n"]
    dtype = qs.QS_C64 if w["dtype"] == "c64" else qs.QS_C128
    amp_bytes = 8 if dtype == qs.QS_C64 else 16
    gates, x0 = make_circuit(w)
    opts = qs.options(dtype=dtype)
    if args.fuse is not None:
        opts.fuse_width = args.fuse
    if args.slab_bits:
        opts.slab_bits = args.slab_bits
    if args.slab_mode == "remap":
        opts.slab_mode = qs.QS_SLAB_REMAP
    if args.stage_bits:
        opts.stage_bits = args.stage_bits
    if args.seg_bits:
        opts.seg_bits = args.seg_bits
    if w["kind"] == "random":
        opts.fuse_width, opts.blocking = 0, 0
    if (w.get("tc") and args.tc != "off") or args.tc == "bf16x3":
        opts.tc = qs.QS_TC_BF16X3
    if args.tc == "tf32x3":
        opts.tc = qs.QS_TC_TF32X3
    if args.arith == "df":
        opts.arith = qs.QS_ARITH_DF

    t_plan0 = time.perf_counter()
    plan = qs.qs_fuse(gates, n, opts)
    t_plan = time.perf_counter() - t_plan0
    info = qs.qs_plan_info_get(plan)
    nsteps = info["passes"] + info["remaps"] + info["unblocked"] + info["tc_gates"]
    plan_fma_per_amp = float(qs.qs_plan_features(plan)[:, 26].sum())

    stream = torch.cuda.Stream()
    state = qs.State(n, dtype)
    qs.qs_set_stream(state.h, stream.cuda_stream)
    qs.qs_set_basis(state.h, x0)

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    for _ in range(args.warmup):
        qs.qs_apply_plan(state.h, plan)
    barrier()
    qs.qs_stats_reset(state.h)
    qs.qs_set_profiling(state.h, True)
    clocks = ClockSampler(local)
    clocks.start()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier()
    ev0.record(stream)
    for _ in range(args.steps):
        qs.qs_apply_plan(state.h, plan)
    ev1.record(stream)
    barrier()
    clk = clocks.stop()
    qs.qs_set_profiling(state.h, False)
    ms = ev0.elapsed_time(ev1)
    st = qs.qs_stats(state.h)
    ms = max_over_ranks(ms, dist, "cuda")
    ms_step = ms / args.steps
    gates_per_s = replica_throughput(len(gates), args.steps, ms, ws)
    pass_bytes = 2.0 * (1 << n) * amp_bytes
    passes_per_step = info["passes"] + info["remaps"] + info["unblocked"]
    eff_gbs = passes_per_step * pass_bytes / (ms_step / 1e3) / 1e9
    npass_timed = st["passes"] + st["remaps"] + st["unblocked"]
    dom_ms = (st["pass_ms"] + st["remap_ms"] + st["unblocked_ms"]) / max(1, npass_timed)
    peaks = measured_peaks()
    achieved = pass_bytes / (dom_ms / 1e3) / 1e9
    # arithmetic side: the real FMAs the plan's ops execute per amplitude (2 flops each) over
    # the summed pass time, against the FP32 / FP64 ALU peak; the circuit's algorithmic flops
    # (8 * 2^k per amplitude for a dense k-qubit gate, 6 on the amplitudes a diagonal changes)
    # are reported beside it
    pass_ms_total = st["pass_ms"] + st["remap_ms"] + st["unblocked_ms"]
    exec_flops_amp = 2.0 * float(plan_fma_per_amp)
    alu_tflops = exec_flops_amp * (1 << n) * args.steps / (pass_ms_total / 1e3) / 1e12
    algo_flops_amp = circuit_flops_per_amp(gates)
    traffic = measured_traffic(n, w["dtype"])
    roof = {"bound": "hbm", "achieved": achieved, "peak": peaks["hbm_gbs"], "unit": "GB/s",
            "frac": achieved / peaks["hbm_gbs"], "traffic": traffic,
            "kernel": "slab_pass_kernel", "peak_source": peaks["source"],
            "avg_launch_ms": dom_ms, "bytes_per_launch": pass_bytes}
    tc_roof = None
    if st["tc_gates"] and st["tc_ms"] > pass_ms_total:
        # the tensor-core kernel dominates: one launch streams the state once (HBM) and applies a
        # 6-qubit gate as 3 BF16 products of the 128 x 128 real embedding, 24 * 2^6 flop/amplitude
        tc_launch_ms = st["tc_ms"] / st["tc_gates"]
        tc_gbs = pass_bytes / (tc_launch_ms / 1e3) / 1e9
        roof = {"bound": "hbm", "achieved": tc_gbs, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                "frac": tc_gbs / peaks["hbm_gbs"], "traffic": None, "kernel": "tc_kernel",
                "peak_source": peaks["source"], "avg_launch_ms": tc_launch_ms, "bytes_per_launch": pass_bytes}
        tc_tflops = 24.0 * 64 * (1 << n) / (tc_launch_ms / 1e3) / 1e12
        tc_roof = {"bound": "tensor", "achieved": tc_tflops, "peak": peaks["bf16_tflops"], "unit": "TFLOP/s",
                   "frac": tc_tflops / peaks["bf16_tflops"], "kernel": "tc_kernel",
                   "peak_source": "BF16 dense, " + peaks["source"]}
    alu_peak = ALU_PEAK_TFLOPS["c64" if dtype == qs.QS_C64 else "c128"]
    roof_alu = {"bound": "alu", "achieved": alu_tflops, "peak": alu_peak, "unit": "TFLOP/s",
                "frac": alu_tflops / alu_peak, "traffic": traffic, "kernel": "slab_pass_kernel",
                "avg_launch_ms": dom_ms,
                "flops_per_launch": exec_flops_amp * (1 << n) / max(1, passes_per_step),
                "algorithmic_flops_per_amp": exec_flops_amp,
                "algorithmic_basis": "the fused plan's ops: 8 * 2^k flops per amplitude for a dense "
                                     "k-qubit op, 4 for a real 2 x 2 rotation, 6 for a diagonal",
                "circuit_flops_per_amp": algo_flops_amp,
                "peak_source": "152 SMs x 2.07 GHz x (128 FP32 | 2 FP64) FMA/clk x 2 (unit counts "
                               "and the maximum SM clock)"}
    # the roofline that binds is the one whose floor (work / peak) is the larger: memory for a
    # pass with little arithmetic, the FMA pipe of the state precision for a deep gate block
    if tc_roof is None and roof_alu["frac"] > roof["frac"]:
        roof, roof_other = roof_alu, roof
    else:
        roof_other = roof_alu
    norm = qs.qs_norm2(state.h)
    fidelity = None if args.no_fidelity else fidelity_check(w, opts, dtype)
    fidelity_fp64 = fidelity_vs_fp64_path(w, opts) if (opts.tc and not args.no_fidelity) else None

    # ---- e2e through the public API with host inputs
    H = W.zz_chain_hamiltonian(n)
    e2e_steps = max(1, min(args.steps, args.e2e_steps))
    barrier()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        qs.qs_set_basis(state.h, x0)
        qs.qs_apply_circuit(state.h, gates, opts)
        e = qs.qs_expect_pauli_sum(state.h, H)
    barrier()
    e2e_s = (time.perf_counter() - t0) / e2e_steps
    h2d = info["device_bytes"] + 16 * 256 * 3  # plan upload + one Pauli term group
    e2e = {"value": ws * len(gates) / e2e_s, "unit": "gates/s", "h2d_bytes_per_step": int(h2d),
           "d2h_bytes_per_step": 16, "expect_H": e.real}

    state.close()
    qs.qs_plan_destroy(plan)
    if dist is not None:
        dist.destroy_process_group()
    if rank != 0:
        return None
    line = {
        "metric": "gates/s",
        "value": gates_per_s,
        "unit": "gates/s",
        "n_gpus": ws,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": ms_step,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": (gates_per_s / PAPER_GATES_PER_S[args.workload]) if args.workload in PAPER_GATES_PER_S else None,
        "dtype": "c64" if dtype == qs.QS_C64 else ("c128" if args.arith == "fp64" else "c128-storage/df32x2-arith"),
        "data": "synthetic (seeded generator, paper-shaped circuit)",
        "config": {"workload": args.workload, "qubits": n, "gates": len(gates),
                   "state_bytes": (1 << n) * amp_bytes, "l2": "state larger than L2",
                   "slab_bits": info["slab_bits"], "seg_bits": info["seg_bits"],
                   "fused_ops": info["ops"], "passes_per_step": info["passes"],
                   "remaps_per_step": info["remaps"], "unblocked_per_step": info["unblocked"],
                   "parallelism": f"replicas x{ws}"},
        "effective_hbm_gbs": eff_gbs,
        "effective_frac_of_nominal_8tbs": eff_gbs / HBM_NOMINAL_GBS,
        "plan_s": t_plan,
        "norm_after": norm,
        "fidelity": fidelity,
        "fidelity_vs_fp64_path": fidelity_fp64,
        "tc": bool(opts.tc),
        "roofline": roof,
        "roofline_other": roof_other,
        "roofline_tensor": tc_roof,
        "clocks": clk,
        "gpu_launches": args.steps * nsteps,
        "e2e": e2e,
    }
    return line


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)  # about half a minute of timed work
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD, choices=sorted(WORKLOADS))
    ap.add_argument("--fuse", type=int, default=None)
    ap.add_argument("--slab-bits", type=int, default=0)
    ap.add_argument("--slab-mode", default="gather", choices=["gather", "remap"])
    ap.add_argument("--stage-bits", type=int, default=0)
    ap.add_argument("--seg-bits", type=int, default=0)
    ap.add_argument("--tc", default="auto", choices=["auto", "off", "bf16x3", "tf32x3"])
    ap.add_argument("--arith", default="fp64", choices=["fp64", "df"],
                    help="complex128 register stages in FP64 or in double-float form")
    ap.add_argument("--no-fidelity", action="store_true")
    ap.add_argument("--e2e-steps", type=int, default=2)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-budget", type=float, default=15.0)
    ap.add_argument("--forms", default="auto", choices=["auto", "on", "off"])
    ap.add_argument("--forms-budget", type=float, default=720.0)
    ap.add_argument("--learned-n", type=int, default=30)
    args = ap.parse_args()
    ws, rank, local = dist_env()
    w = WORKLOADS[args.workload]

    if args.impl == "reference":
        if rank != 0:
            return
        print(json.dumps(run_reference(args, w)))
        return

    if w["kind"] == "batch":
        if rank != 0:
            return
        line = run_batch(args, w)
    elif w["kind"] == "learned":
        if rank != 0:
            return
        line = run_learned(args, w)
    elif w["kind"] in ("gatesweep", "hsweep"):
        if rank != 0:
            return
        line = run_gate_sweeps(args, w)
    elif w["kind"] == "readout":
        if rank != 0:
            return
        line = run_readouts(args, w)
    else:
        line = run_gpu(args, w, ws, rank, local)
    if line is None:
        return
    if args.forms == "on" or (args.forms == "auto" and args.workload == DEFAULT_WORKLOAD and ws == 1
                              and w["kind"] not in ("batch", "learned", "gatesweep", "hsweep", "readout")):
        line["forms"] = run_forms(args)
    if not args.no_cpu_baseline and ws == 1 and w["kind"] not in ("gatesweep", "hsweep", "learned", "readout"):
        line["cpu_baseline"] = oracle_sample(w, budget_s=args.cpu_budget)
    print(json.dumps(line))


if __name__ == "__main__":
    main()
