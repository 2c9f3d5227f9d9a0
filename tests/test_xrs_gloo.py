"""Cross-rank swapping on CPU ranks (gloo): the distributed exchange equals the remap (Eq. 4)
of the full state by the FP64 oracle, for 2 and 4 ranks."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def rank_main(rank, world, port, n, pairs, state, out):
    import sys

    import torch.distributed as dist

    sys.path.insert(0, ROOT)
    from paper_2406_14084_gb300 import xrs

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        full = torch.from_numpy(state)
        local = xrs.split_state(full, n, world, rank)
        n_local = n - (world.bit_length() - 1)
        xrs.cross_rank_swap(local, n_local, pairs, rank, world)
        out[rank] = local.numpy().copy()
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world,pairs", [(2, [(3, 0)]), (2, [(0, 0)]), (4, [(0, 1), (5, 0)]), (4, [(7, 1)])])
def test_cross_rank_swap_equals_remap(world, pairs):
    import oracle
    from paper_2406_14084_gb300 import workloads as W

    n = 10
    state = oracle.apply_circuit(n, W.random_circuit(n, 60, 41))
    R = world.bit_length() - 1
    n_local = n - R
    want = state.copy()
    oracle.remap(want, n, [l for l, _ in pairs], [n_local + j for _, j in pairs])
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(rank_main, args=(world, free_port(), n, pairs, state, out), nprocs=world, join=True)
    got = np.concatenate([out[r] for r in range(world)])
    assert np.array_equal(got, want)


def test_bad_arguments_on_a_single_rank():
    import sys

    sys.path.insert(0, ROOT)
    from paper_2406_14084_gb300 import xrs

    with pytest.raises(ValueError):
        xrs.cross_rank_swap(torch.zeros(8, dtype=torch.complex128), 4, [(0, 0)], 0, 2)
    with pytest.raises(ValueError):
        xrs.cross_rank_swap(torch.zeros(16, dtype=torch.complex128), 4, [(4, 0)], 0, 2)
    with pytest.raises(ValueError):
        xrs.cross_rank_swap(torch.zeros(16, dtype=torch.complex128), 4, [(0, 0)], 0, 3)
