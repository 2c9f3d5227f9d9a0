"""Cross-rank swapping (XRS, Sec. V-C, Alg. 5): exchange local and global qubits of a state split
over 2^R ranks.

The state of n qubits is split by its top R physical bits: rank r holds the 2^(n-R) amplitudes
whose global bits equal r, as a local slice indexed by the low n-R bits.  Swapping local bit l
with global bit j (physical position n-R+j) moves every amplitude whose bit l differs from its
rank's bit j to the partner rank r ^ 2^j, into the position with bit l flipped; the others stay.
So each pair of ranks exchanges exactly half of its slice, and no arithmetic is done.  A list of
(l, j) pairs is applied one pair after another (each pair is its own exchange, matching a
``CSQS k l1..lk g1..gk`` line read left to right).

Works on any tensor torch.distributed can send: CPU tensors over gloo, device tensors over NCCL.
Only data movement happens here; gates on local bits run through the single-GPU library.
"""
from __future__ import annotations

import torch


def _half_index(n_local: int, l: int, bit_value: int, device) -> torch.Tensor:
    """Local indices whose bit l equals bit_value, ascending."""
    idx = torch.arange(1 << (n_local - 1), device=device, dtype=torch.int64)
    low = idx & ((1 << l) - 1)
    return ((idx >> l) << (l + 1)) | (bit_value << l) | low


def cross_rank_swap(local: torch.Tensor, n_local: int, pairs, rank: int, world_size: int, group=None):
    """In place on `local` (1-D, 2^n_local entries): exchange local bit l with global bit j for
    each (l, j) in `pairs`.  world_size = 2^R; every rank of the group must call this with the
    same pairs."""
    import torch.distributed as dist

    if local.dim() != 1 or local.numel() != (1 << n_local):
        raise ValueError("local slice must be a 1-D tensor of 2^n_local entries")
    R = world_size.bit_length() - 1
    if (1 << R) != world_size:
        raise ValueError("world size must be a power of two")
    for l, j in pairs:
        if not (0 <= l < n_local and 0 <= j < R):
            raise ValueError("bad (local, global) bit pair")
        my_bit = (rank >> j) & 1
        partner = rank ^ (1 << j)
        # amplitudes whose local bit l differs from this rank's bit j leave; the partner's
        # matching half arrives in the same positions
        idx = _half_index(n_local, l, 1 - my_bit, local.device)
        send = local.index_select(0, idx).contiguous()
        recv = torch.empty_like(send)
        ops = [dist.P2POp(dist.isend, send, partner, group), dist.P2POp(dist.irecv, recv, partner, group)]
        for req in dist.batch_isend_irecv(ops):
            req.wait()
        local.index_copy_(0, idx, recv)
    return local


def split_state(state: torch.Tensor, n: int, world_size: int, rank: int) -> torch.Tensor:
    """Rank r's slice of a full state (top log2(world_size) bits = r)."""
    n_local = n - (world_size.bit_length() - 1)
    return state[rank << n_local:(rank + 1) << n_local].clone()
