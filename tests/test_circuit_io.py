"""Circuit text I/O: the paper's raw format (parse / write) and optimized listings of plans
replayed with the FP64 oracle against the raw circuit (host only)."""
import os

import numpy as np
import pytest

import oracle
from listing_replay import replay_listing
from paper_2406_14084_gb300 import circuit_io
from paper_2406_14084_gb300 import qs
from paper_2406_14084_gb300 import workloads as W
from paper_2406_14084_gb300.workloads import Gate

GOLD = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def test_parse_worked_example_raw():
    text = open(os.path.join(GOLD, "worked_example_raw.txt")).read()
    n, gates, ids = circuit_io.parse_circuit(text, angle_from_id=True)
    assert n == 10 and len(gates) == len(ids)
    assert gates[0] == Gate("H", (0,), (), ()) and ids[0] == 0
    rzz = [(g, i) for g, i in zip(gates, ids) if g.kind == "RZZ"]
    assert rzz[0][0].targets == (2, 4) and rzz[0][0].params == (2.0,)  # angle read from the ID
    assert sorted(ids) == list(range(len(ids)))


def test_write_parse_round_trip():
    n = 9
    g = W.random_circuit(n, 80, 3, alphabet=("H", "X", "S", "T", "RZ", "U3", "CX", "CZ", "SWAP", "CP", "RZZ"))
    text = circuit_io.write_circuit(g)
    m, g2, ids = circuit_io.parse_circuit(text)
    assert g2 == [x._replace(params=tuple(float(p) for p in x.params)) for x in g]
    assert ids == list(range(len(g)))
    assert m <= n


@pytest.mark.parametrize("bad", ["FOO 1 0", "H", "RX 0 3", "CZ 1 1 4"])
def test_parse_rejects_bad_lines(bad):
    with pytest.raises(ValueError):
        circuit_io.parse_circuit(bad)


@pytest.mark.parametrize("mode", ["remap", "gather"])
def test_plan_listing_replays_to_the_raw_circuit(mode):
    """Low-block plan of the worked example (4-qubit block): its SQS lines, fused D<k>/U<k> ops
    and final layout, replayed on physical positions, give the raw circuit's state."""
    text = open(os.path.join(GOLD, "worked_example_raw.txt")).read()
    n, gates, _ = circuit_io.parse_circuit(text, angle_from_id=True)
    opts = qs.options(fuse_width=2, slab_bits=4, seg_bits=1,
                      slab_mode=qs.QS_SLAB_REMAP if mode == "remap" else qs.QS_SLAB_GATHER)
    p = qs.qs_fuse(gates, n, opts)
    try:
        listing = circuit_io.plan_listing(p)
    finally:
        qs.qs_plan_destroy(p)
    if mode == "remap":
        assert any(line.startswith("SQS ") for line in listing.splitlines())
    a0 = oracle.apply_circuit(n, [Gate("H", (q,)) for q in range(n)] + [Gate("T", (3,)), Gate("S", (7,))])
    want = oracle.apply_circuit(n, gates, a0.copy())
    got = a0.copy()
    layout = replay_listing(listing, n, got)
    # physical -> logical: logical qubit q sits at physical position layout[q]
    idx = np.arange(1 << n)
    phys = np.zeros_like(idx)
    for q in range(n):
        phys |= ((idx >> q) & 1) << layout[q]
    assert np.max(np.abs(got[phys] - want)) < 1e-12
