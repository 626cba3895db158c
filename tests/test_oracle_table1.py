"""Pins Algs 2-4 of the oracle to the paper's worked example (Table 1)."""
import os

import numpy as np

import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "table1_worked_example.txt")


def _load():
    rows = {}
    with open(GOLDEN) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            key, *vals = line.split()
            rows[key] = vals
    return rows


def _label_ids(rows):
    """Node labels 1..10 -> 0-based ids; X (no receiver) -> self."""
    labels = [int(v) for v in rows["cell"]]
    idx = {lab: i for i, lab in enumerate(labels)}
    rec = np.array([idx[int(v)] if v != "X" else i for i, v in enumerate(rows["rec"])],
                   np.int32)
    return labels, idx, rec


def test_table1_donors_dnum():
    rows = _load()
    labels, idx, rec = _label_ids(rows)
    dnum, donor = oracle.donors_graph(rec, dmax=8)
    assert dnum.tolist() == [int(v) for v in rows["dnum"]]
    want = {lab: [] for lab in labels}
    for item in rows["donors"]:
        c, ds = item.split(":")
        want[int(c)] = [int(d) for d in ds.split(",")]
    for lab in labels:
        i = idx[lab]
        got = [labels[d] for d in donor[i, :dnum[i]]]
        assert got == want[lab], (lab, got)


def test_table1_queue_levels():
    rows = _load()
    labels, idx, rec = _label_ids(rows)
    dnum, donor = oracle.donors_graph(rec, dmax=8)
    q, lev, depth = oracle.queue(rec, dnum, donor)
    assert [labels[c] for c in q] == [int(v) for v in rows["queue"]]
    assert lev.tolist() == [int(v) for v in rows["levels"]]
    # depth of every node = number of receiver hops to node 5 (the outlet)
    for i in range(len(labels)):
        hops, c = 0, i
        while rec[c] != c:
            c = rec[c]
            hops += 1
        assert depth[i] == hops


def test_table1_accumulation():
    rows = _load()
    labels, idx, rec = _label_ids(rows)
    dnum, donor = oracle.donors_graph(rec, dmax=8)
    q, lev, depth = oracle.queue(rec, dnum, donor)
    acc = oracle.accumulate(q, lev, dnum, donor)
    assert acc.tolist() == [int(v) for v in rows["accum"]]
