"""The clean-set bookkeeping of the FP32 error split (tests/fp32_split.py) on
hand-made graphs: a receiver flip or a count change marks the cell and every
cell that drains through it; the rest stays clean."""
import numpy as np

from fp32_split import clean_update


def _chain_graph():
    # cells 0..5: 0 is a root; 1->0, 2->1, 3->2, 4->0, 5->4 (self = root)
    rec = np.array([0, 0, 1, 2, 0, 4], np.int32)
    queue = np.array([0, 1, 4, 2, 5, 3], np.int32)
    levels = np.array([0, 1, 3, 5, 6], np.int64)
    cnt = np.array([6, 3, 2, 1, 2, 1], np.int64)
    return rec, cnt, queue, levels


def test_identical_runs_stay_clean():
    rec, cnt, q, lev = _chain_graph()
    c = clean_update(np.ones(6, bool), rec, cnt, rec.copy(), cnt.copy(), q, lev)
    assert c.all()


def test_flip_marks_the_cell_and_its_upstream_cells():
    rec, cnt, q, lev = _chain_graph()
    rec32 = rec.copy()
    rec32[2] = 4  # cell 2 drains to 4 in the FP32 run; counts along both paths change
    cnt32 = np.array([6, 1, 2, 1, 4, 1], np.int64)
    c = clean_update(np.ones(6, bool), rec, cnt, rec32, cnt32, q, lev)
    # 2 flipped; 3 drains through 2; 1 and 4 changed counts; 5 drains through 4
    assert c.tolist() == [True, False, False, False, False, False]


def test_dirty_state_persists_and_propagates_upstream_only():
    rec, cnt, q, lev = _chain_graph()
    prev = np.ones(6, bool)
    prev[4] = False  # 4's elevation already differs
    c = clean_update(prev, rec, cnt, rec.copy(), cnt.copy(), q, lev)
    assert c.tolist() == [True, True, True, True, False, False]
