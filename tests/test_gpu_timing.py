"""Event timing of rounds (vjb_set_timing / vjb_get_timing and the batch's).

The benchmark's roofline figure is the search kernel's average launch time
from these events, so they must cover every round run while timing is on,
order correctly (search inside round), and change no result: a timed run
keeps the same stumps and weights as an untimed one.
"""

import numpy as np
import pytest

from paper_1306_1467_gb300 import synth

pytestmark = pytest.mark.gpu


def _check(t, rounds):
    assert t["rounds"] == rounds
    assert t["search_ms_total"] > 0.0
    assert 0.0 < t["search_ms_min"] <= t["search_ms_total"] / rounds <= t["search_ms_max"]
    # each round holds its search, so the rounds take at least as long
    assert t["round_ms_total"] >= t["search_ms_total"]


def test_timed_rounds_are_counted_and_change_nothing():
    from paper_1306_1467_gb300 import vjb
    px, y = synth.make_windows(700, 1300, 12, 12, seed=61)
    with vjb.Trainer(0) as a, vjb.Trainer(0) as b:
        a.prepare(px, y)
        b.prepare(px, y)
        a.set_timing(True)
        sa = a.train_strong(6)
        _check(a.timing(), 6)
        sa2 = a.train_round()
        _check(a.timing(), 7)  # single rounds are timed too
        sa3 = a.train_strong(4)
        _check(a.timing(), 11)  # accumulated over calls
        a.set_timing(True)  # re-enabling clears the figures
        assert a.timing()["rounds"] == 0
        sb = b.train_strong(6)
        sb2 = b.train_round()
        sb3 = b.train_strong(4)
        assert sa == sb and sa2 == sb2 and sa3 == sb3
        assert np.array_equal(a.get_weights(), b.get_weights())
        a.set_timing(False)
        a.train_strong(2)
        assert a.timing()["rounds"] == 0  # nothing is timed while timing is off


def test_batch_rounds_are_timed():
    from paper_1306_1467_gb300 import vjb
    jobs = [synth.make_windows(400, 600, 10, 10, seed=62), synth.make_windows(900, 700, 12, 12, seed=63)]
    budget = sum(vjb.Batch.table_bytes(px.shape[0], px.shape[1], px.shape[2]) for px, _ in jobs)
    with vjb.Batch(budget) as b:
        for px, y in jobs:
            b.add_job(px, y, 5)
        b.set_timing(True)
        assert b.train() == 5
        _check(b.timing(), 5)
