"""Batched training (vjb_batch_*) against the plain path, through the C ABI.

A batch runs every job's round with one launch of each round kernel; each
job must come out exactly as it does alone in a context: the same stumps
(feature, threshold, polarity, split, FP64 error, beta, alpha) and the same
FP32 weights, bit for bit.  The plain path itself is held to the oracle by
the parity tests; here the first stump of every job is also checked against
the oracle directly.
"""

import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_1306_1467_gb300 import synth

pytestmark = pytest.mark.gpu

REL = 1e-6


def _plain(px, y, rounds):
    from paper_1306_1467_gb300 import vjb
    with vjb.Trainer(0) as tr:
        tr.prepare(px, y)
        st, stumps = tr.train_strong(rounds)
        return st, stumps, tr.get_weights()


def _perfect_job():
    px = np.zeros((8, 4, 4), np.uint8)
    y = np.array([1, 0, 1, 0, 0, 1, 0, 0], np.uint8)
    px[y == 1, 1, 2] = 200
    return px, y


def _nogain_job():
    return np.full((6, 4, 4), 77, np.uint8), np.array([1, 0, 1, 0, 1, 0], np.uint8)


def _jobs():
    """Uneven jobs: ragged N, odd windows, a single-copy weight layout (N > 16351),
    one that ends with a perfect stump and one that can gain nothing."""
    out = []
    for (n_pos, n_neg, h, w, seed, rounds) in [(300, 477, 9, 7, 41, 6), (700, 1400, 12, 16, 42, 9),
                                                (1, 1, 3, 3, 43, 2), (5000, 11400, 8, 8, 44, 4),
                                                (2500, 3100, 10, 10, 45, 12)]:
        px, y = synth.make_windows(n_pos, n_neg, h, w, seed=seed)
        out.append((px, y, rounds))
    px, y = _perfect_job()
    out.append((px, y, 5))
    px, y = _nogain_job()
    out.append((px, y, 5))
    return out


def _same(batch, jid, px, y, rounds):
    from paper_1306_1467_gb300 import vjb
    st_p, stumps_p, w_p = _plain(px, y, rounds)
    got = batch.stumps(jid)
    assert got == stumps_p, jid
    assert np.array_equal(batch.get_weights(jid), w_p), jid
    done, st = batch.job_state(jid)
    assert done == len(stumps_p)
    if st_p != vjb.OK:
        assert st == st_p
    return got


def test_batch_equals_plain_per_job():
    from paper_1306_1467_gb300 import vjb
    jobs = _jobs()
    budget = sum(vjb.Batch.table_bytes(px.shape[0], px.shape[1], px.shape[2]) for px, _, _ in jobs)
    with vjb.Batch(budget) as b:
        ids = [b.add_job(px, y, r) for px, y, r in jobs]
        assert b.info()["free_bytes"] == 0
        ran = b.train()
        assert ran == max(r for _, _, r in jobs)
        for jid, (px, y, r) in zip(ids, jobs):
            got = _same(b, jid, px, y, r)
            if got:  # the first stump against the oracle (Sec. 2.3 step 2, FP64)
                P = O.Prepared(px, y)
                ref = O.select(O.feature_best_sorted(P.vals, P.order, y, O.initial_weights(y)))
                assert abs(got[0]["error"] - ref["err"]) <= REL * max(ref["err"], 1e-300)
        assert b.job_state(ids[5]) == (1, vjb.DONE_PERFECT) and math.isinf(b.stumps(ids[5])[0]["alpha"])
        assert b.job_state(ids[6]) == (0, vjb.DONE_NOGAIN)
        assert b.train() == 0  # nothing left to do


def test_batch_jobs_change_between_calls():
    """Jobs leave and join between calls; a job trained across several calls,
    in changing company, still equals its plain run."""
    from paper_1306_1467_gb300 import vjb
    ja = synth.make_windows(400, 900, 12, 12, seed=51)
    jb = synth.make_windows(1500, 2100, 10, 14, seed=52)
    jc = synth.make_windows(777, 1234, 11, 9, seed=53)
    tb = [vjb.Batch.table_bytes(px.shape[0], px.shape[1], px.shape[2]) for px, _ in (ja, jb, jc)]
    with vjb.Batch(max(tb[0] + tb[1], tb[1] + tb[2])) as b:
        a = b.add_job(*ja, rounds=7)
        bb = b.add_job(*jb, rounds=10)
        assert b.train(3) == 3
        assert b.job_state(a)[0] == 3 and b.job_state(bb)[0] == 3
        _same(b, a, *ja, 3)  # a's first three rounds
        b.remove_job(a)
        c = b.add_job(*jc, rounds=5)
        assert b.train(2) == 2
        assert b.info()["rows_per_warp"] == vjb.BATCH_INTERLEAVED
        b.set_search_shape(warps=8, stages=3, rows_per_warp=4)  # work queue; results do not depend on it
        b.train()
        _same(b, bb, *jb, 10)
        _same(b, c, *jc, 5)


def test_batch_budget_admission():
    from paper_1306_1467_gb300 import vjb
    ja = synth.make_windows(600, 600, 12, 12, seed=61)
    jb = synth.make_windows(900, 1100, 12, 12, seed=62)
    ta = vjb.Batch.table_bytes(1200, 12, 12)
    tbb = vjb.Batch.table_bytes(2000, 12, 12)
    assert ta == 2 * O.haar_enumerate(12, 12)[0].shape[0] * 1280  # 2 F npad, npad = N rounded up to 256
    with vjb.Batch(max(ta, tbb) + 128) as b:
        a = b.add_job(*ja, rounds=2)
        with pytest.raises(vjb.VJBError) as ei:
            b.add_job(*jb, rounds=2)
        assert ei.value.code == vjb.EFULL
        b.train()
        b.remove_job(a)
        assert b.info()["free_bytes"] == b.info()["budget_bytes"]
        j = b.add_job(*jb, rounds=2)
        b.train()
        _same(b, j, *jb, 2)
    with pytest.raises(vjb.VJBError) as ei:
        vjb.Batch(64)
    assert ei.value.code == vjb.EINVAL


def test_batch_autotune_keeps_results():
    from paper_1306_1467_gb300 import vjb
    ja = synth.make_windows(2000, 3000, 16, 16, seed=71)
    jb = synth.make_windows(1000, 1900, 14, 14, seed=72)
    budget = sum(vjb.Batch.table_bytes(px.shape[0], px.shape[1], px.shape[2]) for px, _ in (ja, jb))
    with vjb.Batch(budget) as b:
        a = b.add_job(*ja, rounds=30)
        c = b.add_job(*jb, rounds=30)
        ran = b.autotune(trial_rounds=1)
        assert 2 <= ran <= 30
        info = b.info()
        assert info["warps"] >= 1 and info["rows_per_warp"] != 0
        b.train()
        _same(b, a, *ja, 30)
        _same(b, c, *jb, 30)


def test_batch_schedules_agree():
    """The interleaved, partitioned and work-queue schedules, switched between
    rounds, give every job its plain result."""
    from paper_1306_1467_gb300 import vjb
    jobs = [synth.make_windows(700, 1200, 12, 12, seed=81), synth.make_windows(3000, 5200, 10, 10, seed=82),
            synth.make_windows(90, 150, 14, 14, seed=83)]
    budget = sum(vjb.Batch.table_bytes(px.shape[0], px.shape[1], px.shape[2]) for px, _ in jobs)
    with vjb.Batch(budget) as b:
        ids = [b.add_job(px, y, rounds=9) for px, y in jobs]
        for sched, warps, unroll, box in ((vjb.BATCH_INTERLEAVED, 16, 3, 24), (vjb.BATCH_PARTITIONED, 12, 4, 32),
                                          (8, 16, 2, 16)):
            b.set_search_shape(warps=warps, unroll=unroll, rows_per_warp=sched, box_lines=box)
            assert b.info()["rows_per_warp"] == sched and b.info()["box_lines"] == box
            b.train(3)
        for jid, (px, y) in zip(ids, jobs):
            _same(b, jid, px, y, 9)
