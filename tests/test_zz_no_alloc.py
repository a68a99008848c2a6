"""The allocation-free search entry point, vjb_screen_noalloc.

It is for callers that cannot allocate device memory when they search: a
real-time loop whose memory is fixed up front, or a framework whose memory
pool owns the whole device.  The test builds a caller-owned copy of a trained
context's sorted table and weights with torch (the test may allocate; the
entry point must not) and calls the entry point through the C ABI twice in a
row, each time on the weights of the next round.  Each call's per-feature
errors are compared with the FP64 oracle's per-feature minima on the same
weights (within the screening bound), with the library's own search of that
round (vjb_train_round, read back with vjb_screen_errors), and with the same
call at one CTA and at 1024 CTAs, the most its scratch array holds (bit for
bit: a feature's error does not depend on the grid).  Free device memory must
not change across the calls after the first.

The file is named so that pytest collects it last.
"""

import ctypes as C

import numpy as np
import pytest

import oracle as O

pytestmark = pytest.mark.gpu

SCREEN_TOL = 36 * 2.0 ** -24  # the screening bound used by the parity tests
# both searches lie within SCREEN_TOL of the exact errors, summed in different orders
PAIR_TOL = 2 * SCREEN_TOL


def test_noalloc_search_matches_library_search():
    torch = pytest.importorskip("torch")
    from paper_1306_1467_gb300 import synth, vjb

    px, y = synth.make_windows(300, 477, 12, 10, seed=31)  # ragged N, non-square window
    n = px.shape[0]
    npad = (n + 63) // 64 * 64
    P = O.Prepared(px, y)
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    lib = vjb.load_library()
    with vjb.Trainer(0) as tr:
        feats = tr.prepare(px, y)
        assert np.array_equal(feats, P.desc)
        nf = feats.shape[0]
        table = np.full((nf, npad), n, np.uint16)
        table[:, :n] = tr.sorted_rows(0, nf)
        rows_d = torch.from_numpy(table.view(np.int16)).to(dev)
        ferr_d = torch.empty(nf, dtype=torch.float32, device=dev)
        best_e = torch.empty(1, dtype=torch.float32, device=dev)
        best_f = torch.empty(1, dtype=torch.int32, device=dev)
        v_d = torch.empty(n + 1, dtype=torch.float32, device=dev)

        def screen(t_pos, t_neg, ctas):
            ferr_d.fill_(-1.0)
            best_e.fill_(-1.0)
            best_f.fill_(-2)
            rc = lib.vjb_screen_noalloc(rows_d.data_ptr(), v_d.data_ptr(), n, npad, nf, t_pos, t_neg,
                                        ctas, ferr_d.data_ptr(), best_e.data_ptr(), best_f.data_ptr(), None)
            assert rc == vjb.OK, lib.vjb_last_error()
            torch.cuda.synchronize()
            return ferr_d.cpu().numpy(), float(best_e.item()), int(best_f.item())

        for call in range(2):
            w = tr.get_weights()
            v = np.append(np.where(y == 1, w, -w), np.float32(0)).astype(np.float32)
            t_pos = float(np.sum(w[y == 1], dtype=np.float64))
            t_neg = float(np.sum(w[y == 0], dtype=np.float64))
            v_d.copy_(torch.from_numpy(v))
            torch.cuda.synchronize()
            free0 = torch.cuda.mem_get_info()[0]
            got, be, bf = screen(t_pos, t_neg, 0)
            # the grid's extremes: one CTA, and the 1024 partials the scratch array holds
            for ctas in (1, 1024):
                g2, be2, bf2 = screen(t_pos, t_neg, ctas)
                assert np.array_equal(g2, got) and be2 == be and bf2 == bf, (call, ctas)
            if call > 0:  # the first call on the device did its one-time set-up
                assert torch.cuda.mem_get_info()[0] == free0, call
            # the oracle's per-feature minima on the same weights (FP64, not renormalised)
            ref = O.feature_best_sorted(P.vals, P.order, y, w.astype(np.float64))["err"]
            assert np.max(np.abs(got.astype(np.float64) - ref)) <= SCREEN_TOL, call
            assert bf == int(np.argmin(got)) and be == float(got[bf]), call
            # the chosen feature is the oracle's best unless another lies within
            # both screens' error of it
            assert ref[bf] - ref.min() <= PAIR_TOL, call
            if np.sort(ref)[1] - ref.min() > PAIR_TOL:
                assert bf == int(np.argmin(ref)), call
            # the library's own search of the same round, on the same weights
            st, _ = tr.train_round()
            assert st == vjb.OK
            lib_err = tr.screen_errors()
            assert np.max(np.abs(got.astype(np.float64) - lib_err)) <= PAIR_TOL, call
            assert abs(be - float(tr.info()["screen_min"])) <= PAIR_TOL, call


def test_noalloc_rejects_sizes_beyond_its_scratch():
    from paper_1306_1467_gb300 import vjb
    lib = vjb.load_library()
    dummy = C.c_void_p(16)  # never dereferenced: the call is rejected before any launch
    rc = lib.vjb_screen_noalloc(dummy, dummy, 100, 128, 10, 0.5, 0.5, 1025, dummy, dummy, dummy, None)
    assert rc == vjb.EINVAL
    assert b"1024" in lib.vjb_last_error()
    rc = lib.vjb_screen_noalloc(dummy, dummy, 100, 100, 10, 0.5, 0.5, 0, dummy, dummy, dummy, None)
    assert rc == vjb.EINVAL  # npad not a multiple of 64
