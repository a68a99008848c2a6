"""The allocation-free search entry point, vjb_screen_noalloc.

It is for callers that cannot allocate device memory when they search (a host
capturing its own CUDA graph, a real-time loop with memory fixed up front, a
framework whose pool owns the device).  The test builds a caller-owned copy of
a trained context's sorted table and weights with torch (the test may
allocate; the entry point must not), calls the entry point through the C ABI
twice in a row -- each time on the weights of the next round -- and compares
its per-feature errors and its best feature with the library's own search of
that round (vjb_train_round, read back with vjb_screen_errors).  Each search
is within the screening tolerance of the other GPU tests of the exact errors,
so the two agree within twice that tolerance.

The file is named so that pytest collects it last.
"""

import ctypes as C

import numpy as np
import pytest

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
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    lib = vjb.load_library()
    with vjb.Trainer(0) as tr:
        feats = tr.prepare(px, y)
        nf = feats.shape[0]
        table = np.full((nf, npad), n, np.uint16)
        table[:, :n] = tr.sorted_rows(0, nf)
        rows_d = torch.from_numpy(table.view(np.int16)).to(dev)
        ferr_d = torch.empty(nf, dtype=torch.float32, device=dev)
        best_e = torch.empty(1, dtype=torch.float32, device=dev)
        best_f = torch.empty(1, dtype=torch.int32, device=dev)
        for call in range(2):
            w = tr.get_weights()
            v = np.append(np.where(y == 1, w, -w), np.float32(0)).astype(np.float32)
            t_pos = float(np.sum(w[y == 1], dtype=np.float64))
            t_neg = float(np.sum(w[y == 0], dtype=np.float64))
            v_d = torch.from_numpy(v).to(dev)
            ferr_d.fill_(-1.0)
            torch.cuda.synchronize()
            rc = lib.vjb_screen_noalloc(rows_d.data_ptr(), v_d.data_ptr(), n, npad, nf, t_pos, t_neg,
                                        0, ferr_d.data_ptr(), best_e.data_ptr(), best_f.data_ptr(), None)
            assert rc == vjb.OK, lib.vjb_last_error()
            torch.cuda.synchronize()
            got = ferr_d.cpu().numpy()
            # the library's own search of the same round, on the same weights
            st, _ = tr.train_round()
            assert st == vjb.OK
            ref = tr.screen_errors()
            assert np.max(np.abs(got.astype(np.float64) - ref)) <= PAIR_TOL, call
            bf = int(best_f.item())
            assert bf == int(np.argmin(got)), call
            assert abs(float(best_e.item()) - float(tr.info()["screen_min"])) <= PAIR_TOL, call


def test_noalloc_rejects_sizes_beyond_its_scratch():
    from paper_1306_1467_gb300 import vjb
    lib = vjb.load_library()
    dummy = C.c_void_p(16)  # never dereferenced: the call is rejected before any launch
    rc = lib.vjb_screen_noalloc(dummy, dummy, 100, 128, 10, 0.5, 0.5, 1025, dummy, dummy, dummy, None)
    assert rc == vjb.EINVAL
    assert b"1024" in lib.vjb_last_error()
    rc = lib.vjb_screen_noalloc(dummy, dummy, 100, 100, 10, 0.5, 0.5, 0, dummy, dummy, dummy, None)
    assert rc == vjb.EINVAL  # npad not a multiple of 64
