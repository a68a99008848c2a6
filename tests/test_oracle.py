"""Pins for the CPU oracle: each test checks the oracle against something other
than itself -- numbers printed in the paper, closed forms, library routines,
brute force on tiny inputs, and identities of discrete AdaBoost."""

import math
import os

import numpy as np
import pytest

import oracle as O
from paper_1306_1467_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
TYPES = ["3H", "3V", "2H", "2V", "4"]
BASE = {"3H": (3, 1), "3V": (1, 3), "2H": (2, 1), "2V": (1, 2), "4": (2, 2)}


def _read_golden(name):
    out = {}
    with open(os.path.join(GOLDEN, name)) as fh:
        for line in fh:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            k, v = line.split()
            out[k] = int(v)
    return out


# ------------------------------------------------------------------ Sec. 2.2

def test_counts_match_paper():
    g = _read_golden("haar_counts_24x24.txt")
    desc, per = O.haar_enumerate(24, 24)
    for t, name in enumerate(TYPES):
        assert per[t] == g[name], name
    assert desc.shape[0] == g["total"] == 162336


def test_paper_training_set_arithmetic():
    g = _read_golden("paper_training_set.txt")
    n = g["faces"] + g["nonfaces"]
    desc, _ = O.haar_enumerate(24, 24)
    assert desc.shape[0] == g["features"]
    assert desc.shape[0] * n == g["feature_values"]


def _closed_form(W, H, bw, bh):
    # a feature k*bw wide fits at W - k*bw + 1 horizontal positions
    sx = sum(W - k * bw + 1 for k in range(1, W // bw + 1))
    sy = sum(H - j * bh + 1 for j in range(1, H // bh + 1))
    return sx * sy


@pytest.mark.parametrize("W,H", [(10, 10), (20, 20), (24, 24), (32, 32), (7, 13), (3, 2), (1, 1)])
def test_counts_closed_form(W, H):
    desc, per = O.haar_enumerate(W, H)
    for t, name in enumerate(TYPES):
        assert per[t] == _closed_form(W, H, *BASE[name]), (W, H, name)
    assert desc.shape[0] == sum(per)


def test_known_totals():
    # totals for other window sizes from the same closed form
    assert O.haar_enumerate(10, 10)[0].shape[0] == 5025
    assert O.haar_enumerate(20, 20)[0].shape[0] == 78460
    assert O.haar_enumerate(32, 32)[0].shape[0] == 510112


def test_enumeration_canonical_order_and_fit():
    W, H = 11, 9
    desc, _ = O.haar_enumerate(W, H)
    t, x, y, w, h = desc.T
    assert np.all(x + w <= W) and np.all(y + h <= H) and np.all(x >= 0) and np.all(y >= 0)
    for k, name in enumerate(TYPES):
        bw, bh = BASE[name]
        m = t == k
        assert np.all(w[m] % bw == 0) and np.all(h[m] % bh == 0)
    key = np.lexsort((x, y, h, w, t))  # primary key last: type, width, height, y, x
    assert np.array_equal(key, np.arange(desc.shape[0]))
    assert len({tuple(r) for r in desc.tolist()}) == desc.shape[0]


# ------------------------------------------------------------------ Sec. 2.1

def test_integral_matches_cumsum():
    rng = np.random.default_rng(1)
    px = rng.integers(0, 256, size=(7, 9, 13), dtype=np.uint8)
    ii = O.integral(px)
    ref = np.zeros((7, 10, 14), np.int64)
    ref[:, 1:, 1:] = np.cumsum(np.cumsum(px.astype(np.int64), axis=1), axis=2)
    assert np.array_equal(ii, ref)
    # the largest value a 24x24 window can reach fits int32
    full = np.full((1, 24, 24), 255, np.uint8)
    assert O.integral(full)[0, 24, 24] == 24 * 24 * 255


def test_values_direct_vs_integral(tiny):
    px, _ = tiny
    desc, _ = O.haar_enumerate(10, 10)
    a = O.feature_values_direct(px, desc)
    b = O.feature_values(px, desc)
    assert np.array_equal(a, b)


def _slice_sum(img, x, y, w, h):
    return int(img[y:y + h, x:x + w].astype(np.int64).sum())


def test_values_vs_numpy_slices():
    rng = np.random.default_rng(2)
    px = rng.integers(0, 256, size=(5, 24, 24), dtype=np.uint8)
    desc, _ = O.haar_enumerate(24, 24)
    pick = rng.choice(desc.shape[0], size=400, replace=False)
    sub = desc[pick]
    got = O.feature_values(px, sub)
    for r, (t, x, y, w, h) in enumerate(sub):
        for i in range(px.shape[0]):
            img = px[i]
            S = lambda xx, yy, ww, hh: _slice_sum(img, xx, yy, ww, hh)  # noqa: E731
            if TYPES[t] == "2H":
                a = w // 2
                exp = S(x + a, y, a, h) - S(x, y, a, h)
            elif TYPES[t] == "2V":
                b = h // 2
                exp = S(x, y + b, w, b) - S(x, y, w, b)
            elif TYPES[t] == "3H":
                a = w // 3
                exp = S(x + a, y, a, h) - S(x, y, a, h) - S(x + 2 * a, y, a, h)
            elif TYPES[t] == "3V":
                b = h // 3
                exp = S(x, y + b, w, b) - S(x, y, w, b) - S(x, y + 2 * b, w, b)
            else:
                a, b = w // 2, h // 2
                exp = S(x + a, y, a, b) + S(x, y + b, a, b) - S(x, y, a, b) - S(x + a, y + b, a, b)
            assert got[r, i] == exp


def _impulse(W, H, px_x, px_y):
    img = np.zeros((1, H, W), np.uint8)
    img[0, px_y, px_x] = 1
    return img


@pytest.mark.parametrize("name,feat,probes", [
    # (x, y, w, h); probes: pixel -> expected value (dark +1, white -1)
    ("2H", (2, 1, 4, 3), {(2, 1): -1, (3, 3): -1, (4, 1): +1, (5, 3): +1, (6, 1): 0}),
    ("2V", (1, 2, 3, 4), {(1, 2): -1, (3, 3): -1, (1, 4): +1, (3, 5): +1, (1, 6): 0}),
    ("3H", (0, 0, 6, 2), {(0, 0): -1, (1, 1): -1, (2, 0): +1, (3, 1): +1, (4, 0): -1, (5, 1): -1}),
    ("3V", (0, 0, 2, 6), {(0, 0): -1, (1, 1): -1, (0, 2): +1, (1, 3): +1, (0, 4): -1, (1, 5): -1}),
    ("4", (1, 1, 4, 4), {(1, 1): -1, (2, 2): -1, (3, 1): +1, (4, 2): +1,
                         (1, 3): +1, (2, 4): +1, (3, 3): -1, (4, 4): -1, (0, 0): 0}),
])
def test_impulse_sign_convention(name, feat, probes):
    W = H = 8
    t = TYPES.index(name)
    desc = np.array([[t, *feat]], np.int32)
    for (px_x, px_y), want in probes.items():
        img = _impulse(W, H, px_x, px_y)
        assert O.feature_values(img, desc)[0, 0] == want, (px_x, px_y)
        assert O.feature_values_direct(img, desc)[0, 0] == want


# ------------------------------------------------------------ value order

def test_sort_matches_numpy_stable():
    rng = np.random.default_rng(3)
    vals = rng.integers(-5, 6, size=(50, 301)).astype(np.int32)  # many ties
    order = O.sort_rows(vals)
    ref = np.argsort(vals, axis=1, kind="stable")
    assert np.array_equal(order, ref)


# ------------------------------------------------------------ Sec. 2.2-2.3 stump

def test_hand_worked_stump():
    # one feature, six samples; sample 2 carries twice the weight.
    # value order: 1(y0) 2(y0) 3(y0,w2) 3(y1) 5(y1) 7(y1); split 3 is inside a tie.
    # p=-1 (above is a face): s=4 leaves only sample 3 (face, value 3) wrong: 1/7.
    vals = np.array([[5, 1, 3, 3, 7, 2]], np.int32)
    y = np.array([1, 0, 0, 1, 1, 0], np.uint8)
    w = O.normalize(np.array([1, 1, 2, 1, 1, 1], np.float64))
    for best in (O.feature_best_sorted(vals, O.sort_rows(vals), y, w), O.feature_best_brute(vals, y, w)):
        assert best["split"][0] == 4 and best["polarity"][0] == -1 and best["threshold"][0] == 3
        assert abs(best["err"][0] - 1 / 7) < 1e-15
        assert abs(best["err2"][0] - 2 / 7) < 1e-15


def test_brute_force_pins_sorted_scan(tiny_prepared):
    P = tiny_prepared
    rng = np.random.default_rng(4)
    for w in (O.normalize(O.initial_weights(P.y)), O.normalize(rng.random(P.y.shape[0]) ** 3)):
        a = O.feature_best_brute(P.vals, P.y, w)
        b = O.feature_best_sorted(P.vals, P.order, P.y, w)
        assert np.max(np.abs(a["err"] - b["err"])) < 1e-12
        assert np.max(np.abs(a["err2"] - b["err2"])) < 1e-12
        clear = (b["err2"] - b["err"]) > 1e-12
        assert clear.sum() > 0.5 * clear.size
        for k in ("split", "polarity", "threshold"):
            assert np.array_equal(a[k][clear], b[k][clear]), k
        ca, cb = O.select(a), O.select(b)
        assert abs(ca["err"] - cb["err"]) < 1e-12
        if cb["second_err"] - cb["err"] > 1e-12:
            assert (ca["feature"], ca["split"], ca["polarity"]) == (cb["feature"], cb["split"], cb["polarity"])


def test_threshold_reproduces_split_and_error(tiny_prepared):
    P = tiny_prepared
    w = O.normalize(O.initial_weights(P.y))
    b = O.feature_best_sorted(P.vals, P.order, P.y, w)
    rng = np.random.default_rng(5)
    for f in rng.choice(P.vals.shape[0], size=300, replace=False):
        v, th, p, s = P.vals[f], b["threshold"][f], b["polarity"][f], b["split"][f]
        h = (v < th) if p > 0 else (v > th)
        below = h if p > 0 else ~h
        assert below.sum() == s
        direct = float(np.sum(w[h.astype(np.uint8) != P.y]))
        assert abs(direct - b["err"][f]) < 1e-12
        assert abs(O.stump_error(v, P.y, w, int(th), int(p)) - direct) < 1e-12


# ------------------------------------------------------------ Sec. 2.3 boosting

def test_initial_weights_table2(tiny):
    _, y = tiny
    w = O.initial_weights(y)
    l, m = int(y.sum()), int((1 - y).sum())
    assert np.allclose(w[y == 1], 1 / (2 * l)) and np.allclose(w[y == 0], 1 / (2 * m))
    assert abs(w[y == 1].sum() - 0.5) < 1e-12 and abs(w[y == 0].sum() - 0.5) < 1e-12


def test_round_invariants(tiny_prepared):
    """eps <= 1/2, weights a distribution, and after the update the stump just
    chosen has weighted error exactly 1/2 (misclassified mass eps against
    correctly classified mass (1 - eps) beta = eps)."""
    P = tiny_prepared
    w = O.initial_weights(P.y)
    for t in range(8):
        st, s, w_new = O.round_step(P.vals, P.order, P.y, w)
        assert st == O.STATUS_OK
        assert 0.0 < s["err"] <= 0.5
        assert abs(s["beta"] - s["err"] / (1 - s["err"])) < 1e-15
        assert abs(s["alpha"] - math.log(1 / s["beta"])) < 1e-12
        wn = O.normalize(w_new)
        assert abs(wn.sum() - 1.0) < 1e-12
        e_after = O.stump_error(P.vals[s["feature"]], P.y, wn, s["threshold"], s["polarity"])
        assert abs(e_after - 0.5) < 1e-12
        # the round's error is the minimum over every stump: brute force agrees
        brute = O.select(O.feature_best_brute(P.vals, P.y, O.normalize(w)))
        assert abs(brute["err"] - s["err"]) < 1e-12
        w = w_new


def test_freund_schapire_bound(tiny_prepared):
    """Weighted training error of C(x) under the initial distribution is at
    most prod_t 2 sqrt(eps_t (1 - eps_t)) (AdaBoost's training-error bound)."""
    P = tiny_prepared
    w0 = O.normalize(O.initial_weights(P.y))
    st, stumps, _ = O.train(P.vals, P.order, P.y, w0, 10)
    assert st == O.STATUS_OK and len(stumps) == 10
    bound = 1.0
    errs = []
    for T in range(1, 11):
        e = stumps[T - 1]["err"]
        bound *= 2 * math.sqrt(e * (1 - e))
        fval = P.vals[[s["feature"] for s in stumps[:T]]]
        c = O.strong_classify(fval, stumps[:T])
        werr = float(np.sum(w0[c != P.y]))
        assert werr <= bound + 1e-12
        errs.append(werr)
    assert errs[-1] < errs[0]


def test_degenerate_rounds():
    # perfectly separable: one bright pixel marks the faces -> eps = 0, alpha = inf, stop
    px = np.zeros((8, 4, 4), np.uint8)
    y = np.array([1, 0, 1, 0, 0, 1, 0, 0], np.uint8)
    px[y == 1, 1, 2] = 200
    P = O.Prepared(px, y)
    st, stumps, _ = O.train(P.vals, P.order, P.y, O.initial_weights(y), 5)
    assert st == O.STATUS_PERFECT and len(stumps) == 1
    assert stumps[0]["err"] == 0.0 and math.isinf(stumps[0]["alpha"])
    fval = P.vals[[stumps[0]["feature"]]]
    assert np.array_equal(O.strong_classify(fval, stumps), y)
    # identical windows: nothing separates -> eps = 1/2, no stump kept
    px2 = np.full((6, 4, 4), 77, np.uint8)
    y2 = np.array([1, 0, 1, 0, 1, 0], np.uint8)
    P2 = O.Prepared(px2, y2)
    st, stumps, _ = O.train(P2.vals, P2.order, P2.y, O.initial_weights(y2), 5)
    assert st == O.STATUS_NOGAIN and len(stumps) == 0


def test_generator_is_seeded_and_shaped():
    a = synth.make_windows(20, 30, 12, 10, seed=9)
    b = synth.make_windows(20, 30, 12, 10, seed=9)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
    assert a[0].shape == (50, 12, 10) and a[0].dtype == np.uint8
    assert int(a[1].sum()) == 20
