"""The sort evaluates a feature whose box holds at most 257 pixels from the
integral images modulo 2^16 (half the bytes of the int32 ones): its values
span at most 255 * 257 = 65,535 integers, so the residue modulo 2^16 names
one of them, the one in [-255 * (subtracted area), that + 65,535].  Pin of
that reading on the CPU, against the oracle's own values: the oracle's
feature arithmetic (Sec. 2.1-2.2) applied to the integral images reduced
modulo 2^16, then lifted, gives the oracle's values for every small box, on
random windows and on windows that drive features to both ends of their
range; for boxes above the bound the same lift fails on such windows, so
the bound is not loose in the wrong direction."""

import numpy as np

import oracle as O

TYPES = ("3H", "3V", "2H", "2V", "4")  # canonical type order (vjb.h)
NARROW = 257


def _windows(side, n, seed):
    rng = np.random.Generator(np.random.PCG64(seed))
    grid = np.indices((side, side))
    pats = [np.zeros((side, side)), np.full((side, side), 255)]
    for axis in (0, 1):
        c = grid[axis]
        pats += [np.where(c < side // 2, 255, 0), np.where(c < side // 2, 0, 255)]
        for k in range(3):
            band = (c >= k * side // 3) & (c < (k + 1) * side // 3)
            pats += [np.where(band, 255, 0), np.where(band, 0, 255)]
    quad = (grid[0] < side // 2) ^ (grid[1] < side // 2)
    pats += [np.where(quad, 255, 0), np.where(quad, 0, 255)]
    px = rng.integers(0, 256, size=(n, side, side))
    px[: len(pats)] = np.stack(pats)
    px[len(pats): 2 * len(pats)] = (rng.random((len(pats), side, side)) < 0.5) * 255
    return px.astype(np.uint8)


def _subtracted_area(desc):
    t, w, h = desc[:, 0], desc[:, 3].astype(np.int64), desc[:, 4].astype(np.int64)
    three = (t == TYPES.index("3H")) | (t == TYPES.index("3V"))
    return np.where(three, 2 * w * h // 3, w * h // 2)


def test_small_boxes_from_integral_images_modulo_2_16():
    side = 24
    px = _windows(side, 160, seed=1311)
    desc, _ = O.haar_enumerate(side, side)
    ii = O.integral(px)
    exact = O.feature_values(px, desc, ii).astype(np.int64)
    resid = O.feature_values(px, desc, (ii % 65536).astype(ii.dtype)).astype(np.int64)
    lo = -255 * _subtracted_area(desc)[:, None]
    lifted = lo + np.mod(resid - lo, 65536)
    area = desc[:, 3].astype(np.int64) * desc[:, 4]
    small = area <= NARROW
    assert small.mean() > 0.95  # 96% of the 24x24 features
    # the range bound itself: every value lies in [lo, lo + 255 * area]
    assert (exact >= lo).all() and (exact <= lo + 255 * area[:, None]).all()
    assert np.array_equal(lifted[small], exact[small])
    # some small boxes reach both ends of their range on these windows
    ends = (exact.min(axis=1) == lo[:, 0]) & (exact.max(axis=1) == lo[:, 0] + 255 * area)
    assert (ends & small & (area >= 250)).any()
    # above the bound the residue no longer names the value
    big = area > NARROW
    assert (lifted[big] != exact[big]).any(axis=1).sum() > 0.5 * big.sum()
