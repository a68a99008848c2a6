"""ctypes wrapper around the plain-C oracle in ``vjb_oracle.c``.

TEST INFRASTRUCTURE ONLY: imported by tests, the smoke check and the benchmark's
CPU-baseline leg, never by the library.  The C file is compiled with gcc on
first use (or by ``build()``) into ``oracle/_build/``.

Every function here only marshals numpy arrays; the arithmetic is in the C
file, whose header lists the paper passages each part follows.
"""

from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "vjb_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "liboracle.so")
_lock = threading.Lock()
_lib = None

STATUS_OK, STATUS_PERFECT, STATUS_NOGAIN = 0, 1, 2


class OrcChoice(C.Structure):
    _fields_ = [("feature", C.c_int64), ("split", C.c_int32), ("polarity", C.c_int32),
                ("threshold", C.c_int32), ("pad", C.c_int32), ("err", C.c_double),
                ("second_err", C.c_double)]


class OrcStump(C.Structure):
    _fields_ = [("feature", C.c_int64), ("threshold", C.c_int32), ("polarity", C.c_int32),
                ("split", C.c_int32), ("pad", C.c_int32), ("err", C.c_double),
                ("beta", C.c_double), ("alpha", C.c_double), ("second_err", C.c_double)]


def build(force: bool = False) -> str:
    """Compile the oracle (gcc, OpenMP) if it is missing or older than its source."""
    with _lock:
        if (not force and os.path.exists(_LIB_PATH)
                and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
            return _LIB_PATH
        os.makedirs(_OUT_DIR, exist_ok=True)
        tmp = _LIB_PATH + f".{os.getpid()}.tmp"
        cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB_PATH)
        return _LIB_PATH


def _load():
    global _lib
    if _lib is None:
        build()
        lib = C.CDLL(_LIB_PATH)
        P = C.c_void_p
        i64, i32 = C.c_int64, C.c_int32
        lib.orc_num_threads.restype = C.c_int
        lib.orc_set_num_threads.argtypes = [C.c_int]
        lib.orc_haar_enumerate.argtypes = [C.c_int, C.c_int, P, P]
        lib.orc_haar_enumerate.restype = i64
        lib.orc_integral.argtypes = [P, i64, C.c_int, C.c_int, P]
        lib.orc_feature_values_direct.argtypes = [P, i64, C.c_int, C.c_int, P, i64, P]
        lib.orc_feature_values_integral.argtypes = [P, i64, C.c_int, C.c_int, P, i64, P]
        lib.orc_sort_rows.argtypes = [P, i64, i64, P]
        lib.orc_feature_best_sorted.argtypes = [P, P, i64, i64, P, P, P, P, P, P, P]
        lib.orc_feature_best_brute.argtypes = [P, i64, i64, P, P, P, P, P, P, P]
        lib.orc_select.argtypes = [P, P, P, P, P, i64, P]
        lib.orc_initial_weights.argtypes = [P, i64, P]
        lib.orc_normalize.argtypes = [P, i64]
        lib.orc_stump_error.argtypes = [P, i64, P, P, i32, i32]
        lib.orc_stump_error.restype = C.c_double
        lib.orc_update.argtypes = [P, i64, P, P, i32, i32, C.c_double]
        lib.orc_round.argtypes = [P, P, i64, i64, P, P, P]
        lib.orc_round.restype = C.c_int
        lib.orc_train.argtypes = [P, P, i64, i64, P, P, i32, P, P]
        lib.orc_train.restype = C.c_int
        lib.orc_strong_classify.argtypes = [P, i64, P, i32, P]
        _lib = lib
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


def num_threads() -> int:
    return int(_load().orc_num_threads())


def set_num_threads(k: int) -> None:
    """Threads the oracle's parallel loops use from now on (k > 0)."""
    _load().orc_set_num_threads(int(k))


def haar_enumerate(W: int, H: int):
    """(desc int32 [F, 5] = (type, x, y, w, h), per_type int64 [5])."""
    lib = _load()
    per = np.zeros(5, np.int64)
    nf = lib.orc_haar_enumerate(W, H, None, _p(per))
    desc = np.zeros((nf, 5), np.int32)
    lib.orc_haar_enumerate(W, H, _p(desc), _p(per))
    return desc, per


def integral(px: np.ndarray) -> np.ndarray:
    """int32 [N, H+1, W+1] integral images with a zero first row and column."""
    px = np.ascontiguousarray(px, np.uint8)
    n, H, W = px.shape
    out = np.zeros((n, H + 1, W + 1), np.int32)
    _load().orc_integral(_p(px), n, H, W, _p(out))
    return out


def feature_values_direct(px: np.ndarray, desc: np.ndarray) -> np.ndarray:
    px = np.ascontiguousarray(px, np.uint8)
    desc = np.ascontiguousarray(desc, np.int32)
    n, H, W = px.shape
    out = np.zeros((desc.shape[0], n), np.int32)
    _load().orc_feature_values_direct(_p(px), n, H, W, _p(desc), desc.shape[0], _p(out))
    return out


def feature_values(px: np.ndarray, desc: np.ndarray, ii: np.ndarray | None = None) -> np.ndarray:
    """int32 [F, N] feature values through the oracle's own integral images."""
    px = np.ascontiguousarray(px, np.uint8)
    desc = np.ascontiguousarray(desc, np.int32)
    n, H, W = px.shape
    if ii is None:
        ii = integral(px)
    out = np.zeros((desc.shape[0], n), np.int32)
    _load().orc_feature_values_integral(_p(ii), n, H, W, _p(desc), desc.shape[0], _p(out))
    return out


def sort_rows(vals: np.ndarray) -> np.ndarray:
    """int32 [F, N]: stable ascending order of each row (ties by sample index)."""
    vals = np.ascontiguousarray(vals, np.int32)
    nf, n = vals.shape
    order = np.zeros((nf, n), np.int32)
    _load().orc_sort_rows(_p(vals), nf, n, _p(order))
    return order


def _best(fn, *args, nf):
    err = np.zeros(nf, np.float64)
    err2 = np.zeros(nf, np.float64)
    split = np.zeros(nf, np.int32)
    pol = np.zeros(nf, np.int32)
    theta = np.zeros(nf, np.int32)
    fn(*args, _p(err), _p(split), _p(pol), _p(theta), _p(err2))
    return dict(err=err, split=split, polarity=pol, threshold=theta, err2=err2)


def feature_best_sorted(vals, order, y, w):
    """Tier (b): per-feature best (err, split, polarity, threshold, err2)."""
    vals = np.ascontiguousarray(vals, np.int32)
    order = np.ascontiguousarray(order, np.int32)
    y = np.ascontiguousarray(y, np.uint8)
    w = np.ascontiguousarray(w, np.float64)
    nf, n = vals.shape
    return _best(_load().orc_feature_best_sorted, _p(vals), _p(order), nf, n, _p(y), _p(w), nf=nf)


def feature_best_brute(vals, y, w):
    """Tier (a): per-feature best by trying every threshold."""
    vals = np.ascontiguousarray(vals, np.int32)
    y = np.ascontiguousarray(y, np.uint8)
    w = np.ascontiguousarray(w, np.float64)
    nf, n = vals.shape
    return _best(_load().orc_feature_best_brute, _p(vals), nf, n, _p(y), _p(w), nf=nf)


def select(best: dict) -> dict:
    """Global best (err, feature, split, polarity) with its runner-up error."""
    nf = best["err"].shape[0]
    c = OrcChoice()
    _load().orc_select(_p(best["err"]), _p(best["split"]), _p(best["polarity"]),
                       _p(best["threshold"]), _p(best["err2"]), nf, C.byref(c))
    return dict(feature=int(c.feature), split=int(c.split), polarity=int(c.polarity),
                threshold=int(c.threshold), err=float(c.err), second_err=float(c.second_err))


def initial_weights(y) -> np.ndarray:
    y = np.ascontiguousarray(y, np.uint8)
    w = np.zeros(y.shape[0], np.float64)
    _load().orc_initial_weights(_p(y), y.shape[0], _p(w))
    return w


def normalize(w) -> np.ndarray:
    w = np.array(w, np.float64, copy=True)
    _load().orc_normalize(_p(w), w.shape[0])
    return w


def stump_error(val, y, w, threshold: int, polarity: int) -> float:
    val = np.ascontiguousarray(val, np.int32)
    y = np.ascontiguousarray(y, np.uint8)
    w = np.ascontiguousarray(w, np.float64)
    return float(_load().orc_stump_error(_p(val), val.shape[0], _p(y), _p(w), threshold, polarity))


def update(val, y, w, threshold: int, polarity: int, beta: float) -> np.ndarray:
    val = np.ascontiguousarray(val, np.int32)
    y = np.ascontiguousarray(y, np.uint8)
    w = np.array(w, np.float64, copy=True)
    _load().orc_update(_p(val), val.shape[0], _p(y), _p(w), threshold, polarity, beta)
    return w


def _stump_dict(s: OrcStump) -> dict:
    return dict(feature=int(s.feature), threshold=int(s.threshold), polarity=int(s.polarity),
                split=int(s.split), err=float(s.err), beta=float(s.beta), alpha=float(s.alpha),
                second_err=float(s.second_err))


def round_step(vals, order, y, w):
    """One round (normalise, search, update) on prepared data.

    Returns (status, stump dict, new weights).  ``w`` is not modified."""
    vals = np.ascontiguousarray(vals, np.int32)
    order = np.ascontiguousarray(order, np.int32)
    y = np.ascontiguousarray(y, np.uint8)
    w = np.array(w, np.float64, copy=True)
    nf, n = vals.shape
    s = OrcStump()
    st = _load().orc_round(_p(vals), _p(order), nf, n, _p(y), _p(w), C.byref(s))
    return int(st), _stump_dict(s), w


def train(vals, order, y, w, T: int):
    """T rounds; returns (status, list of stump dicts, final weights)."""
    vals = np.ascontiguousarray(vals, np.int32)
    order = np.ascontiguousarray(order, np.int32)
    y = np.ascontiguousarray(y, np.uint8)
    w = np.array(w, np.float64, copy=True)
    nf, n = vals.shape
    out = (OrcStump * max(T, 1))()
    done = C.c_int32(0)
    st = _load().orc_train(_p(vals), _p(order), nf, n, _p(y), _p(w), T, out, C.byref(done))
    return int(st), [_stump_dict(out[t]) for t in range(done.value)], w


def strong_classify(fval, stumps) -> np.ndarray:
    """C(x) for each sample; fval is [T, N], row t = stump t's feature values."""
    fval = np.ascontiguousarray(fval, np.int32)
    T, n = fval.shape
    arr = (OrcStump * max(T, 1))()
    for t, s in enumerate(stumps):
        arr[t].threshold = s["threshold"]
        arr[t].polarity = s["polarity"]
        arr[t].alpha = s["alpha"]
    out = np.zeros(n, np.uint8)
    _load().orc_strong_classify(_p(fval), n, arr, T, _p(out))
    return out


class Prepared:
    """Feature values and value orders of one training set, computed once."""

    def __init__(self, px, y, desc=None):
        px = np.ascontiguousarray(px, np.uint8)
        n, H, W = px.shape
        self.px, self.y = px, np.ascontiguousarray(y, np.uint8)
        self.desc = haar_enumerate(W, H)[0] if desc is None else np.ascontiguousarray(desc, np.int32)
        self.ii = integral(px)
        self.vals = feature_values(px, self.desc, self.ii)
        self.order = sort_rows(self.vals)
