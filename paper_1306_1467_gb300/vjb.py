"""Thin ctypes binding of the C ABI in ``include/vjb.h``.

Only argument marshalling happens here: every step of training runs in the
library's CUDA kernels.  There is no CPU fallback -- if the library has not
been built, or no GPU is visible, calls raise.

Host inputs are numpy arrays; device inputs may be torch CUDA tensors (their
``data_ptr()`` is passed through), so PyTorch only provides device memory and
streams.
"""

from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

OK, DONE_PERFECT, DONE_NOGAIN = 0, 1, 2
EINVAL, ESTATE, ENOMEM, ECUDA, EDEVICE, EFULL = -1, -2, -3, -4, -5, -6
MAX_SAMPLES = 32766
REQ_QUEUED, REQ_PREPARING, REQ_TRAINING, REQ_DONE, REQ_FAILED = 0, 1, 2, 3, 4
BATCH_PARTITIONED, BATCH_INTERLEAVED = -1, -2
HAAR_TYPES = ("3H", "3V", "2H", "2V", "4")


class VJBError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"vjb error {code}: {msg}")
        self.code = code


class Feature(C.Structure):
    _fields_ = [("type", C.c_uint8), ("x", C.c_uint8), ("y", C.c_uint8), ("w", C.c_uint8),
                ("h", C.c_uint8)]


class Stump(C.Structure):
    _fields_ = [("feature", C.c_int32), ("threshold", C.c_int32), ("polarity", C.c_int32),
                ("split", C.c_int32), ("error", C.c_double), ("beta", C.c_double),
                ("alpha", C.c_double)]

    def as_dict(self) -> dict:
        return dict(feature=int(self.feature), threshold=int(self.threshold),
                    polarity=int(self.polarity), split=int(self.split), error=float(self.error),
                    beta=float(self.beta), alpha=float(self.alpha))


class Info(C.Structure):
    _fields_ = [("n", C.c_int32), ("h", C.c_int32), ("w", C.c_int32), ("npad", C.c_int32),
                ("features", C.c_int64), ("rounds_done", C.c_int32), ("status", C.c_int32),
                ("t_pos", C.c_double), ("t_neg", C.c_double), ("weight_sum", C.c_double),
                ("screen_min", C.c_float), ("candidates", C.c_int32),
                ("device_flags", C.c_int32), ("kernel_warps", C.c_int32),
                ("kernel_stages", C.c_int32), ("kernel_ctas", C.c_int32),
                ("kernel_unroll", C.c_int32), ("kernel_box_lines", C.c_int32), ("pad0", C.c_int32),
                ("search_bytes", C.c_double),
                ("launches", C.c_int64), ("dual_weights", C.c_int32), ("pad", C.c_int32)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_ if not k.startswith("pad")}


class RoundDiag(C.Structure):
    _fields_ = [("search_error", C.c_double), ("screen_error", C.c_float), ("screen_min", C.c_float),
                ("candidates", C.c_int32), ("forced", C.c_int32)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


class SearchShapeC(C.Structure):
    _fields_ = [("warps", C.c_int32), ("stages", C.c_int32), ("ctas_per_sm", C.c_int32),
                ("unroll", C.c_int32), ("box_lines", C.c_int32)]


class Timing(C.Structure):
    _fields_ = [("rounds", C.c_int32), ("pad", C.c_int32), ("search_ms_total", C.c_double),
                ("search_ms_min", C.c_double), ("search_ms_max", C.c_double),
                ("round_ms_total", C.c_double)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_ if k != "pad"}


class BatchInfo(C.Structure):
    _fields_ = [("jobs", C.c_int32), ("warps", C.c_int32), ("stages", C.c_int32), ("unroll", C.c_int32),
                ("rows_per_warp", C.c_int32), ("box_lines", C.c_int32), ("budget_bytes", C.c_int64),
                ("free_bytes", C.c_int64), ("largest_free_bytes", C.c_int64),
                ("search_bytes", C.c_double), ("launches", C.c_int64)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_ if k != "pad"}


class BatchTrial(C.Structure):
    _fields_ = [("warps", C.c_int32), ("stages", C.c_int32), ("unroll", C.c_int32),
                ("rows_per_warp", C.c_int32), ("box_lines", C.c_int32), ("ms_per_round", C.c_float)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


class RequestInfo(C.Structure):
    _fields_ = [("request_id", C.c_int64), ("state", C.c_int32), ("status", C.c_int32),
                ("rounds_done", C.c_int32), ("rounds_target", C.c_int32), ("n", C.c_int32),
                ("h", C.c_int32), ("w", C.c_int32), ("rounds_timed", C.c_int32), ("pad", C.c_int32),
                ("table_bytes", C.c_int64), ("t_submit_ms", C.c_double), ("t_admit_ms", C.c_double),
                ("t_ready_ms", C.c_double), ("t_done_ms", C.c_double), ("round_ms_sum", C.c_double)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_ if k != "pad"}


class ServerSummary(C.Structure):
    _fields_ = [("queued", C.c_int32), ("preparing", C.c_int32), ("training", C.c_int32),
                ("done", C.c_int32), ("failed", C.c_int32), ("pad", C.c_int32), ("rounds", C.c_int64),
                ("job_rounds", C.c_int64), ("budget_bytes", C.c_int64), ("free_bytes", C.c_int64),
                ("round_ms_total", C.c_double), ("clock_ms", C.c_double)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_ if k != "pad"}


# Every exported symbol with its (restype, argtypes).
_P, _I32, _I64 = C.c_void_p, C.c_int32, C.c_int64
SIGNATURES = {
    "vjb_create": (C.c_int, [C.POINTER(C.c_void_p), C.c_int, _P]),
    "vjb_destroy": (None, [_P]),
    "vjb_last_error": (C.c_char_p, []),
    "vjb_load_windows": (C.c_int, [_P, _P, _P, _I32, _I32, _I32]),
    "vjb_load_windows_device": (C.c_int, [_P, _P, _P, _I32, _I32, _I32]),
    "vjb_build_integral": (C.c_int, [_P]),
    "vjb_enumerate_haar": (C.c_int, [_P, C.POINTER(C.c_int64), _P]),
    "vjb_train_round": (C.c_int, [_P, _P]),
    "vjb_train_strong": (C.c_int, [_P, _I32, _P, C.POINTER(C.c_int32)]),
    "vjb_get_weights": (C.c_int, [_P, _P]),
    "vjb_set_weights": (C.c_int, [_P, _P]),
    "vjb_force_stump": (C.c_int, [_P, _I32, _I32, _I32, _P]),
    "vjb_get_info": (C.c_int, [_P, _P]),
    "vjb_get_integral": (C.c_int, [_P, _P]),
    "vjb_classify": (C.c_int, [_P, _P, _I32, _P, _I32, _P, _P]),
    "vjb_feature_values": (C.c_int, [_P, _I64, _I64, _P]),
    "vjb_sorted_rows": (C.c_int, [_P, _I64, _I64, _P]),
    "vjb_screen_errors": (C.c_int, [_P, _P]),
    "vjb_set_search_shape": (C.c_int, [_P, _P]),
    "vjb_get_search_shape": (C.c_int, [_P, _P]),
    "vjb_get_round_diag": (C.c_int, [_P, _I32, _I32, _P]),
    "vjb_set_timing": (C.c_int, [_P, _I32]),
    "vjb_get_timing": (C.c_int, [_P, _P]),
    "vjb_batch_create": (C.c_int, [C.POINTER(C.c_void_p), C.c_int, _P, _I64]),
    "vjb_batch_destroy": (None, [_P]),
    "vjb_batch_table_bytes": (C.c_int, [_I32, _I32, _I32, C.POINTER(C.c_int64)]),
    "vjb_batch_add_job": (C.c_int, [_P, _P, _P, _I32, _I32, _I32, _I32, C.POINTER(C.c_int32)]),
    "vjb_batch_remove_job": (C.c_int, [_P, _I32]),
    "vjb_batch_train": (C.c_int, [_P, _I32, C.POINTER(C.c_int32)]),
    "vjb_batch_autotune": (C.c_int, [_P, _I32, C.POINTER(C.c_int32), _P, _I32, C.POINTER(C.c_int32)]),
    "vjb_batch_job_state": (C.c_int, [_P, _I32, C.POINTER(C.c_int32), C.POINTER(C.c_int32)]),
    "vjb_batch_get_stumps": (C.c_int, [_P, _I32, _I32, _I32, _P]),
    "vjb_batch_get_weights": (C.c_int, [_P, _I32, _P]),
    "vjb_batch_set_search_shape": (C.c_int, [_P, _P, _I32]),
    "vjb_batch_get_info": (C.c_int, [_P, _P]),
    "vjb_batch_set_timing": (C.c_int, [_P, _I32]),
    "vjb_batch_get_timing": (C.c_int, [_P, _P]),
    "vjb_server_create": (C.c_int, [C.POINTER(C.c_void_p), C.c_int, _I64, _I32]),
    "vjb_server_destroy": (None, [_P]),
    "vjb_server_submit": (C.c_int, [_P, _P, _P, _I32, _I32, _I32, _I32, C.POINTER(C.c_int64)]),
    "vjb_server_step": (C.c_int, [_P, _I32, C.POINTER(C.c_int32)]),
    "vjb_server_request": (C.c_int, [_P, _I64, _P]),
    "vjb_server_result": (C.c_int, [_P, _I64, _P, _I32, _P]),
    "vjb_server_release": (C.c_int, [_P, _I64]),
    "vjb_server_stats": (C.c_int, [_P, _P]),
    "vjb_server_round_times": (C.c_int, [_P, _I64, _I32, _P, _P]),
    "vjb_screen_noalloc": (C.c_int, [_P, _P, _I32, _I32, _I64, C.c_double, C.c_double, _I32,
                                     _P, _P, _P, _P]),
}

_lib = None


def library_path() -> str:
    return _build.LIB_PATH


def load_library(build_if_missing: bool = True):
    """Load libvjb.so (building it with nvcc if it is missing)."""
    global _lib
    if _lib is None:
        path = library_path()
        if not os.path.exists(path):
            if not build_if_missing:
                raise RuntimeError(f"CUDA library not built: {path}")
            _build.build()
        lib = C.CDLL(path)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


def _is_torch_cuda(x) -> bool:
    return hasattr(x, "is_cuda") and bool(x.is_cuda)


class Trainer:
    """One training context (``vjb_ctx``) on one GPU.

    Method names follow the C ABI: load_windows, build_integral,
    enumerate_haar, train_round, train_strong, ...
    """

    def __init__(self, device: int = 0, stream=None):
        self._lib = load_library()
        h = C.c_void_p()
        s = None if stream is None else C.c_void_p(int(stream))
        self._check(self._lib.vjb_create(C.byref(h), int(device), s))
        self._h = h
        self.n = self.h = self.w = 0
        self.features = None

    # -- plumbing ---------------------------------------------------------
    def _check(self, rc: int) -> int:
        if rc < 0:
            raise VJBError(rc, self._lib.vjb_last_error().decode())
        return rc

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            self._lib.vjb_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # -- steps ------------------------------------------------------------------
    def load_windows(self, pixels, labels):
        """pixels [N, H, W] uint8 and labels [N] in {0, 1}: numpy (host) or torch CUDA tensors."""
        if _is_torch_cuda(pixels):
            n, h, w = (int(d) for d in pixels.shape)
            assert pixels.is_contiguous() and labels.is_contiguous()
            self._check(self._lib.vjb_load_windows_device(
                self._h, C.c_void_p(pixels.data_ptr()), C.c_void_p(labels.data_ptr()), n, h, w))
        else:
            px = np.ascontiguousarray(pixels, np.uint8)
            y = np.ascontiguousarray(labels, np.uint8)
            n, h, w = px.shape
            if y.shape != (n,):
                raise ValueError("labels must have shape [N]")
            self._check(self._lib.vjb_load_windows(self._h, _ptr(px), _ptr(y), n, h, w))
        self.n, self.h, self.w = n, h, w
        self.features = None

    def build_integral(self):
        self._check(self._lib.vjb_build_integral(self._h))

    def enumerate_haar(self) -> np.ndarray:
        """Feature list [F, 5] int32 rows (type, x, y, w, h) in canonical order."""
        cnt = C.c_int64(0)
        self._check(self._lib.vjb_enumerate_haar(self._h, C.byref(cnt), None))
        arr = (Feature * cnt.value)()
        self._check(self._lib.vjb_enumerate_haar(self._h, C.byref(cnt), arr))
        raw = np.frombuffer(arr, dtype=np.uint8).reshape(cnt.value, 5)
        self.features = raw.astype(np.int32)
        return self.features

    def feature_count(self) -> int:
        """enumerate_haar without copying the feature list out; returns F."""
        cnt = C.c_int64(0)
        self._check(self._lib.vjb_enumerate_haar(self._h, C.byref(cnt), None))
        return int(cnt.value)

    def prepare(self, pixels, labels) -> np.ndarray:
        """load_windows + build_integral + enumerate_haar."""
        self.load_windows(pixels, labels)
        self.build_integral()
        return self.enumerate_haar()

    def train_round(self):
        """(status, stump dict) of one round."""
        s = Stump()
        st = self._check(self._lib.vjb_train_round(self._h, C.byref(s)))
        return st, s.as_dict()

    def train_strong(self, T: int):
        """(status, list of kept stump dicts) of T rounds replayed as a CUDA graph."""
        arr = (Stump * max(int(T), 1))()
        done = C.c_int32(0)
        st = self._check(self._lib.vjb_train_strong(self._h, int(T), arr, C.byref(done)))
        return st, [arr[t].as_dict() for t in range(done.value)]

    def force_stump(self, feature: int, threshold: int, polarity: int):
        s = Stump()
        st = self._check(self._lib.vjb_force_stump(self._h, int(feature), int(threshold),
                                                   int(polarity), C.byref(s)))
        return st, s.as_dict()

    # -- state --------------------------------------------------------------------
    def get_weights(self) -> np.ndarray:
        out = np.zeros(self.n, np.float32)
        self._check(self._lib.vjb_get_weights(self._h, _ptr(out)))
        return out

    def set_weights(self, w):
        w = np.ascontiguousarray(w, np.float32)
        if w.shape != (self.n,):
            raise ValueError("weights must have shape [N]")
        self._check(self._lib.vjb_set_weights(self._h, _ptr(w)))

    def info(self) -> dict:
        i = Info()
        self._check(self._lib.vjb_get_info(self._h, C.byref(i)))
        return i.as_dict()

    def set_search_shape(self, warps: int = 0, stages: int = 0, ctas_per_sm: int = 0, unroll: int = 0,
                         box_lines: int = 0):
        """Launch shape of the search kernel; 0 keeps a field's current value."""
        sh = SearchShapeC(int(warps), int(stages), int(ctas_per_sm), int(unroll), int(box_lines))
        self._check(self._lib.vjb_set_search_shape(self._h, C.byref(sh)))

    def search_shape(self) -> dict:
        sh = SearchShapeC()
        self._check(self._lib.vjb_get_search_shape(self._h, C.byref(sh)))
        return {k: getattr(sh, k) for k, _ in sh._fields_}

    def round_diag(self, first: int = 0, count: int | None = None) -> list:
        """Per-round search diagnostics of kept rounds [first, first + count)."""
        if count is None:
            count = self.info()["rounds_done"] - first
        arr = (RoundDiag * max(int(count), 1))()
        self._check(self._lib.vjb_get_round_diag(self._h, int(first), int(count), arr))
        return [arr[k].as_dict() for k in range(int(count))]

    def set_timing(self, enable: bool = True):
        """Enable (and reset) CUDA-event timing of every round's search kernel."""
        self._check(self._lib.vjb_set_timing(self._h, 1 if enable else 0))

    def timing(self) -> dict:
        t = Timing()
        self._check(self._lib.vjb_get_timing(self._h, C.byref(t)))
        return t.as_dict()

    # -- the strong classifier ----------------------------------------------------
    def classify(self, pixels, stumps):
        """C(x) and the FP64 scores of windows pixels [N, H, W] (host) under ``stumps``
        (dicts as returned by train_round / train_strong)."""
        px = np.ascontiguousarray(pixels, np.uint8)
        n = px.shape[0]
        arr = (Stump * max(len(stumps), 1))()
        for t, s in enumerate(stumps):
            for k, _ in Stump._fields_:
                setattr(arr[t], k, s[k])
        lab = np.zeros(n, np.uint8)
        sc = np.zeros(n, np.float64)
        self._check(self._lib.vjb_classify(self._h, _ptr(px), n, arr, len(stumps), _ptr(lab), _ptr(sc)))
        return lab, sc

    # -- inspection -------------------------------------------------------------------
    def get_integral(self) -> np.ndarray:
        out = np.zeros((self.n, self.h + 1, self.w + 1), np.int32)
        self._check(self._lib.vjb_get_integral(self._h, _ptr(out)))
        return out

    def feature_values(self, f0: int, nf: int) -> np.ndarray:
        out = np.zeros((nf, self.n), np.int32)
        self._check(self._lib.vjb_feature_values(self._h, int(f0), int(nf), _ptr(out)))
        return out

    def sorted_rows(self, f0: int, nf: int) -> np.ndarray:
        out = np.zeros((nf, self.n), np.uint16)
        self._check(self._lib.vjb_sorted_rows(self._h, int(f0), int(nf), _ptr(out)))
        return out

    def screen_errors(self) -> np.ndarray:
        nf = self.info()["features"]
        out = np.zeros(nf, np.float32)
        self._check(self._lib.vjb_screen_errors(self._h, _ptr(out)))
        return out


class Batch:
    """Many training jobs trained together (``vjb_batch``): one launch of each
    round kernel covers every job, and each job's stumps and weights are the
    ones it would get alone in a :class:`Trainer`.

    ``table_budget_bytes`` is the HBM arena for the jobs' sorted tables; a job
    whose table does not fit what is free raises :class:`VJBError` with code
    ``EFULL``.
    """

    def __init__(self, table_budget_bytes: int, device: int = 0, stream=None):
        self._lib = load_library()
        h = C.c_void_p()
        s = None if stream is None else C.c_void_p(int(stream))
        self._check(self._lib.vjb_batch_create(C.byref(h), int(device), s, int(table_budget_bytes)))
        self._h = h
        self.jobs = {}  # id -> n

    def _check(self, rc: int) -> int:
        if rc < 0:
            raise VJBError(rc, self._lib.vjb_last_error().decode())
        return rc

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            self._lib.vjb_batch_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    @staticmethod
    def table_bytes(n: int, h: int, w: int) -> int:
        lib = load_library()
        out = C.c_int64()
        rc = lib.vjb_batch_table_bytes(int(n), int(h), int(w), C.byref(out))
        if rc < 0:
            raise VJBError(rc, lib.vjb_last_error().decode())
        return int(out.value)

    def add_job(self, pixels, labels, rounds: int) -> int:
        """Add a job (host pixels [N, H, W] uint8, labels [N]); returns its id."""
        px = np.ascontiguousarray(pixels, np.uint8)
        y = np.ascontiguousarray(labels, np.uint8)
        n, h, w = px.shape
        if y.shape != (n,):
            raise ValueError("labels must have shape [N]")
        jid = C.c_int32()
        self._check(self._lib.vjb_batch_add_job(self._h, _ptr(px), _ptr(y), n, h, w, int(rounds),
                                                C.byref(jid)))
        self.jobs[int(jid.value)] = int(n)
        return int(jid.value)

    def remove_job(self, job_id: int):
        self._check(self._lib.vjb_batch_remove_job(self._h, int(job_id)))
        self.jobs.pop(int(job_id), None)

    def train(self, max_rounds: int = 1 << 30) -> int:
        """Run batched rounds until every job is done or ``max_rounds`` ran; returns rounds run."""
        r = C.c_int32()
        self._check(self._lib.vjb_batch_train(self._h, int(max_rounds), C.byref(r)))
        return int(r.value)

    def autotune(self, trial_rounds: int = 2) -> int:
        """Time real rounds with each candidate launch shape and keep the fastest; returns rounds
        run.  The timed shapes are left in ``self.trials``."""
        r, nt = C.c_int32(), C.c_int32()
        arr = (BatchTrial * 32)()
        self._check(self._lib.vjb_batch_autotune(self._h, int(trial_rounds), C.byref(r), arr, 32, C.byref(nt)))
        self.trials = [arr[k].as_dict() for k in range(nt.value)]
        return int(r.value)

    def job_state(self, job_id: int):
        """(kept stumps, status) of a job."""
        d, st = C.c_int32(), C.c_int32()
        self._check(self._lib.vjb_batch_job_state(self._h, int(job_id), C.byref(d), C.byref(st)))
        return int(d.value), int(st.value)

    def stumps(self, job_id: int) -> list:
        done, _ = self.job_state(job_id)
        arr = (Stump * max(done, 1))()
        self._check(self._lib.vjb_batch_get_stumps(self._h, int(job_id), 0, done, arr))
        return [arr[t].as_dict() for t in range(done)]

    def get_weights(self, job_id: int) -> np.ndarray:
        out = np.zeros(self.jobs[int(job_id)], np.float32)
        self._check(self._lib.vjb_batch_get_weights(self._h, int(job_id), _ptr(out)))
        return out

    def set_search_shape(self, warps: int = 0, stages: int = 0, unroll: int = 0, rows_per_warp: int = 0,
                         box_lines: int = 0):
        """Batched search launch shape; rows_per_warp > 0 selects the work queue with that many
        features per warp and item, BATCH_INTERLEAVED / BATCH_PARTITIONED the other schedules, 0 keeps a field."""
        sh = SearchShapeC(int(warps), int(stages), 0, int(unroll), int(box_lines))
        self._check(self._lib.vjb_batch_set_search_shape(self._h, C.byref(sh), int(rows_per_warp)))

    def info(self) -> dict:
        i = BatchInfo()
        self._check(self._lib.vjb_batch_get_info(self._h, C.byref(i)))
        return i.as_dict()

    def set_timing(self, enable: bool = True):
        """Enable (and reset) CUDA-event timing of every batched round and its search kernel."""
        self._check(self._lib.vjb_batch_set_timing(self._h, 1 if enable else 0))

    def timing(self) -> dict:
        t = Timing()
        self._check(self._lib.vjb_batch_get_timing(self._h, C.byref(t)))
        return t.as_dict()


class Server:
    """Continuous batching of training requests on one GPU (``vjb_server``).

    ``submit`` queues a request; ``step`` admits what fits the table budget,
    lets the library's worker thread prepare admitted requests while the batch
    trains, and runs batched rounds.  Every request's stumps and weights equal
    those of a plain run of the same job.
    """

    def __init__(self, table_budget_bytes: int, max_jobs: int = 64, device: int = 0):
        self._lib = load_library()
        h = C.c_void_p()
        self._check(self._lib.vjb_server_create(C.byref(h), int(device), int(table_budget_bytes), int(max_jobs)))
        self._h = h
        self._n = {}

    def _check(self, rc: int) -> int:
        if rc < 0:
            raise VJBError(rc, self._lib.vjb_last_error().decode())
        return rc

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            self._lib.vjb_server_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def submit(self, pixels, labels, rounds: int) -> int:
        px = np.ascontiguousarray(pixels, np.uint8)
        y = np.ascontiguousarray(labels, np.uint8)
        n, h, w = px.shape
        if y.shape != (n,):
            raise ValueError("labels must have shape [N]")
        rid = C.c_int64()
        self._check(self._lib.vjb_server_submit(self._h, _ptr(px), _ptr(y), n, h, w, int(rounds), C.byref(rid)))
        self._n[int(rid.value)] = (int(n), int(rounds))
        return int(rid.value)

    def step(self, max_rounds: int = 1) -> int:
        r = C.c_int32()
        self._check(self._lib.vjb_server_step(self._h, int(max_rounds), C.byref(r)))
        return int(r.value)

    def request(self, rid: int) -> dict:
        i = RequestInfo()
        self._check(self._lib.vjb_server_request(self._h, int(rid), C.byref(i)))
        return i.as_dict()

    def result(self, rid: int):
        """(status, stumps, weights) of a finished request."""
        n, rounds = self._n[int(rid)]
        arr = (Stump * max(rounds, 1))()
        w = np.zeros(n, np.float32)
        st = self._check(self._lib.vjb_server_result(self._h, int(rid), arr, rounds, _ptr(w)))
        done = self.request(rid)["rounds_done"]
        return st, [arr[t].as_dict() for t in range(done)], w

    def release(self, rid: int):
        self._check(self._lib.vjb_server_release(self._h, int(rid)))
        self._n.pop(int(rid), None)

    def stats(self) -> dict:
        s = ServerSummary()
        self._check(self._lib.vjb_server_stats(self._h, C.byref(s)))
        return s.as_dict()

    def round_times(self):
        """(durations in ms, jobs in the round) of every batched round so far."""
        k = self.stats()["rounds"]
        ms = np.zeros(max(k, 1), np.float32)
        jobs = np.zeros(max(k, 1), np.int32)
        self._check(self._lib.vjb_server_round_times(self._h, 0, int(k), _ptr(ms), _ptr(jobs)))
        return ms[:k], jobs[:k]
