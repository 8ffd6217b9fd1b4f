"""ctypes binding of the C ABI in include/ace.h (argument marshalling only).

Every step of the hot path runs in the CUDA library; torch is used for device buffers and
streams.  If the library has not been built, the first call raises — there is no CPU path.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libace_gb300.so")

ACE_OK, ACE_ERR_ARG, ACE_ERR_OOM, ACE_ERR_OVERFLOW, ACE_ERR_TIMEOUT, ACE_ERR_CUDA, ACE_ERR_UNSUPPORTED = range(7)
ACE_STATUS_TIMEOUT = 2  # a bounded device wait gave up (ace_stats status bits)
ACE_F32, ACE_BF16 = 0, 1
ACE_PROJ_AUTO, ACE_PROJ_FP32, ACE_PROJ_BF16, ACE_PROJ_FP8, ACE_PROJ_FWHT = -1, 0, 1, 2, 3
ACE_W_BF16 = 1
ACE_W_COUNTER = 2
ACE_W_HADAMARD = 4
PRECISIONS = {"auto": ACE_PROJ_AUTO, "fp32": ACE_PROJ_FP32, "bf16": ACE_PROJ_BF16, "fp8": ACE_PROJ_FP8,
              "fwht": ACE_PROJ_FWHT}

# Every symbol include/ace.h declares (checked by the tests).
EXPORTS = [
    "ace_create", "ace_create_ex", "ace_create_with_projection", "ace_destroy", "ace_reset", "ace_set_precision",
    "ace_set_privacy", "ace_get_privacy",
    "ace_insert", "ace_score", "ace_insert_score", "ace_insert_score_host",
    "ace_insert_score_host_async", "ace_host_wait", "ace_delete", "ace_project", "ace_hash",
    "ace_batch_insert_score", "ace_server_create", "ace_server_submit", "ace_server_wait", "ace_server_drain", "ace_server_destroy", "ace_server_info", "ace_stats",
    "ace_get_counts", "ace_get_projection", "ace_get_shape", "ace_last_error", "ace_version",
    "ace_profile_enable", "ace_profile_phases", "ace_profile_read", "ace_insert_score_noalloc",
    "ace_tc_probe", "ace_tc_probe_fp8", "ace_wait_probe", "ace_exact_score", "ace_save_size", "ace_save", "ace_load", "ace_window_enable", "ace_set_graph",
    "ace_batch_tile",
]
NOALLOC_SCRATCH_BYTES = 32 * 1024 * 1024
PHASES = ("hash", "score", "flags", "other", "recheck", "insert")


class AceError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"ace error {code}: {msg}")
        self.code = code


class ace_stats_t(ctypes.Structure):
    _fields_ = [
        ("n_ins", ctypes.c_uint64), ("n_scored", ctypes.c_uint64),
        ("Q_lo", ctypes.c_uint64), ("Q_hi", ctypes.c_uint64),
        ("S1_lo", ctypes.c_uint64), ("S1_hi", ctypes.c_uint64),
        ("S2_lo", ctypes.c_uint64), ("S2_hi", ctypes.c_uint64),
        ("mu_ins", ctypes.c_double), ("mu", ctypes.c_double), ("sigma", ctypes.c_double),
        ("rechecks", ctypes.c_uint64), ("nonfinite_points", ctypes.c_uint64),
        ("status", ctypes.c_uint32), ("precision", ctypes.c_int32), ("deferred", ctypes.c_uint64),
        ("tc_products", ctypes.c_int32),
    ]


class ace_profile_t(ctypes.Structure):
    _fields_ = [("launches", ctypes.c_uint64 * 6), ("ms", ctypes.c_double * 6), ("timed", ctypes.c_uint64 * 6)]


_lib = None
_lock = threading.Lock()


def load_library(path: str = LIB_PATH):
    """Loads libace_gb300.so and declares the ABI (raises if it was not built)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(path):
            raise RuntimeError(f"CUDA library not built: {path} is missing (run __graft_entry__.build())")
        lib = ctypes.CDLL(path)
        P, i32, i64, u64, f64 = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_uint64, ctypes.c_double
        H = ctypes.c_void_p
        decl = {
            "ace_create": ([i32, i32, i32, u64, ctypes.POINTER(H)], i32),
            "ace_create_ex": ([i32, i32, i32, u64, ctypes.c_uint32, ctypes.POINTER(H)], i32),
            "ace_create_with_projection": ([i32, i32, i32, P, ctypes.POINTER(H)], i32),
            "ace_destroy": ([H], i32),
            "ace_reset": ([H, P], i32),
            "ace_set_precision": ([H, i32], i32),
            "ace_wait_probe": ([i32, ctypes.c_int64, ctypes.POINTER(ctypes.c_uint32), ctypes.POINTER(ctypes.c_int64)], i32),
            "ace_set_privacy": ([H, ctypes.c_float, ctypes.c_uint64], i32),
            "ace_get_privacy": ([H, ctypes.POINTER(ctypes.c_float), ctypes.POINTER(ctypes.c_uint64),
                                 ctypes.POINTER(ctypes.c_uint64)], i32),
            "ace_insert": ([H, P, i64, i32, P], i32),
            "ace_score": ([H, P, i64, i32, f64, P, P, P, P], i32),
            "ace_insert_score": ([H, P, i64, i32, f64, P, P, P, P], i32),
            "ace_insert_score_host": ([H, P, i64, i32, f64, P, P, P, P], i32),
            "ace_insert_score_host_async": ([H, P, i64, i32, f64, P, P, P, P], i32),
            "ace_host_wait": ([H], i32),
            "ace_delete": ([H, P, i64, i32, P], i32),
            "ace_project": ([H, P, i64, i32, P, P], i32),
            "ace_batch_insert_score": ([P, i32, P, P, i32, f64, P, P, P, P], i32),
            "ace_server_create": ([P, i32, ctypes.c_size_t, P], i32),
            "ace_server_submit": ([P, i32, i32, P, i64, i32, f64, P, P, P, P], i32),
            "ace_server_wait": ([P, ctypes.c_uint64, P], i32),
            "ace_server_drain": ([P], i32),
            "ace_server_destroy": ([P], i32),
            "ace_server_info": ([P, P, P], i32),
            "ace_insert_score_noalloc": ([H, P, i64, i32, f64, P, P, P, P], i32),
            "ace_hash": ([H, P, i64, i32, P, P], i32),
            "ace_stats": ([H, P, ctypes.POINTER(ace_stats_t)], i32),
            "ace_get_counts": ([H, P, P], i32),
            "ace_get_projection": ([H, P], i32),
            "ace_get_shape": ([H, P, P, P], i32),
            "ace_profile_enable": ([H, i32], i32),
            "ace_profile_phases": ([H, ctypes.c_uint32], i32),
            "ace_profile_read": ([H, ctypes.POINTER(ace_profile_t)], i32),
            "ace_tc_probe": ([P, P, i32, i32, P], i32),
            "ace_tc_probe_fp8": ([P, P, i32, i32, P], i32),
            "ace_exact_score": ([P, i64, P, i64, i32, i32, i32, P, P], i32),
            "ace_window_enable": ([H, i64], i32),
            "ace_set_graph": ([H, i32], i32),
            "ace_batch_tile": ([i32, i32, i32, i32, P, P], i32),
            "ace_save_size": ([H, ctypes.POINTER(ctypes.c_size_t)], i32),
            "ace_save": ([H, P, ctypes.c_size_t, P], i32),
            "ace_load": ([P, ctypes.c_size_t, ctypes.POINTER(H)], i32),
            "ace_last_error": ([], ctypes.c_char_p),
            "ace_version": ([], ctypes.c_char_p),
        }
        for name, (args, res) in decl.items():
            fn = getattr(lib, name)
            fn.argtypes = args
            fn.restype = res
        _lib = lib
        return lib


def _check(rc: int):
    if rc != ACE_OK:
        raise AceError(rc, _lib.ace_last_error().decode())


def _torch():
    import torch
    return torch


def _stream_ptr(stream):
    torch = _torch()
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _x_dtype(X):
    torch = _torch()
    if X.dtype == torch.float32:
        return ACE_F32
    if X.dtype in (torch.bfloat16, torch.int16, torch.uint16):
        return ACE_BF16
    raise TypeError("X must be float32 or bfloat16 (or int16/uint16 bfloat16 bit patterns)")


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else ctypes.c_void_p(0)


class Detector:
    """One ACE detector (W, L count arrays of 2^K uint32, running score statistics) on the
    current CUDA device."""

    def __init__(self, d: int, K: int, L: int, seed: int = 0, W: np.ndarray | None = None,
                 precision: str = "auto", w_bf16: bool = False, w_counter: bool = False, w_hadamard: bool = False):
        lib = load_library()
        self.d, self.K, self.L = int(d), int(K), int(L)
        h = ctypes.c_void_p()
        if W is None:
            flags = (ACE_W_BF16 if w_bf16 else 0) | (ACE_W_COUNTER if w_counter else 0) | \
                (ACE_W_HADAMARD if w_hadamard else 0)
            _check(lib.ace_create_ex(self.d, self.K, self.L, ctypes.c_uint64(int(seed) & (2**64 - 1)),
                                     flags, ctypes.byref(h)))
        else:
            Wc = np.ascontiguousarray(W, dtype=np.float32)
            assert Wc.shape == (self.d, self.K * self.L)
            _check(lib.ace_create_with_projection(self.d, self.K, self.L, Wc.ctypes.data_as(ctypes.c_void_p),
                                                  ctypes.byref(h)))
        self._h = h
        self.set_precision(precision)

    # -- lifecycle ---------------------------------------------------------------------
    def close(self):
        if self._h is not None and self._h.value:
            load_library().ace_destroy(self._h)
        self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def set_precision(self, precision):
        p = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
        _check(load_library().ace_set_precision(self._h, p))

    def set_privacy(self, sigma: float, noise_seed: int = 0):
        """§4.5 privacy noise before the sign (ace_set_privacy); sigma = 0 turns it off."""
        _check(load_library().ace_set_privacy(self._h, ctypes.c_float(sigma), ctypes.c_uint64(noise_seed & (2**64 - 1))))

    def privacy(self) -> dict:
        """{"sigma", "noise_seed", "next_index"} (ace_get_privacy)."""
        sg, sd, nx = ctypes.c_float(), ctypes.c_uint64(), ctypes.c_uint64()
        _check(load_library().ace_get_privacy(self._h, ctypes.byref(sg), ctypes.byref(sd), ctypes.byref(nx)))
        return {"sigma": sg.value, "noise_seed": sd.value, "next_index": nx.value}

    def reset(self, stream=None):
        _check(load_library().ace_reset(self._h, _stream_ptr(stream)))

    # -- hot path ------------------------------------------------------------------------
    def _xcheck(self, X):
        assert X.is_cuda and X.is_contiguous() and X.dim() == 2 and X.shape[1] == self.d, "X must be n x d on CUDA"

    def insert(self, X, stream=None):
        self._xcheck(X)
        _check(load_library().ace_insert(self._h, _ptr(X), X.shape[0], _x_dtype(X), _stream_ptr(stream)))

    def project(self, X, stream=None):
        """The active engine's binary32 projection estimates, n x KL (a measurement hook)."""
        self._xcheck(X)
        torch = _torch()
        out = torch.empty((X.shape[0], self.K * self.L), dtype=torch.float32, device=X.device)
        _check(load_library().ace_project(self._h, _ptr(X), X.shape[0], _x_dtype(X), _ptr(out), _stream_ptr(stream)))
        return out

    def delete(self, X, stream=None):
        """§3.4.1 deletion of the batch's points (all or nothing; synchronises the stream)."""
        self._xcheck(X)
        _check(load_library().ace_delete(self._h, _ptr(X), X.shape[0], _x_dtype(X), _stream_ptr(stream)))

    def _outs(self, n, scores, sums, flags, device):
        torch = _torch()

        def pick(v, dt):
            if v is True:
                return torch.empty(n, dtype=dt, device=device)
            return None if (v is None or v is False) else v

        return pick(scores, torch.float64), pick(sums, torch.int32), pick(flags, torch.uint8)

    def score(self, X, alpha: float = 1.0, scores=True, sums=True, flags=True, stream=None):
        """Returns (scores float64, sums int32 holding uint32 bits, flags uint8) tensors."""
        self._xcheck(X)
        sc, su, fl = self._outs(X.shape[0], scores, sums, flags, X.device)
        _check(load_library().ace_score(self._h, _ptr(X), X.shape[0], _x_dtype(X), float(alpha), _ptr(sc),
                                        _ptr(su), _ptr(fl), _stream_ptr(stream)))
        return sc, su, fl

    def insert_score(self, X, alpha: float = 1.0, scores=True, sums=True, flags=True, stream=None):
        self._xcheck(X)
        sc, su, fl = self._outs(X.shape[0], scores, sums, flags, X.device)
        _check(load_library().ace_insert_score(self._h, _ptr(X), X.shape[0], _x_dtype(X), float(alpha), _ptr(sc),
                                               _ptr(su), _ptr(fl), _stream_ptr(stream)))
        return sc, su, fl

    def insert_score_noalloc(self, X, alpha: float = 1.0, scores=True, sums=True, flags=True, stream=None):
        """ace_insert_score through the allocation-free entry point (static library scratch)."""
        self._xcheck(X)
        sc, su, fl = self._outs(X.shape[0], scores, sums, flags, X.device)
        _check(load_library().ace_insert_score_noalloc(self._h, _ptr(X), X.shape[0], _x_dtype(X), float(alpha),
                                                       _ptr(sc), _ptr(su), _ptr(fl), _stream_ptr(stream)))
        return sc, su, fl

    def insert_score_host(self, X: np.ndarray, alpha: float = 1.0, scores=None, sums=None, flags=None,
                          stream=None):
        """Host buffers in, host buffers out (copies are part of the call)."""
        n = X.shape[0]
        dt = ACE_F32 if X.dtype == np.float32 else ACE_BF16
        if X.dtype not in (np.float32, np.uint16):
            raise TypeError("X must be float32 or uint16 bfloat16 bits")

        def p(a):
            return ctypes.c_void_p(a.ctypes.data) if a is not None else ctypes.c_void_p(0)

        _check(load_library().ace_insert_score_host(self._h, ctypes.c_void_p(X.ctypes.data), n, dt, float(alpha),
                                                    p(scores), p(sums), p(flags), _stream_ptr(stream)))
        return scores, sums, flags

    def insert_score_host_async(self, X: np.ndarray, alpha: float = 1.0, scores=None, sums=None, flags=None,
                                stream=None):
        """Enqueues one host-buffer batch and returns; X must stay unchanged and the outputs
        are valid only after host_wait()."""
        n = X.shape[0]
        dt = ACE_F32 if X.dtype == np.float32 else ACE_BF16
        if X.dtype not in (np.float32, np.uint16):
            raise TypeError("X must be float32 or uint16 bfloat16 bits")

        def p(a):
            return ctypes.c_void_p(a.ctypes.data) if a is not None else ctypes.c_void_p(0)

        _check(load_library().ace_insert_score_host_async(self._h, ctypes.c_void_p(X.ctypes.data), n, dt,
                                                          float(alpha), p(scores), p(sums), p(flags),
                                                          _stream_ptr(stream)))
        return scores, sums, flags

    def host_wait(self):
        """Waits for every batch enqueued by insert_score_host_async."""
        _check(load_library().ace_host_wait(self._h))

    def hash(self, X, stream=None):
        """n x L bucket ids (int32 tensor holding uint32 values)."""
        self._xcheck(X)
        torch = _torch()
        ids = torch.empty((X.shape[0], self.L), dtype=torch.int32, device=X.device)
        _check(load_library().ace_hash(self._h, _ptr(X), X.shape[0], _x_dtype(X), _ptr(ids), _stream_ptr(stream)))
        return ids

    # -- introspection -----------------------------------------------------------------
    def stats(self, stream=None) -> dict:
        st = ace_stats_t()
        _check(load_library().ace_stats(self._h, _stream_ptr(stream), ctypes.byref(st)))
        return {
            "n_ins": st.n_ins, "n_scored": st.n_scored,
            "Q": st.Q_lo | (st.Q_hi << 64), "S1": st.S1_lo | (st.S1_hi << 64), "S2": st.S2_lo | (st.S2_hi << 64),
            "mu_ins": st.mu_ins, "mu": st.mu, "sigma": st.sigma, "rechecks": st.rechecks,
            "nonfinite_points": st.nonfinite_points, "status": st.status, "precision": st.precision,
            "deferred": st.deferred, "tc_products": st.tc_products,
        }

    def counts(self, stream=None) -> np.ndarray:
        out = np.empty((self.L, 1 << self.K), dtype=np.uint32)
        _check(load_library().ace_get_counts(self._h, ctypes.c_void_p(out.ctypes.data), _stream_ptr(stream)))
        return out

    def profile(self, enable: bool = True, phases=None):
        """Turns the per-phase timing hook on or off; `phases` (names from PHASES) limits the
        events to those phases (None: all)."""
        mask = 0 if phases is None else sum(1 << PHASES.index(p) for p in phases)
        _check(load_library().ace_profile_phases(self._h, mask))
        _check(load_library().ace_profile_enable(self._h, 1 if enable else 0))

    def profile_read(self) -> dict:
        """Per-phase kernel launches and summed CUDA-event milliseconds since the last read."""
        p = ace_profile_t()
        _check(load_library().ace_profile_read(self._h, ctypes.byref(p)))
        return {name: {"launches": int(p.launches[i]), "ms": float(p.ms[i]), "timed": int(p.timed[i])}
                for i, name in enumerate(PHASES)}

    def set_graph(self, enable: bool = True):
        """Replay a captured CUDA graph for repeated score / insert_score calls (ace_set_graph)."""
        _check(load_library().ace_set_graph(self._h, 1 if enable else 0))

    def window(self, points: int):
        """Sliding window over the last `points` inserted points (ace_window_enable; 0: off)."""
        _check(load_library().ace_window_enable(self._h, int(points)))

    def save(self, stream=None) -> bytes:
        """Checkpoint blob (ace_save): shape, W, counts and running statistics."""
        lib = load_library()
        nb = ctypes.c_size_t()
        _check(lib.ace_save_size(self._h, ctypes.byref(nb)))
        buf = ctypes.create_string_buffer(nb.value)
        _check(lib.ace_save(self._h, buf, nb.value, _stream_ptr(stream)))
        return buf.raw

    @classmethod
    def load(cls, blob: bytes, precision: str = "auto") -> "Detector":
        """A new detector on the current CUDA device from a checkpoint blob (ace_load)."""
        lib = load_library()
        h = ctypes.c_void_p()
        _check(lib.ace_load(blob, len(blob), ctypes.byref(h)))
        self = cls.__new__(cls)
        self._h = h
        d, K, L = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        _check(lib.ace_get_shape(h, ctypes.byref(d), ctypes.byref(K), ctypes.byref(L)))
        self.d, self.K, self.L = d.value, K.value, L.value
        self.set_precision(precision)
        return self

    def projection(self) -> np.ndarray:
        out = np.empty((self.d, self.K * self.L), dtype=np.float32)
        _check(load_library().ace_get_projection(self._h, ctypes.c_void_p(out.ctypes.data)))
        return out


def batch_insert_score(detectors, Xs, alpha: float = 1.0, stream=None):
    """ace_batch_insert_score: insert_score on many detectors in one set of launches.
    Xs are device tensors (one per detector, same dtype).  Returns lists of (scores, sums,
    flags) device tensors."""
    torch = _torch()
    cnt = len(detectors)
    if cnt != len(Xs) or cnt == 0:
        raise ValueError("one X per detector")
    for d, X in zip(detectors, Xs):
        d._xcheck(X)
    dt = _x_dtype(Xs[0])
    dev = Xs[0].device
    sc = [torch.empty(X.shape[0], dtype=torch.float64, device=dev) for X in Xs]
    su = [torch.empty(X.shape[0], dtype=torch.int32, device=dev) for X in Xs]
    fl = [torch.empty(X.shape[0], dtype=torch.uint8, device=dev) for X in Xs]
    V = ctypes.c_void_p * cnt
    hs = V(*[d._h for d in detectors])
    xs = V(*[X.data_ptr() for X in Xs])
    ns = (ctypes.c_int64 * cnt)(*[X.shape[0] for X in Xs])
    _check(load_library().ace_batch_insert_score(hs, cnt, xs, ns, dt, float(alpha), V(*[t.data_ptr() for t in sc]),
                                                 V(*[t.data_ptr() for t in su]), V(*[t.data_ptr() for t in fl]),
                                                 _stream_ptr(stream)))
    return sc, su, fl


def batch_tile(d: int, K: int, L: int, dtype: int = ACE_F32):
    """(points, columns) per block the batched engine's autotuner chose for this shape, or
    (0, 0) before any batch has met it."""
    p, c = ctypes.c_int(), ctypes.c_int()
    _check(load_library().ace_batch_tile(int(d), int(K), int(L), int(dtype), ctypes.byref(p), ctypes.byref(c)))
    return p.value, c.value


OP_INSERT, OP_SCORE, OP_INSERT_SCORE = 0, 1, 2


class Server:
    """Continuous batching of host-buffer requests over several detectors (ace_server_*).
    Keeps every request's arrays alive until its ticket has been waited for."""

    def __init__(self, detectors, mem_budget_bytes: int = 1 << 30):
        self._dets = list(detectors)
        arr = (ctypes.c_void_p * len(self._dets))(*[d._h for d in self._dets])
        h = ctypes.c_void_p()
        _check(load_library().ace_server_create(arr, len(self._dets), int(mem_budget_bytes), ctypes.byref(h)))
        self._h = h
        self._submit = load_library().ace_server_submit
        self._live = {}

    def submit(self, det: int, op: int, X: np.ndarray, alpha: float = 1.0, scores=None, sums=None, flags=None) -> int:
        if X.dtype not in (np.float32, np.uint16):
            raise TypeError("X must be float32 or uint16 bfloat16 bits")
        dt = ACE_F32 if X.dtype == np.float32 else ACE_BF16

        def p(a):  # argtypes turn an int or None into the pointer argument
            return a.ctypes.data if a is not None else None

        t = ctypes.c_uint64()
        _check(self._submit(self._h, int(det), int(op), X.ctypes.data, X.shape[0], dt, float(alpha), p(scores), p(sums),
                            p(flags), ctypes.byref(t)))
        self._live[t.value] = (X, scores, sums, flags)
        return t.value

    def wait(self, ticket: int) -> float:
        """Blocks until the request has completed; returns its latency in seconds."""
        lat = ctypes.c_double()
        try:
            _check(load_library().ace_server_wait(self._h, ctypes.c_uint64(ticket), ctypes.byref(lat)))
        finally:
            self._live.pop(ticket, None)
        return lat.value

    def drain(self):
        _check(load_library().ace_server_drain(self._h))

    def info(self) -> dict:
        """Scheduler threads, and requests admitted inside another request's launch set."""
        t, c = ctypes.c_int(), ctypes.c_uint64()
        _check(load_library().ace_server_info(self._h, ctypes.byref(t), ctypes.byref(c)))
        return {"threads": t.value, "coalesced": c.value}

    def close(self):
        if self._h:
            load_library().ace_server_destroy(self._h)
            self._h = None
            self._live.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def tc_probe(A: np.ndarray, B: np.ndarray) -> np.ndarray:
    """ace_tc_probe: D = A . B^T on the tensor cores (A 128 x kd, B N x kd bfloat16 bit patterns
    as uint16; kd and N multiples of 16 up to 256), accumulated as kd/16 MMA instructions."""
    A = np.ascontiguousarray(A, dtype=np.uint16)
    B = np.ascontiguousarray(B, dtype=np.uint16)
    assert A.shape[0] == 128 and A.shape[1] == B.shape[1]
    D = np.empty((128, B.shape[0]), dtype=np.float32)
    _check(load_library().ace_tc_probe(ctypes.c_void_p(A.ctypes.data), ctypes.c_void_p(B.ctypes.data), A.shape[1],
                                       B.shape[0], ctypes.c_void_p(D.ctypes.data)))
    return D


def exact_score(Q, D, K: int, stream=None):
    """ace_exact_score: S(q, D) = sum_i p(q, x_i)^K (Eq. 3, SRP's p) for every row q of Q, in
    binary64 (Q and D device tensors of the same dtype, binary32 or bfloat16)."""
    torch = _torch()
    if Q.dtype != D.dtype:
        raise TypeError("Q and D must have the same dtype")
    S = torch.empty(Q.shape[0], dtype=torch.float64, device=Q.device)
    _check(load_library().ace_exact_score(_ptr(Q), Q.shape[0], _ptr(D), D.shape[0], Q.shape[1], _x_dtype(Q), int(K),
                                          _ptr(S), _stream_ptr(stream)))
    return S


def wait_probe(kind: int, limit_cycles: int) -> dict:
    """ace_wait_probe: {"status", "cycles", "aborted_cycles"} of a bounded wait made to run out."""
    st = ctypes.c_uint32()
    cyc = (ctypes.c_int64 * 2)()
    _check(load_library().ace_wait_probe(int(kind), int(limit_cycles), ctypes.byref(st), cyc))
    return {"status": st.value, "cycles": cyc[0], "aborted_cycles": cyc[1]}


def tc_probe_fp8(A: np.ndarray, B: np.ndarray) -> np.ndarray:
    """ace_tc_probe_fp8: D = A . B^T on the tensor cores (A 128 x kd, B N x kd E4M3 bytes as
    uint8; kd a multiple of 32, N of 16, up to 256), accumulated as kd/32 MMA instructions."""
    A = np.ascontiguousarray(A, dtype=np.uint8)
    B = np.ascontiguousarray(B, dtype=np.uint8)
    assert A.shape[0] == 128 and A.shape[1] == B.shape[1]
    D = np.empty((128, B.shape[0]), dtype=np.float32)
    _check(load_library().ace_tc_probe_fp8(ctypes.c_void_p(A.ctypes.data), ctypes.c_void_p(B.ctypes.data),
                                           A.shape[1], B.shape[0], ctypes.c_void_p(D.ctypes.data)))
    return D


def u32(t) -> np.ndarray:
    """int32 tensor holding uint32 bit patterns -> numpy uint32."""
    return t.cpu().numpy().view(np.uint32)
