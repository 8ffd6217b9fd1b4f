"""CPU oracle for the ACE hot path (Luo & Shrivastava, Arrays of locality-sensitive Count
Estimators) — TEST INFRASTRUCTURE.

Only the test suite, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline leg may
import this package.  The CUDA library never imports, links or calls it, and it never
imports the CUDA library: the two share no code.

The arithmetic lives in ``ace_oracle.c`` (plain C, binary64, ``-ffp-contract=off``); this
module builds it with gcc, loads it with ctypes and strings its steps together with the
same call semantics as the library's C ABI:

* ``insert(X)``       Algorithm 1 pre-processing phase (§3.2 counting phase).
* ``score(X, alpha)`` Algorithm 1 query phase, then the §5.3 threshold rule
                      (score < mu - alpha*sigma over every score returned so far).
* ``insert_score``    insert the whole batch, then score it against the updated arrays.
* ``WindowDetector``  the same over a sliding window of the last W inserted points: before a
                      batch is inserted, the oldest points beyond W are removed by §3.4.1
                      deletion (Eq. 12), so the arrays always count the most recent points.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ace_oracle.c")
_LIB_PATH = os.path.join(_HERE, "_ace_oracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile ace_oracle.c into _ace_oracle.so with gcc (OpenMP if available)."""
    if not force and os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC):
        return _LIB_PATH
    base = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared", "-std=c11"]
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = base + ["-fopenmp", "-o", tmp, _SRC, "-lm"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        cmd = base + ["-o", tmp, _SRC, "-lm"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("oracle build failed:\n" + r.stderr)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(build())
        P = ctypes.c_void_p
        i32, i64, u64, f64 = ctypes.c_int, ctypes.c_int64, ctypes.c_uint64, ctypes.c_double
        lib.oracle_projection_from_seed.argtypes = [i32, i32, i32, u64, P]
        lib.oracle_projection_from_seed_bf16.argtypes = [i32, i32, i32, u64, P]
        lib.oracle_projection_counter.argtypes = [i32, i32, i32, u64, P]
        lib.oracle_projection_hadamard.argtypes = [i32, i32, i32, u64, P]
        lib.oracle_splitmix64_draw.argtypes = [u64, u64]
        lib.oracle_splitmix64_draw.restype = u64
        lib.oracle_hash.argtypes = [P, i32, i64, i32, P, i32, i32, P]
        lib.oracle_hash_noisy.argtypes = [P, i32, i64, i32, P, i32, i32, ctypes.c_float, u64, u64, P]
        lib.oracle_project.argtypes = [P, i32, i64, i32, P, i32, P]
        lib.oracle_insert.argtypes = [P, i64, i32, i32, P]
        lib.oracle_insert.restype = i32
        lib.oracle_delete.argtypes = [P, i64, i32, i32, P]
        lib.oracle_delete.restype = i32
        lib.oracle_mu_decremental.argtypes = [P, i64, i32, i32, P, i64, f64, P]
        lib.oracle_mu_decremental.restype = f64
        lib.oracle_sum_squares.argtypes = [P, i32, i32, P]
        lib.oracle_mu_incremental.argtypes = [P, i64, i32, i32, P, i64, f64, P]
        lib.oracle_mu_incremental.restype = f64
        lib.oracle_gather.argtypes = [P, i64, i32, i32, P, P]
        lib.oracle_gather.restype = i32
        lib.oracle_stats_fold.argtypes = [P, P, i64]
        lib.oracle_stats_threshold.argtypes = [P, i32, f64, P]
        lib.oracle_stats_threshold.restype = i32
        lib.oracle_score_flags.argtypes = [P, i64, i32, f64, P, P]
        lib.oracle_mu_from_q.argtypes = [P, u64, i32]
        lib.oracle_mu_from_q.restype = f64
        lib.oracle_num_threads.restype = i32
        lib.oracle_set_num_threads.argtypes = [i32]
        _lib = lib
        return lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def num_threads() -> int:
    return int(_load().oracle_num_threads())


def set_num_threads(t: int) -> None:
    _load().oracle_set_num_threads(int(t))


def splitmix64_draw(seed: int, t: int) -> int:
    """Draw number t of SplitMix64 started at state ``seed`` (counter mode)."""
    return int(_load().oracle_splitmix64_draw(ctypes.c_uint64(seed), ctypes.c_uint64(t)))


def projection_from_seed(d: int, K: int, L: int, seed: int, w_bf16: bool = False, counter: bool = False,
                         hadamard: bool = False) -> np.ndarray:
    """d x (K*L) binary32 Gaussian matrix (SplitMix64 counter mode + Box-Muller); with w_bf16
    every value is then rounded to bfloat16 (nearest even); with counter, the integer-only
    matrix (popcount of each draw - 32) / 4 instead; with hadamard, the structured +-1 matrix
    (Sylvester-Hadamard rows with random signs per block of columns)."""
    W = np.empty((d, K * L), dtype=np.float32)
    if hadamard:
        fn = _load().oracle_projection_hadamard
    elif counter:
        fn = _load().oracle_projection_counter
    else:
        fn = _load().oracle_projection_from_seed_bf16 if w_bf16 else _load().oracle_projection_from_seed
    fn(d, K, L, ctypes.c_uint64(seed & (2**64 - 1)), _ptr(W))
    return W


def _x_args(X: np.ndarray):
    if X.dtype == np.float32:
        return np.ascontiguousarray(X), 0
    if X.dtype == np.uint16:  # bfloat16 bit patterns
        return np.ascontiguousarray(X), 1
    raise TypeError("X must be float32 or uint16 (bfloat16 bits)")


def hash_ids(X: np.ndarray, W: np.ndarray, K: int, L: int) -> np.ndarray:
    """Eq. 1 + Eq. 2: n x L bucket ids, H_j(x) = sum_k [w_{jK+k}^T x > 0] 2^k."""
    Xc, dt = _x_args(X)
    n, d = Xc.shape
    Wc = np.ascontiguousarray(W, dtype=np.float32)
    assert Wc.shape == (d, K * L)
    ids = np.empty((n, L), dtype=np.uint32)
    _load().oracle_hash(_ptr(Xc), dt, n, d, _ptr(Wc), K, L, _ptr(ids))
    return ids


def hash_ids_noisy(X: np.ndarray, W: np.ndarray, K: int, L: int, sigma: float, noise_seed: int,
                   nbase: int) -> np.ndarray:
    """§4.5 privacy-preserving SRP: bit c of row i is [w_c^T x + eta > 0] with
    eta = sigma * (popcount(draw (nbase + i) K L + c of noise_seed) - 32) / 4."""
    Xc, dt = _x_args(X)
    n, d = Xc.shape
    Wc = np.ascontiguousarray(W, dtype=np.float32)
    assert Wc.shape == (d, K * L)
    ids = np.empty((n, L), dtype=np.uint32)
    _load().oracle_hash_noisy(_ptr(Xc), dt, n, d, _ptr(Wc), K, L, ctypes.c_float(sigma),
                              ctypes.c_uint64(noise_seed & (2**64 - 1)), ctypes.c_uint64(nbase), _ptr(ids))
    return ids


def project(X: np.ndarray, W: np.ndarray) -> np.ndarray:
    """Binary64 projections in index order, n x KL."""
    Xc, dt = _x_args(X)
    n, d = Xc.shape
    Wc = np.ascontiguousarray(W, dtype=np.float32)
    s = np.empty((n, Wc.shape[1]), dtype=np.float64)
    _load().oracle_project(_ptr(Xc), dt, n, d, _ptr(Wc), Wc.shape[1], _ptr(s))
    return s


def insert_ids(ids: np.ndarray, counts: np.ndarray, K: int) -> None:
    n, L = ids.shape
    ids = np.ascontiguousarray(ids, dtype=np.uint32)
    if _load().oracle_insert(_ptr(ids), n, K, L, _ptr(counts)) != 0:
        raise OverflowError("a count would pass 2^32-1")


def delete_ids(ids: np.ndarray, counts: np.ndarray, K: int) -> None:
    """§3.4.1 deletion: counts[j][ids[i, j]] -= 1; raises (counts unchanged) if a count
    would go below zero."""
    n, L = ids.shape
    ids = np.ascontiguousarray(ids, dtype=np.uint32)
    if _load().oracle_delete(_ptr(ids), n, K, L, _ptr(counts)) != 0:
        raise ValueError("deleting points that were not inserted (a count would go below zero)")


def mu_decremental(ids: np.ndarray, counts: np.ndarray, K: int, n_before: int, mu_before: float):
    """Eq. 12 point by point (pre-decrement counts); updates counts; returns (mu, trace)."""
    n, L = ids.shape
    ids = np.ascontiguousarray(ids, dtype=np.uint32)
    trace = np.empty(n, dtype=np.float64)
    mu = _load().oracle_mu_decremental(_ptr(ids), n, K, L, _ptr(counts), n_before, mu_before, _ptr(trace))
    return mu, trace


def sum_squares(counts: np.ndarray, K: int, L: int) -> int:
    q = np.zeros(2, dtype=np.uint64)
    _load().oracle_sum_squares(_ptr(counts), K, L, _ptr(q))
    return int(q[0]) | (int(q[1]) << 64)


def mu_incremental(ids: np.ndarray, counts: np.ndarray, K: int, n_before: int = 0,
                   mu_before: float = 0.0):
    """Eq. 11 point by point (pre-increment counts); updates counts; returns (mu, trace)."""
    n, L = ids.shape
    ids = np.ascontiguousarray(ids, dtype=np.uint32)
    trace = np.empty(n, dtype=np.float64)
    mu = _load().oracle_mu_incremental(_ptr(ids), n, K, L, _ptr(counts), n_before, mu_before, _ptr(trace))
    return mu, trace


def gather(ids: np.ndarray, counts: np.ndarray, K: int) -> np.ndarray:
    n, L = ids.shape
    ids = np.ascontiguousarray(ids, dtype=np.uint32)
    sums = np.empty(n, dtype=np.uint32)
    if _load().oracle_gather(_ptr(ids), n, K, L, _ptr(counts), _ptr(sums)) != 0:
        raise OverflowError("a per-point count sum does not fit in 32 bits")
    return sums


class Detector:
    """The oracle's detector state: W, the L count arrays, and the running sums."""

    def __init__(self, d: int, K: int, L: int, seed: int | None = None, W: np.ndarray | None = None,
                 w_bf16: bool = False):
        self.d, self.K, self.L = d, K, L
        if W is None:
            W = projection_from_seed(d, K, L, seed if seed is not None else 0, w_bf16=w_bf16)
        self.W = np.ascontiguousarray(W, dtype=np.float32)
        assert self.W.shape == (d, K * L)
        self.counts = np.zeros((L, 1 << K), dtype=np.uint32)
        self.n_ins = 0
        self.st = np.zeros(5, dtype=np.uint64)  # N, S1 lo/hi, S2 lo/hi
        self.sigma, self.noise_seed, self.nbase = 0.0, 0, 0

    def set_privacy(self, sigma: float, noise_seed: int = 0):
        """§4.5: noise before the sign from now on; the noise index restarts at 0."""
        self.sigma, self.noise_seed, self.nbase = float(np.float32(sigma)), noise_seed, 0

    def hash(self, X):
        if self.sigma == 0.0:
            return hash_ids(X, self.W, self.K, self.L)
        ids = hash_ids_noisy(X, self.W, self.K, self.L, self.sigma, self.noise_seed, self.nbase)
        self.nbase += ids.shape[0]
        return ids

    def insert(self, X):
        ids = self.hash(X)
        insert_ids(ids, self.counts, self.K)
        self.n_ins += ids.shape[0]
        return ids

    def delete(self, X):
        """Removes the batch's points from the arrays (§3.4.1); all or nothing."""
        if self.sigma != 0.0:
            raise ValueError("with privacy noise a point does not hash to its inserted ids")
        ids = self.hash(X)
        if ids.shape[0] > self.n_ins:
            raise ValueError("deleting more points than were inserted")
        delete_ids(ids, self.counts, self.K)
        self.n_ins -= ids.shape[0]
        return ids

    def _score_ids(self, ids, alpha):
        lib = _load()
        sums = gather(ids, self.counts, self.K)
        lib.oracle_stats_fold(_ptr(self.st), _ptr(sums), sums.shape[0])
        out = np.zeros(3, dtype=np.float64)
        rc = lib.oracle_stats_threshold(_ptr(self.st), self.L, float(alpha), _ptr(out))
        if rc == 2:
            raise OverflowError("N*S2 does not fit in 128 bits")
        n = sums.shape[0]
        scores = np.empty(n, dtype=np.float64)
        flags = np.empty(n, dtype=np.uint8)
        lib.oracle_score_flags(_ptr(sums), n, self.L, float(out[2]), _ptr(scores), _ptr(flags))
        return scores, sums, flags

    def score(self, X, alpha: float = 1.0):
        return self._score_ids(self.hash(X), alpha)

    def insert_score(self, X, alpha: float = 1.0):
        ids = self.insert(X)
        return self._score_ids(ids, alpha)

    def q(self) -> int:
        return sum_squares(self.counts, self.K, self.L)

    def stats(self, alpha: float = 1.0) -> dict:
        lib = _load()
        out = np.zeros(3, dtype=np.float64)
        rc = lib.oracle_stats_threshold(_ptr(self.st), self.L, float(alpha), _ptr(out))
        qv = self.q()
        ql = np.array([qv & (2**64 - 1), qv >> 64], dtype=np.uint64)
        mu_ins = lib.oracle_mu_from_q(_ptr(ql), self.n_ins, self.L) if self.n_ins else 0.0
        st = [int(v) for v in self.st]
        return {
            "n_ins": self.n_ins, "n_scored": st[0], "Q": qv,
            "S1": st[1] | (st[2] << 64), "S2": st[3] | (st[4] << 64),
            "mu_ins": mu_ins, "mu": out[0] if rc == 0 else 0.0, "sigma": out[1] if rc == 0 else 0.0,
            "threshold": out[2] if rc == 0 else 0.0,
        }


class WindowDetector(Detector):
    """A detector whose arrays count only the last `window` inserted points (in insertion
    order: earlier batches first, rows of a batch in order).  Inserting a batch of n <= window
    points first removes the oldest max(0, held + n - window) points, each by §3.4.1 deletion
    of its ids (the decrements of Eq. 12), then inserts the batch.  Scoring is unchanged."""

    def __init__(self, d: int, K: int, L: int, window: int, seed: int | None = None, W: np.ndarray | None = None):
        super().__init__(d, K, L, seed=seed, W=W)
        if window < 1:
            raise ValueError("window must be at least 1")
        self.window = int(window)
        self.held = np.zeros((0, L), dtype=np.uint32)  # ids of the points in the window, oldest first

    def insert(self, X):
        ids = self.hash(X)
        n = ids.shape[0]
        if n > self.window:
            raise ValueError("a batch larger than the window")
        m = max(0, self.held.shape[0] + n - self.window)
        if m:
            delete_ids(self.held[:m], self.counts, self.K)
            self.held = self.held[m:]
            self.n_ins -= m
        insert_ids(ids, self.counts, self.K)
        self.held = np.concatenate([self.held, ids], axis=0)
        self.n_ins += n
        return ids

    def insert_score(self, X, alpha: float = 1.0):
        ids = self.insert(X)
        return self._score_ids(ids, alpha)


def exact_score(Q: np.ndarray, D: np.ndarray, K: int) -> np.ndarray:
    """Eq. 3 with SRP's collision probability (§3): S(q, D) = sum_i p(q, x_i)^K,
    p(q, x) = 1 - acos(q.x / (||q|| ||x||)) / pi, in binary64, for every row q of Q (binary32
    or bfloat16 bits).  A zero vector has no angle; its SRP bits are all 0 (sign(0) = 0), so
    against a non-zero point each of its bits agrees with probability 1/2: p = 1/2 (and p = 1
    between two zero vectors)."""
    def f64(A):
        A = np.asarray(A)
        if A.dtype == np.uint16:
            return (A.astype(np.uint32) << 16).view(np.float32).astype(np.float64)
        return A.astype(np.float64)
    Qd, Dd = f64(Q), f64(D)
    qq = (Qd * Qd).sum(axis=1)
    xx = (Dd * Dd).sum(axis=1)
    dot = Qd @ Dd.T
    with np.errstate(divide="ignore", invalid="ignore"):
        c = dot / np.sqrt(qq[:, None] * xx[None, :])
    p = 1.0 - np.arccos(np.clip(c, -1.0, 1.0)) / np.pi
    zq, zx = (qq == 0)[:, None], (xx == 0)[None, :]
    p = np.where(zq & zx, 1.0, np.where(zq | zx, 0.5, p))
    return (p ** K).sum(axis=1)


def rse(Q: np.ndarray, D: np.ndarray, K: int, idx: np.ndarray) -> np.ndarray:
    """The random sampling estimator (Eq. 10): n / |S| times sum over the sample S = D[idx]
    of p(q, x_i)^K."""
    return exact_score(Q, np.asarray(D)[idx], K) * (len(D) / len(idx))
