"""Seeded synthetic inputs shared by the FP64 oracle and the CUDA path.

This package draws inputs only (subject sizes, row non-zero counts, distinct
column ids, values and uniform initial factors).  It holds none of the
PARAFAC2 arithmetic, so it cannot carry a mistake from one side to the other.

The generator itself is C (``p2synth.c``, OpenMP, counter-based SplitMix64),
built on first use into ``_p2synth.so`` next to this file.

Workloads (shapes of the paper's synthetic experiment, Section 5: K subjects,
J variables, at most 100 observations each; the paper reports 63M-500M
non-zeros at R = 10 and 40):

* ``tiny``  K=200, J=100, I_k ~ U{1..20}, Poisson(3)+1 nnz/row, uniform columns, R=5
* ``c63m``  K=1,000,000, J=5,000, I_k ~ U{1..100}, Poisson(0.25)+1 nnz/row,
  Zipf(1.1) columns through a seeded permutation, R=10 (about 63M nnz)
* ``c555m`` as c63m with Poisson(10)+1 nnz/row, R=40 (about 555M nnz)
* ``c250m`` as c63m with Poisson(3.95)+1 nnz/row, R=40 (about 250M nnz)
* ``serve`` projection requests: I ~ round(lognormal(3, 1)) clipped to
  [1, 1000], Poisson(2)+1 nnz/row, Zipf(1.1) columns, J=5,000

Values are 1 + Poisson(1) stored as FP32 in these workloads.

Paper-shaped planted workloads (the recipe of Section 5, "Synthetic Data"):
dense 100 x J slices X_k = Q_k H S_k V^T at planted rank 40, entries kept
uniformly with probability p, empty rows dropped:

* ``p63m``  K=1,000,000, J=5,000, p = 1.26e-4 (about 63M nnz, mean I_k ~ 46.7), R=10
* ``p500m`` K=1,000,000, J=5,000, p = 1e-3 (about 500M nnz, mean I_k ~ 99.3), R=40
* ``ptiny`` K=50, J=200, 20 dense rows, planted rank 6, p = 0.05, R=5
"""
from __future__ import annotations

import ctypes
import hashlib
import os
import subprocess
from dataclasses import dataclass, replace

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "p2synth.c")
_LIB = None


def _so_path() -> str:
    with open(_SRC, "rb") as f:
        h = hashlib.sha1(f.read()).hexdigest()[:12]
    import platform
    return os.path.join(_HERE, f"_p2synth_{platform.machine()}_{h}.so")


def build() -> str:
    """Compile the generator (gcc, OpenMP) if its shared object is missing."""
    so = _so_path()
    if not os.path.exists(so):
        tmp = so + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared",
               "-ffp-contract=off", "-fno-fast-math", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, so)
    return so


class _Cfg(ctypes.Structure):
    _fields_ = [("K", ctypes.c_int64), ("J", ctypes.c_int32), ("imin", ctypes.c_int32),
                ("imax", ctypes.c_int32), ("size_mode", ctypes.c_int32),
                ("mu", ctypes.c_double), ("sigma", ctypes.c_double), ("lam", ctypes.c_double),
                ("col_mode", ctypes.c_int32), ("zipf_s", ctypes.c_double),
                ("val_lam", ctypes.c_double), ("seed", ctypes.c_uint64)]


class _PCfg(ctypes.Structure):
    _fields_ = [("K", ctypes.c_int64), ("J", ctypes.c_int32), ("dense_rows", ctypes.c_int32),
                ("rank", ctypes.c_int32), ("keep_p", ctypes.c_double), ("seed", ctypes.c_uint64)]


def _lib():
    global _LIB
    if _LIB is None:
        lib = ctypes.CDLL(build())
        P = ctypes.POINTER
        lib.p2synth_subjects.argtypes = [P(_Cfg), ctypes.c_void_p]
        lib.p2synth_subjects.restype = ctypes.c_int64
        lib.p2synth_rows.argtypes = [P(_Cfg), ctypes.c_int64, ctypes.c_void_p]
        lib.p2synth_rows.restype = ctypes.c_int64
        lib.p2synth_fill.argtypes = [P(_Cfg), ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p,
                                     ctypes.c_void_p]
        lib.p2synth_fill.restype = ctypes.c_int
        lib.p2synth_uniform.argtypes = [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_int64,
                                        ctypes.c_void_p]
        lib.p2synth_planted_subjects.argtypes = [P(_PCfg), ctypes.c_void_p]
        lib.p2synth_planted_subjects.restype = ctypes.c_int64
        lib.p2synth_planted_rows.argtypes = [P(_PCfg), ctypes.c_void_p, ctypes.c_int64,
                                             ctypes.c_void_p]
        lib.p2synth_planted_rows.restype = ctypes.c_int64
        lib.p2synth_planted_fill.argtypes = [P(_PCfg), ctypes.c_void_p, ctypes.c_void_p,
                                             ctypes.c_void_p, ctypes.c_void_p]
        lib.p2synth_planted_fill.restype = ctypes.c_int
        lib.p2synth_planted_factors.argtypes = [P(_PCfg), ctypes.c_int64, ctypes.c_void_p,
                                                ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
        lib.p2synth_planted_factors.restype = None
        lib.p2synth_uniform.restype = None
        lib.p2synth_threads.argtypes = []
        lib.p2synth_threads.restype = ctypes.c_int
        _LIB = lib
    return _LIB


@dataclass(frozen=True)
class Workload:
    """Recipe of one synthetic collection of sparse slices {X_k}."""
    name: str
    K: int
    J: int
    R: int
    imin: int = 1
    imax: int = 100
    size_mode: int = 0          # 0: I_k ~ U{imin..imax}; 1: round(lognormal(mu, sigma)) clipped
    mu: float = 3.0
    sigma: float = 1.0
    lam: float = 0.25           # non-zeros per row = Poisson(lam) + 1
    col_mode: int = 1           # 0: uniform columns; 1: Zipf(zipf_s) through a seeded permutation
    zipf_s: float = 1.1
    val_lam: float = 1.0        # values = 1 + Poisson(val_lam)
    seed: int = 20170314
    planted_rank: int = 0       # > 0: planted PARAFAC2 model (only K, J and the fields below used)
    keep_p: float = 0.0         # keep probability of a planted entry
    dense_rows: int = 100       # planted observations per subject before sparsification

    def scaled(self, K: int) -> "Workload":
        """Same recipe and seed stream with fewer (or more) subjects."""
        return replace(self, K=int(K), name=f"{self.name}[K={int(K)}]")


WORKLOADS = {
    "tiny": Workload("tiny", K=200, J=100, R=5, imin=1, imax=20, lam=3.0, col_mode=0,
                     seed=20170314 + 0),
    "c63m": Workload("c63m", K=1_000_000, J=5000, R=10, lam=0.25, seed=20170314 + 1),
    "c555m": Workload("c555m", K=1_000_000, J=5000, R=40, lam=10.0, seed=20170314 + 2),
    "c250m": Workload("c250m", K=1_000_000, J=5000, R=40, lam=3.95, seed=20170314 + 3),
    "serve": Workload("serve", K=1000, J=5000, R=40, imin=1, imax=1000, size_mode=1, mu=3.0,
                      sigma=1.0, lam=2.0, seed=20170314 + 4),
    "p63m": Workload("p63m", K=1_000_000, J=5000, R=10, planted_rank=40, keep_p=1.26e-4,
                     seed=20170314 + 5),
    "p500m": Workload("p500m", K=1_000_000, J=5000, R=40, planted_rank=40, keep_p=1e-3,
                      seed=20170314 + 6),
    "ptiny": Workload("ptiny", K=50, J=200, R=5, planted_rank=6, keep_p=0.05, dense_rows=20,
                      seed=20170314 + 7),
}


@dataclass
class Slices:
    """A collection {X_k} as one CSR matrix over stacked rows.

    subj_ptr[k]..subj_ptr[k+1] are the rows of X_k; row_ptr indexes col/val.
    Columns are sorted and distinct within each row; every row is non-empty.
    """
    K: int
    J: int
    subj_ptr: np.ndarray   # int64 [K+1]
    row_ptr: np.ndarray    # int64 [N+1]
    col: np.ndarray        # int32 [nnz]
    val: np.ndarray        # float32 [nnz]

    @property
    def n_rows(self) -> int:
        return int(self.subj_ptr[-1])

    @property
    def nnz(self) -> int:
        return int(self.row_ptr[-1])

    def subject(self, k: int):
        """(row_ptr, col, val) of X_k with row_ptr rebased to 0."""
        r0, r1 = int(self.subj_ptr[k]), int(self.subj_ptr[k + 1])
        rp = self.row_ptr[r0:r1 + 1]
        b, e = int(rp[0]), int(rp[-1])
        return rp - b, self.col[b:e], self.val[b:e]

    def take(self, ks) -> "Slices":
        """Sub-collection of the listed subjects, in the listed order."""
        ks = np.asarray(ks, dtype=np.int64)
        sp = [0]
        rps = [np.zeros(1, np.int64)]
        cols, vals = [], []
        off = 0
        for k in ks:
            rp, c, v = self.subject(int(k))
            rps.append(rp[1:] + off)
            off += int(rp[-1])
            sp.append(sp[-1] + len(rp) - 1)
            cols.append(c)
            vals.append(v)
        return Slices(len(ks), self.J, np.asarray(sp, np.int64), np.concatenate(rps),
                      np.concatenate(cols) if cols else np.zeros(0, np.int32),
                      np.concatenate(vals) if vals else np.zeros(0, np.float32))


def _cfg(w: Workload) -> _Cfg:
    return _Cfg(w.K, w.J, w.imin, w.imax, w.size_mode, w.mu, w.sigma, w.lam, w.col_mode,
                w.zipf_s, w.val_lam, w.seed)


def generate(w: Workload | str, K: int | None = None) -> Slices:
    """Draw the slices of workload ``w`` (optionally with K subjects)."""
    if isinstance(w, str):
        w = WORKLOADS[w]
    if K is not None:
        w = w.scaled(K)
    lib = _lib()
    if w.planted_rank > 0:
        return _generate_planted(w)
    cfg = _cfg(w)
    subj_ptr = np.zeros(w.K + 1, np.int64)
    n = lib.p2synth_subjects(ctypes.byref(cfg), subj_ptr.ctypes.data)
    row_ptr = np.zeros(n + 1, np.int64)
    nnz = lib.p2synth_rows(ctypes.byref(cfg), n, row_ptr.ctypes.data)
    col = np.empty(nnz, np.int32)
    val = np.empty(nnz, np.float32)
    if lib.p2synth_fill(ctypes.byref(cfg), n, row_ptr.ctypes.data, col.ctypes.data,
                        val.ctypes.data) != 0:
        raise MemoryError("p2synth_fill: allocation failed")
    return Slices(w.K, w.J, subj_ptr, row_ptr, col, val)


def _pcfg(w: Workload) -> _PCfg:
    return _PCfg(w.K, w.J, w.dense_rows, w.planted_rank, w.keep_p, w.seed)


def _generate_planted(w: Workload) -> Slices:
    lib = _lib()
    cfg = _pcfg(w)
    subj_ptr = np.zeros(w.K + 1, np.int64)
    n = lib.p2synth_planted_subjects(ctypes.byref(cfg), subj_ptr.ctypes.data)
    row_ptr = np.zeros(n + 1, np.int64)
    nnz = lib.p2synth_planted_rows(ctypes.byref(cfg), subj_ptr.ctypes.data, n,
                                   row_ptr.ctypes.data)
    col = np.empty(nnz, np.int32)
    val = np.empty(nnz, np.float32)
    if lib.p2synth_planted_fill(ctypes.byref(cfg), subj_ptr.ctypes.data, row_ptr.ctypes.data,
                                col.ctypes.data, val.ctypes.data) != 0:
        raise MemoryError("p2synth_planted_fill: allocation failed")
    return Slices(w.K, w.J, subj_ptr, row_ptr, col, val)


def planted_factors(w: Workload | str, k: int):
    """The planted H (Rp x Rp), V (J x Rp) and subject k's S_k diagonal (Rp)
    and reflector vector v (dense_rows): Q_k = (I - 2 v v^T)[:, :Rp]."""
    if isinstance(w, str):
        w = WORKLOADS[w]
    Rp = w.planted_rank
    H = np.empty((Rp, Rp), np.float32)
    V = np.empty((w.J, Rp), np.float32)
    s = np.empty(Rp, np.float32)
    v = np.empty(w.dense_rows, np.float64)
    _lib().p2synth_planted_factors(ctypes.byref(_pcfg(w)), int(k), H.ctypes.data,
                                   V.ctypes.data, s.ctypes.data, v.ctypes.data)
    return H, V, s, v


def uniform(seed: int, stream: int, shape) -> np.ndarray:
    """FP32 values uniform in [0,1), multiples of 2^-24 (exact in FP32 and FP64)."""
    n = int(np.prod(shape))
    out = np.empty(n, np.float32)
    _lib().p2synth_uniform(seed, stream, n, out.ctypes.data)
    return out.reshape(shape)


def init_factors(R: int, J: int, K: int, seed: int):
    """Initial H (R x R), V (J x R), W (K x R), all U[0,1) in FP32.

    The paper leaves the initialisation open (Algorithm 2 only says
    "Initialize"); both the oracle and the CUDA path start from these arrays.
    """
    return uniform(seed, 1, (R, R)), uniform(seed, 2, (J, R)), uniform(seed, 3, (K, R))


def host_threads() -> int:
    """OpenMP threads the generator uses on this host."""
    return int(_lib().p2synth_threads())
