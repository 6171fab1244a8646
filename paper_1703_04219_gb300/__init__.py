"""p2: PARAFAC2-ALS in SPARTan's formulation on one GB300 GPU.

Thin ctypes binding of ``libp2.so`` (C ABI declared in ``include/p2.h``).
The functions below carry the C names and only marshal arguments; every
step of the computation runs in the library's CUDA kernels.  There is no
CPU fallback: importing this package fails if ``libp2.so`` has not been
built (``python paper_1703_04219_gb300/build.py`` or
``__graft_entry__.build()``).
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libp2.so")

P2_OK, P2_EINVAL, P2_ENOMEM, P2_ECUDA, P2_ENUMERIC, P2_ETIMEOUT, P2_ESTATE, P2_EEXCHANGE = range(8)
P2_FP32, P2_BF16 = 0, 1
_NAMES = {0: "P2_OK", 1: "P2_EINVAL", 2: "P2_ENOMEM", 3: "P2_ECUDA", 4: "P2_ENUMERIC",
          5: "P2_ETIMEOUT", 6: "P2_ESTATE", 7: "P2_EEXCHANGE"}

# every symbol include/p2.h declares
EXPORTED = ("p2_default_options", "p2_create", "p2_destroy", "p2_load_slices", "p2_init",
            "p2_init_eig",
            "p2_iterate", "p2_fit", "p2_get_factors", "p2_set_factors", "p2_get_mttkrp",
            "p2_get_procrustes", "p2_get_U", "p2_iterate_until", "p2_stats", "p2_device_bytes", "p2_mode1_stats_noalloc",
            "p2_projector_create", "p2_projector_destroy", "p2_project", "p2_projector_sync",
            "p2_set_exchange", "p2_projector_bytes", "p2_get_tuning", "p2_set_tuning",
            "p2_tuning_note", "p2_last_error")


class p2_options(ctypes.Structure):
    _fields_ = [("R", ctypes.c_int32), ("precision", ctypes.c_int32), ("device", ctypes.c_int32),
                ("use_graph", ctypes.c_int32), ("rank_rtol", ctypes.c_double),
                ("stream", ctypes.c_void_p), ("timing", ctypes.c_int32),
                ("seed", ctypes.c_uint64), ("nonneg", ctypes.c_int32),
                ("fp64_procrustes", ctypes.c_int32), ("autotune", ctypes.c_int32),
                ("tune_cache", ctypes.c_char_p), ("tensor_core_m", ctypes.c_int32)]


class p2_tuning(ctypes.Structure):
    _fields_ = [("procrustes_split", ctypes.c_int32), ("subject_bins", ctypes.c_int32),
                ("split_record_cap", ctypes.c_int32), ("m2_block_kib", ctypes.c_int32)]


class p2_stats_t(ctypes.Structure):
    _fields_ = [("kernel_launches", ctypes.c_int64), ("iterations", ctypes.c_int64),
                ("polar_fp64_flops", ctypes.c_double), ("n_phases", ctypes.c_int32),
                ("phase_ms", ctypes.c_float * 8)]


PHASES = ("h_solve", "beta_mode2", "v_solve", "alpha_mode3_w_gram", "procrustes",
          "subject_stats_mode1", "fit")


class P2Error(RuntimeError):
    def __init__(self, code, where, msg):
        super().__init__(f"{where}: {_NAMES.get(code, code)}: {msg}")
        self.code = code


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"libp2.so not found at {LIB_PATH}: build it first "
                          "(python paper_1703_04219_gb300/build.py); there is no CPU fallback")
    lib = ctypes.CDLL(LIB_PATH)
    vp, i32, i64, dbl = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_double
    sig = {
        "p2_default_options": ([ctypes.POINTER(p2_options), i32], None),
        "p2_create": ([ctypes.POINTER(vp), ctypes.POINTER(p2_options)], ctypes.c_int),
        "p2_destroy": ([vp], ctypes.c_int),
        "p2_load_slices": ([vp, i64, i32, vp, vp, vp, vp, i32], ctypes.c_int),
        "p2_init": ([vp, vp, vp, vp], ctypes.c_int),
        "p2_init_eig": ([vp, i32, ctypes.c_double, ctypes.POINTER(i32)], ctypes.c_int),
        "p2_iterate": ([vp, i32, ctypes.POINTER(dbl)], ctypes.c_int),
        "p2_fit": ([vp, ctypes.POINTER(dbl), ctypes.POINTER(dbl)], ctypes.c_int),
        "p2_get_factors": ([vp, vp, vp, vp], ctypes.c_int),
        "p2_set_factors": ([vp, vp, vp, vp], ctypes.c_int),
        "p2_get_mttkrp": ([vp, i32, vp], ctypes.c_int),
        "p2_get_procrustes": ([vp, i64, i64, vp], ctypes.c_int),
        "p2_get_U": ([vp, i64, i64, vp], ctypes.c_int),
        "p2_iterate_until": ([vp, i32, ctypes.c_double, ctypes.POINTER(i32),
                              ctypes.POINTER(ctypes.c_double)], ctypes.c_int),
        "p2_stats": ([vp, ctypes.POINTER(p2_stats_t)], ctypes.c_int),
        "p2_device_bytes": ([vp, ctypes.POINTER(i64)], ctypes.c_int),
        "p2_mode1_stats_noalloc": ([i64, i32, vp, vp, vp, vp, vp, vp], ctypes.c_int),
        "p2_projector_create": ([vp, i64, i64, i64, vp, ctypes.POINTER(vp)], ctypes.c_int),
        "p2_projector_destroy": ([vp], ctypes.c_int),
        "p2_project": ([vp, i64, vp, vp, vp, vp, i32, i32, vp, vp, i32], ctypes.c_int),
        "p2_projector_sync": ([vp], ctypes.c_int),
        "p2_set_exchange": ([vp, vp, vp], ctypes.c_int),
        "p2_projector_bytes": ([vp, i64, i64, i64, ctypes.POINTER(i64)], ctypes.c_int),
        "p2_get_tuning": ([vp, ctypes.POINTER(p2_tuning)], ctypes.c_int),
        "p2_set_tuning": ([vp, ctypes.POINTER(p2_tuning)], ctypes.c_int),
        "p2_tuning_note": ([vp], ctypes.c_char_p),
        "p2_last_error": ([], ctypes.c_char_p),
    }
    for name, (args, res) in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = res
    return lib


lib = _load()


def p2_last_error() -> str:
    return lib.p2_last_error().decode(errors="replace")


def _check(rc, where):
    if rc != P2_OK:
        raise P2Error(rc, where, p2_last_error())


def _ptr(a):
    """Address of a contiguous numpy array or torch tensor (None -> NULL)."""
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return ctypes.c_void_p(a.data_ptr())
    if not a.flags["C_CONTIGUOUS"]:
        raise ValueError("array must be C-contiguous")
    return ctypes.c_void_p(a.ctypes.data)


def p2_default_options(R: int) -> p2_options:
    o = p2_options()
    lib.p2_default_options(ctypes.byref(o), R)
    return o


def p2_create(opt: p2_options):
    h = ctypes.c_void_p()
    _check(lib.p2_create(ctypes.byref(h), ctypes.byref(opt)), "p2_create")
    return h


def p2_destroy(ctx):
    _check(lib.p2_destroy(ctx), "p2_destroy")


def p2_load_slices(ctx, K, J, subj_ptr, row_ptr, col, val, location=None):
    if location is None:
        location = 1 if hasattr(subj_ptr, "is_cuda") and subj_ptr.is_cuda else 0
    if location == 0:
        def host(a, dt):
            return a if hasattr(a, "data_ptr") else np.ascontiguousarray(a, dt)
        subj_ptr, row_ptr = host(subj_ptr, np.int64), host(row_ptr, np.int64)
        col, val = host(col, np.int32), host(val, np.float32)
    _check(lib.p2_load_slices(ctx, int(K), int(J), _ptr(subj_ptr), _ptr(row_ptr), _ptr(col),
                              _ptr(val), int(location)), "p2_load_slices")


def p2_init(ctx, H0=None, V0=None, W0=None):
    """H0, V0, W0 all None: the library draws them from the context's seed."""
    if H0 is None and V0 is None and W0 is None:
        _check(lib.p2_init(ctx, None, None, None), "p2_init")
        return
    H0, V0, W0 = (np.ascontiguousarray(a, np.float32) for a in (H0, V0, W0))
    _check(lib.p2_init(ctx, _ptr(H0), _ptr(V0), _ptr(W0)), "p2_init")


def p2_init_eig(ctx, max_iter: int = 500, tol: float = 1e-6) -> int:
    """Rational start (H = I, W = 1, V = leading eigenvectors of sum_k X_k^T X_k);
    returns the number of subspace-iteration products run."""
    n = ctypes.c_int32(0)
    _check(lib.p2_init_eig(ctx, int(max_iter), float(tol), ctypes.byref(n)), "p2_init_eig")
    return int(n.value)


def p2_set_factors(ctx, H, V, W):
    H, V, W = (np.ascontiguousarray(a, np.float32) for a in (H, V, W))
    _check(lib.p2_set_factors(ctx, _ptr(H), _ptr(V), _ptr(W)), "p2_set_factors")


def p2_iterate(ctx, n_iter: int, want_fit: bool = True):
    f = ctypes.c_double()
    _check(lib.p2_iterate(ctx, int(n_iter), ctypes.byref(f) if want_fit else None), "p2_iterate")
    return f.value if want_fit else None


def p2_iterate_until(ctx, max_iter: int, tol: float):
    n = ctypes.c_int32()
    f = ctypes.c_double()
    _check(lib.p2_iterate_until(ctx, int(max_iter), float(tol), ctypes.byref(n), ctypes.byref(f)),
           "p2_iterate_until")
    return n.value, f.value


def p2_fit(ctx):
    f, l = ctypes.c_double(), ctypes.c_double()
    _check(lib.p2_fit(ctx, ctypes.byref(f), ctypes.byref(l)), "p2_fit")
    return f.value, l.value


def p2_get_factors(ctx, R, J, K):
    H = np.empty((R, R), np.float32)
    V = np.empty((J, R), np.float32)
    W = np.empty((K, R), np.float32)
    _check(lib.p2_get_factors(ctx, _ptr(H), _ptr(V), _ptr(W)), "p2_get_factors")
    return H, V, W


def p2_get_mttkrp(ctx, mode, R, J, K):
    shape = {1: (R, R), 2: (J, R), 3: (K, R)}[mode]
    out = np.empty(shape, np.float64)
    _check(lib.p2_get_mttkrp(ctx, int(mode), _ptr(out)), "p2_get_mttkrp")
    return out


def p2_get_procrustes(ctx, k0, k1, R):
    out = np.empty((k1 - k0, R, R), np.float32)
    _check(lib.p2_get_procrustes(ctx, int(k0), int(k1), _ptr(out)), "p2_get_procrustes")
    return out


def p2_get_U(ctx, k0, k1, n_rows, R):
    out = np.empty((int(n_rows), R), np.float32)
    _check(lib.p2_get_U(ctx, int(k0), int(k1), _ptr(out)), "p2_get_U")
    return out


def p2_stats(ctx) -> dict:
    st = p2_stats_t()
    _check(lib.p2_stats(ctx, ctypes.byref(st)), "p2_stats")
    return dict(kernel_launches=st.kernel_launches, iterations=st.iterations,
                polar_fp64_flops=st.polar_fp64_flops,
                phase_ms={PHASES[i]: st.phase_ms[i] for i in range(st.n_phases)})


def p2_device_bytes(ctx) -> int:
    b = ctypes.c_int64()
    _check(lib.p2_device_bytes(ctx, ctypes.byref(b)), "p2_device_bytes")
    return b.value


def p2_mode1_stats_noalloc(K, R, T, G, W, M1, WtW=None, stream=None):
    """Allocation-free mode-1 MTTKRP and W^TW from device tensors (see include/p2.h).

    T (K x R x R float32), G (K x R(R+1)/2 float64), W (K x R float32) and the
    outputs M1, WtW (R x R float64) are contiguous CUDA tensors on the current
    device; stream is a cudaStream_t handle (default: torch's current stream).
    For callers that cannot allocate device memory at the point of the call.
    Tensors of another kind, device, dtype or size raise ValueError here,
    before the library sees them.
    """
    import torch
    K, R = int(K), int(R)
    want = {"T": (T, torch.float32, K * R * R), "G": (G, torch.float64, K * R * (R + 1) // 2),
            "W": (W, torch.float32, K * R), "M1": (M1, torch.float64, R * R)}
    if WtW is not None:
        want["WtW"] = (WtW, torch.float64, R * R)
    dev = torch.cuda.current_device()
    for name, (t, dtype, n) in want.items():
        if not isinstance(t, torch.Tensor) or not t.is_cuda:
            raise ValueError(f"{name} must be a CUDA tensor")
        if t.device.index != dev:
            raise ValueError(f"{name} is on cuda:{t.device.index}, the current device is cuda:{dev}")
        if t.dtype != dtype:
            raise ValueError(f"{name} must be {dtype}, got {t.dtype}")
        if t.numel() != n:
            raise ValueError(f"{name} must hold {n} elements, got {t.numel()}")
        if not t.is_contiguous():
            raise ValueError(f"{name} must be contiguous")
    if stream is None:
        stream = torch.cuda.current_stream().cuda_stream
    _check(lib.p2_mode1_stats_noalloc(K, R, _ptr(T), _ptr(G), _ptr(W), _ptr(M1),
                                      _ptr(WtW), ctypes.c_void_p(stream)),
           "p2_mode1_stats_noalloc")


def p2_projector_bytes(model, max_subjects, max_rows, max_nnz) -> int:
    """Device bytes of a projector with these capacities on the model."""
    b = ctypes.c_int64()
    _check(lib.p2_projector_bytes(model.ctx, int(max_subjects), int(max_rows), int(max_nnz),
                                  ctypes.byref(b)), "p2_projector_bytes")
    return b.value


class Projector:
    """Projects new subjects onto a fitted model (fixed H, V): see p2_project."""

    def __init__(self, model: "Parafac2", max_subjects: int, max_rows: int, max_nnz: int,
                 stream=None):
        self.model = model
        self.R = model.R
        h = ctypes.c_void_p()
        _check(lib.p2_projector_create(model.ctx, int(max_subjects), int(max_rows),
                                       int(max_nnz), stream, ctypes.byref(h)),
               "p2_projector_create")
        self.h = h
        self.capacity = (int(max_subjects), int(max_rows), int(max_nnz))

    def close(self):
        if self.h is not None:
            _check(lib.p2_projector_destroy(self.h), "p2_projector_destroy")
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def submit(self, n_req, subj_ptr, row_ptr, col, val, n_iter, S_out, T_out=None,
               location=0, out_location=0):
        """Enqueue one batch; arrays must stay alive until sync()."""
        _check(lib.p2_project(self.h, int(n_req), _ptr(subj_ptr), _ptr(row_ptr), _ptr(col),
                              _ptr(val), int(location), int(n_iter), _ptr(S_out), _ptr(T_out),
                              int(out_location)), "p2_project")

    def sync(self):
        _check(lib.p2_projector_sync(self.h), "p2_projector_sync")

    def project(self, slices, n_iter=10, want_T=False):
        """Synchronous convenience call on host arrays: returns S (and T)."""
        sp = np.ascontiguousarray(slices.subj_ptr, np.int64)
        rp = np.ascontiguousarray(slices.row_ptr, np.int64)
        col = np.ascontiguousarray(slices.col, np.int32)
        val = np.ascontiguousarray(slices.val, np.float32)
        S = np.empty((slices.K, self.R), np.float32)
        T = np.empty((slices.K, self.R, self.R), np.float32) if want_T else None
        self.submit(slices.K, sp, rp, col, val, n_iter, S, T)
        self.sync()
        return (S, T) if want_T else S


class Parafac2:
    """Owning wrapper of one context: load, init, iterate, read back."""

    def __init__(self, R: int, device: int = 0, use_graph: bool = True, rank_rtol: float = 1e-5,
                 stream=None, timing: bool = False, precision: str = "fp32", seed=None,
                 nonneg: bool = False, fp64_procrustes: bool = False, autotune: bool = False,
                 tune_cache=None, tensor_core_m=None):
        if precision not in ("fp32", "bf16"):
            raise ValueError("precision must be 'fp32' or 'bf16'")
        opt = p2_default_options(R)
        opt.precision = P2_BF16 if precision == "bf16" else P2_FP32
        opt.device = device
        opt.use_graph = 1 if use_graph else 0
        opt.rank_rtol = rank_rtol
        opt.stream = stream
        opt.timing = 1 if timing else 0
        if seed is not None:
            opt.seed = int(seed)
        opt.nonneg = 1 if nonneg else 0
        opt.fp64_procrustes = 1 if fp64_procrustes else 0
        opt.autotune = 1 if autotune else 0
        if tensor_core_m is not None:       # None: the library's rule
            opt.tensor_core_m = 1 if tensor_core_m else 0
        self._tune_cache = tune_cache.encode() if tune_cache else None   # kept alive
        opt.tune_cache = self._tune_cache
        self.R = R
        self.precision = precision
        self.ctx = p2_create(opt)
        self.K = self.J = 0

    def close(self):
        if self.ctx is not None:
            p2_destroy(self.ctx)
            self.ctx = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def load(self, slices, location=None):
        p2_load_slices(self.ctx, slices.K, slices.J, slices.subj_ptr, slices.row_ptr, slices.col,
                       slices.val, location)
        self.K, self.J = int(slices.K), int(slices.J)
        sp = slices.subj_ptr
        self._subj_ptr = np.asarray(sp.cpu() if hasattr(sp, "cpu") else sp, np.int64)

    def init(self, H0=None, V0=None, W0=None):
        p2_init(self.ctx, H0, V0, W0)

    def init_eig(self, max_iter: int = 500, tol: float = 1e-6) -> int:
        """Deterministic rational start; returns the subspace-iteration products run."""
        return p2_init_eig(self.ctx, max_iter, tol)

    def set_factors(self, H, V, W):
        p2_set_factors(self.ctx, H, V, W)

    def iterate(self, n: int, want_fit: bool = True):
        return p2_iterate(self.ctx, n, want_fit)

    def iterate_until(self, max_iter: int, tol: float):
        """(iterations run, fit) of the loop that stops when the fit changes by <= tol."""
        return p2_iterate_until(self.ctx, max_iter, tol)

    def fit(self):
        return p2_fit(self.ctx)

    def factors(self):
        return p2_get_factors(self.ctx, self.R, self.J, self.K)

    def mttkrp(self, mode: int):
        return p2_get_mttkrp(self.ctx, mode, self.R, self.J, self.K)

    def procrustes(self, k0=0, k1=None):
        return p2_get_procrustes(self.ctx, k0, self.K if k1 is None else k1, self.R)

    def U(self, k0=0, k1=None):
        """Rows of U_k = Q_k H for subjects k0 .. k1-1, stacked (Section 3.2)."""
        k1 = self.K if k1 is None else k1
        n = int(self._subj_ptr[k1] - self._subj_ptr[k0])
        return p2_get_U(self.ctx, k0, k1, n, self.R)

    def tuning(self) -> dict:
        """The launch choices in force (p2_get_tuning)."""
        t = p2_tuning()
        _check(lib.p2_get_tuning(self.ctx, ctypes.byref(t)), "p2_get_tuning")
        return {"procrustes_split": t.procrustes_split, "subject_bins": t.subject_bins,
                "split_record_cap": t.split_record_cap, "m2_block_kib": t.m2_block_kib}

    def tuning_note(self) -> str:
        return lib.p2_tuning_note(self.ctx).decode(errors="replace")

    def set_tuning(self, **kw):
        """Change launch choices (p2_set_tuning); results do not change."""
        cur = self.tuning()
        cur.update(kw)
        t = p2_tuning(int(cur["procrustes_split"]), int(cur["subject_bins"]),
                      int(cur["split_record_cap"]), int(cur["m2_block_kib"]))
        _check(lib.p2_set_tuning(self.ctx, ctypes.byref(t)), "p2_set_tuning")

    def set_exchange(self, fn):
        """Make this context one shard of a subject-sharded collection (see
        shard.py and p2_set_exchange): fn(ptr, count, stream) must replace the
        device buffer of `count` doubles at ptr by its sum over all shards.
        Call before load()."""
        from .shard import _Hook
        hook = _Hook(fn)
        _check(lib.p2_set_exchange(self.ctx, ctypes.cast(hook.c_fn, ctypes.c_void_p), None),
               "p2_set_exchange")
        self._hook = hook                  # the C callback must outlive the context's use

    def stats(self) -> dict:
        return p2_stats(self.ctx)

    def device_bytes(self) -> int:
        return p2_device_bytes(self.ctx)
