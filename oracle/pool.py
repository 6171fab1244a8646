"""Algorithm 2's iteration over subject chunks in worker processes.

TEST INFRASTRUCTURE ONLY, like the rest of this package: only ``tests/`` and
``bench.py``'s CPU-baseline / reference arm may use it.

The per-subject oracle functions of ``parafac2.py`` are run unchanged, each
worker process holding one contiguous range of subjects: the Q-step
(``procrustes_q``), Y_k (``form_y``), Algorithm 3's MTTKRPs restricted to the
worker's subjects (``mttkrp_spartan``) and the surrogate loss terms
(``surrogate_loss``).  The parent sums the workers' partial M1, W^TW, M2 and
loss in chunk order (a fixed order, so a run is reproducible) and performs
Algorithm 1's solves exactly as ``parafac2.cp_als_sweep`` does, with the same
functions (``pinv_sym``, ``normalize_columns``, ``nnls_rows``).  Summing
per-chunk partials reorders the FP64 additions and nothing else; a CPU test
checks the result against ``parafac2.als_iteration`` to ~1e-13.

Workers are started with the ``spawn`` method, so the pool may be created in
a process that already initialised CUDA.  Each worker runs numpy with one
BLAS thread.
"""
from __future__ import annotations

import multiprocessing as mp
import os

import numpy as np

from . import parafac2 as P


class _Chunk:
    """A contiguous range of subjects as CSR arrays (the layout of synth.Slices)."""

    def __init__(self, J, subj_ptr, row_ptr, col, val):
        self.K = len(subj_ptr) - 1
        self.J = J
        self.subj_ptr = subj_ptr
        self.row_ptr = row_ptr
        self.col = col
        self.val = val

    def subject(self, k):
        r0, r1 = int(self.subj_ptr[k]), int(self.subj_ptr[k + 1])
        rp = self.row_ptr[r0:r1 + 1]
        b, e = int(rp[0]), int(rp[-1])
        return rp - b, self.col[b:e], self.val[b:e]


def _cut(X, a, b):
    """Subjects a .. b-1 of X as a _Chunk (array slices, rebased to zero)."""
    r0, r1 = int(X.subj_ptr[a]), int(X.subj_ptr[b])
    n0, n1 = int(X.row_ptr[r0]), int(X.row_ptr[r1])
    return _Chunk(X.J, np.ascontiguousarray(X.subj_ptr[a:b + 1] - r0),
                  np.ascontiguousarray(X.row_ptr[r0:r1 + 1] - n0),
                  np.ascontiguousarray(X.col[n0:n1]), np.ascontiguousarray(X.val[n0:n1]))


def _worker(conn):
    blocks = colsets = Ys = None
    Wc = H = V = None
    while True:
        msg = conn.recv()
        op = msg[0]
        if op == "load":
            chunk = msg[1]
            blocks = P.all_blocks(chunk)
            colsets = [cols for _, cols in blocks]
            conn.send(P.norm_x_sq(blocks))
        elif op == "qstep":                       # Algorithm 2: Q-step and Y for (H, V, W)
            _, H, V, Wc, rtol = msg
            Qs = [P.procrustes_q(Xc, cols, H, V, Wc[k], rtol) for k, (Xc, cols) in
                  enumerate(blocks)]
            Ys = [P.form_y(Qs[k], blocks[k][0]) for k in range(len(blocks))]
            conn.send((P.mttkrp_spartan(Ys, colsets, H, V, Wc, 1), Wc.T @ Wc))
        elif op == "mode2":
            H = msg[1]
            conn.send(P.mttkrp_spartan(Ys, colsets, H, V, Wc, 2))
        elif op == "mode3":
            V = msg[1]
            conn.send(P.mttkrp_spartan(Ys, colsets, H, V, Wc, 3))
        elif op == "loss":
            Wc = msg[1]
            conn.send(P.surrogate_loss(blocks, Ys, H, V, Wc))
        elif op == "stop":
            conn.close()
            return


class OraclePool:
    """Worker processes holding contiguous subject ranges of X (balanced by
    non-zeros); ``iteration`` runs one ALS iteration of Algorithm 2."""

    def __init__(self, X, n_workers=None):
        if n_workers is None:
            n_workers = os.cpu_count() or 1
        n_workers = int(max(1, min(n_workers, X.K)))
        # chunk boundaries at equal shares of the non-zeros
        nnz_at = X.row_ptr[X.subj_ptr]
        targets = np.linspace(0, int(nnz_at[-1]), n_workers + 1)
        cuts = np.searchsorted(nnz_at, targets[1:-1], side="left")
        self.bounds = [0] + [int(c) for c in cuts] + [X.K]
        self.bounds = sorted(set(self.bounds))
        self.K, self.J = X.K, X.J
        ctx = mp.get_context("spawn")
        saved = {k: os.environ.get(k) for k in ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS",
                                                 "MKL_NUM_THREADS")}
        for k in saved:
            os.environ[k] = "1"
        self.conns, self.procs = [], []
        try:
            for _ in range(len(self.bounds) - 1):
                a, b = ctx.Pipe()
                p = ctx.Process(target=_worker, args=(b,), daemon=True)
                p.start()
                self.conns.append(a)
                self.procs.append(p)
        finally:
            for k, v in saved.items():
                if v is None:
                    os.environ.pop(k, None)
                else:
                    os.environ[k] = v
        for c, (a, b) in zip(self.conns, zip(self.bounds[:-1], self.bounds[1:])):
            c.send(("load", _cut(X, a, b)))
        self.norm_x_sq = float(sum(c.recv() for c in self.conns))   # chunk order

    @property
    def n_workers(self):
        return len(self.conns)

    def _all(self, msgs):
        for c, m in zip(self.conns, msgs):
            c.send(m)
        return [c.recv() for c in self.conns]

    def iteration(self, H, V, W, rank_rtol=P.RANK_RTOL, nonneg=False):
        """One pass of Algorithm 2's loop body from (H, V, W), as
        parafac2.als_iteration: returns H, V, W, M1, M2, M3 and the loss."""
        H = np.asarray(H, np.float64)
        V = np.asarray(V, np.float64)
        W = np.asarray(W, np.float64)
        Wcs = [W[a:b] for a, b in zip(self.bounds[:-1], self.bounds[1:])]
        parts = self._all([("qstep", H, V, Wc, rank_rtol) for Wc in Wcs])
        M1 = sum(p[0] for p in parts)
        WtW = sum(p[1] for p in parts)
        # Algorithm 1's solves in parafac2.cp_als_sweep's order and form
        H = M1 @ P.pinv_sym(WtW * (V.T @ V))
        H, _ = P.normalize_columns(H)
        M2 = sum(self._all([("mode2", H)] * self.n_workers))
        A2 = WtW * (H.T @ H)
        V = P.nnls_rows(M2, A2) if nonneg else M2 @ P.pinv_sym(A2)
        V, _ = P.normalize_columns(V)
        M3 = np.concatenate(self._all([("mode3", V)] * self.n_workers), axis=0)
        A3 = (V.T @ V) * (H.T @ H)
        W = P.nnls_rows(M3, A3) if nonneg else M3 @ P.pinv_sym(A3)
        Wn = [W[a:b] for a, b in zip(self.bounds[:-1], self.bounds[1:])]
        loss = float(sum(self._all([("loss", Wc) for Wc in Wn])))
        return dict(H=H, V=V, W=W, M1=M1, M2=M2, M3=M3, loss=loss)

    def parafac2_als(self, H0, V0, W0, n_iter, rank_rtol=P.RANK_RTOL, nonneg=False):
        """n_iter iterations from (H0, V0, W0); the per-iteration fit history."""
        H, V, W = H0, V0, W0
        hist, last = [], None
        for _ in range(n_iter):
            last = self.iteration(H, V, W, rank_rtol, nonneg)
            H, V, W = last["H"], last["V"], last["W"]
            hist.append(dict(loss=last["loss"],
                             fit=P.fit_from_loss(last["loss"], self.norm_x_sq)))
        return dict(H=H, V=V, W=W, history=hist, last=last, norm_x_sq=self.norm_x_sq)

    def close(self):
        for c in self.conns:
            try:
                c.send(("stop",))
            except (BrokenPipeError, OSError):
                pass
        for p in self.procs:
            p.join(timeout=10)
            if p.is_alive():
                p.kill()
        self.conns, self.procs = [], []

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
