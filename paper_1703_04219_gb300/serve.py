"""Continuous-batching projection server on top of ``p2_project``.

Requests are new subjects to project onto a fitted model (fixed H, V).  The
server keeps ``n_slots`` projectors, each with its own CUDA stream and pinned
staging buffers.  Requests that arrive while batches are on the GPU wait in a
FIFO queue and are admitted into the next batch as soon as a slot frees up,
as long as the batch fits the slot's memory (its capacities in subjects, rows
and non-zeros, sized from a device-memory budget with p2_projector_bytes, or
given); a request larger than a whole slot is rejected.  Slots run
concurrently on the device.  Completion is detected with CUDA events, so the
host loop never blocks on a running batch.

Every subject is computed independently of the others in its batch, so a
request's result does not depend on what it was batched with.
"""
from __future__ import annotations

import time
from dataclasses import dataclass, field

import numpy as np

from . import Projector


@dataclass
class Request:
    rid: int
    arrival: float                 # seconds since the start of the run
    row_ptr: np.ndarray            # int64 [I+1], rebased to 0
    col: np.ndarray                # int32
    val: np.ndarray                # float32

    @property
    def rows(self):
        return len(self.row_ptr) - 1

    @property
    def nnz(self):
        return int(self.row_ptr[-1])


@dataclass
class Slot:
    pj: Projector
    stream: object
    event: object
    sp: object
    rp: object
    col: object
    val: object
    S: object
    batch: list = field(default_factory=list)
    busy: bool = False


def requests_from_slices(slices, rate_per_s: float, seed: int = 0):
    """One request per subject, Poisson arrivals at ``rate_per_s``."""
    rng = np.random.default_rng(seed)
    gaps = rng.exponential(1.0 / rate_per_s, size=slices.K)
    t = np.cumsum(gaps)
    out = []
    for k in range(slices.K):
        rp, c, v = slices.subject(k)
        out.append(Request(k, float(t[k]), np.asarray(rp, np.int64), c, v))
    return out


def capacities_for_memory(model, slot_bytes, max_subjects, mean_rows, mean_nnz_per_row,
                          headroom=2.0):
    """Capacities (subjects, rows, non-zeros) of one slot whose projector
    takes at most slot_bytes of device memory (p2_projector_bytes), for
    requests of the given mean shape: rows and non-zeros sized for at least
    `headroom` times the mean (more if the budget allows), subjects capped at
    max_subjects and reduced until that headroom fits."""
    from . import p2_projector_bytes

    def need(s, f):
        rows = int(np.ceil(f * s * mean_rows))
        nnz = int(np.ceil(f * s * mean_rows * mean_nnz_per_row))
        return p2_projector_bytes(model, s, rows, nnz), rows, nnz

    s = int(max_subjects)
    while s > 1 and need(s, headroom)[0] > slot_bytes:
        s = max(1, s // 2)
    if need(s, headroom)[0] > slot_bytes:
        raise ValueError(f"slot memory {slot_bytes} B holds no request of the given shape")
    lo, hi = float(headroom), float(headroom)
    while need(s, hi * 2)[0] <= slot_bytes and hi < 1e6:      # largest scale that fits
        hi *= 2
    hi *= 2
    for _ in range(40):
        mid = (lo + hi) / 2
        if need(s, mid)[0] <= slot_bytes:
            lo = mid
        else:
            hi = mid
    b, rows, nnz = need(s, lo)
    return s, rows, nnz, b


class Server:
    """Continuous-batching server.  Capacities per slot either given
    (max_subjects, max_rows, max_nnz) or derived from a device-memory budget:
    memory_bytes for all slots' scratch, or memory_fraction of the device's
    free memory at start-up, with the request shape (mean rows per subject,
    mean non-zeros per row); max_subjects then caps a batch's subjects (a
    latency bound).  A request is admitted into a batch while the batch fits
    the slot's capacities, i.e. its memory."""

    def __init__(self, model, n_slots: int = 4, max_subjects: int = 256,
                 max_rows: int = 65536, max_nnz: int = 262144, n_iter: int = 10,
                 memory_bytes=None, memory_fraction=None, shape=(33.0, 3.0),
                 log_batches: bool = False):
        import torch
        self.torch = torch
        self.R = model.R
        self.n_iter = n_iter
        self.admission = None
        if memory_fraction is not None and memory_bytes is None:
            free, _ = torch.cuda.mem_get_info()
            memory_bytes = int(memory_fraction * free)
            self.admission = {"free_device_bytes": int(free), "memory_fraction": memory_fraction}
        if memory_bytes is not None:
            slot_bytes = int(memory_bytes) // n_slots
            max_subjects, max_rows, max_nnz, used = capacities_for_memory(
                model, slot_bytes, max_subjects, shape[0], shape[1])
            self.admission = dict(self.admission or {}, memory_bytes=int(memory_bytes),
                                  slot_bytes=slot_bytes, slot_projector_bytes=int(used),
                                  capacity={"subjects": max_subjects, "rows": max_rows,
                                            "nnz": max_nnz})
        self.cap = (max_subjects, max_rows, max_nnz)
        self.batch_log = [] if log_batches else None
        self.slots = []
        for _ in range(n_slots):
            st = torch.cuda.Stream()
            pj = Projector(model, max_subjects, max_rows, max_nnz, stream=st.cuda_stream)
            pin = lambda n, dt: torch.empty(n, dtype=dt).pin_memory()   # noqa: E731
            self.slots.append(Slot(pj, st, torch.cuda.Event(), pin(max_subjects + 1, torch.int64),
                                   pin(max_rows + 1, torch.int64), pin(max_nnz, torch.int32),
                                   pin(max_nnz, torch.float32),
                                   pin(max_subjects * self.R, torch.float32)))

    def close(self):
        for s in self.slots:
            s.pj.close()

    def _fits(self, n, rows, nnz, r: Request):
        return (n + 1 <= self.cap[0] and rows + r.rows <= self.cap[1]
                and nnz + r.nnz <= self.cap[2])

    def _launch(self, slot: Slot, batch):
        n = len(batch)
        sp = slot.sp.numpy()
        rp = slot.rp.numpy()
        col = slot.col.numpy()
        val = slot.val.numpy()
        sp[0] = 0
        rp[0] = 0
        row = nz = 0
        for i, r in enumerate(batch):
            rp[row + 1: row + r.rows + 1] = r.row_ptr[1:] + nz
            col[nz: nz + r.nnz] = r.col
            val[nz: nz + r.nnz] = r.val
            row += r.rows
            nz += r.nnz
            sp[i + 1] = row
        if self.batch_log is not None:
            self.batch_log.append((n, row, nz))
        slot.pj.submit(n, slot.sp, slot.rp, slot.col, slot.val, self.n_iter, slot.S)
        slot.event.record(slot.stream)
        slot.batch = batch
        slot.busy = True

    def run(self, requests, time_scale: float = 1.0):
        """Replay the requests in real time; returns results and latencies."""
        queue = []
        i = 0
        results = {}
        lat = {}
        rejected = []
        batches = []
        t0 = time.perf_counter()
        pending = sorted(requests, key=lambda r: r.arrival)
        n_total = len(pending)
        while len(results) + len(rejected) < n_total:
            now = (time.perf_counter() - t0) / time_scale
            while i < n_total and pending[i].arrival <= now:
                r = pending[i]
                if not self._fits(0, 0, 0, r):
                    rejected.append(r.rid)
                else:
                    queue.append(r)
                i += 1
            for slot in self.slots:
                if slot.busy and slot.event.query():
                    slot.pj.sync()
                    done = (time.perf_counter() - t0) / time_scale
                    S = slot.S.numpy()
                    for j, r in enumerate(slot.batch):
                        results[r.rid] = S[j * self.R:(j + 1) * self.R].copy()
                        lat[r.rid] = done - r.arrival
                    batches.append(len(slot.batch))
                    slot.busy = False
                if not slot.busy and queue:
                    batch, n, rows, nnz = [], 0, 0, 0
                    while queue and self._fits(n, rows, nnz, queue[0]):
                        r = queue.pop(0)
                        batch.append(r)
                        n, rows, nnz = n + 1, rows + r.rows, nnz + r.nnz
                    self._launch(slot, batch)
            if i < n_total and not queue and not any(s.busy for s in self.slots):
                wait = pending[i].arrival * time_scale - (time.perf_counter() - t0)
                if wait > 0:
                    time.sleep(min(wait, 1e-3))
        makespan = (time.perf_counter() - t0) / time_scale
        lats = np.array([lat[k] for k in sorted(lat)])
        stats = {
            "requests": n_total, "completed": len(results), "rejected": len(rejected),
            "p50_ms": float(np.percentile(lats, 50) * 1e3) if len(lats) else None,
            "p99_ms": float(np.percentile(lats, 99) * 1e3) if len(lats) else None,
            "subjects_per_s": len(results) / makespan if makespan > 0 else None,
            "batches": len(batches), "mean_batch": float(np.mean(batches)) if batches else 0.0,
            "makespan_s": makespan,
            "admission": self.admission or {"capacity": dict(zip(("subjects", "rows", "nnz"),
                                                                 self.cap))},
        }
        return results, stats
