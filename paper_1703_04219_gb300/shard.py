"""Subject-sharded PARAFAC2-ALS: contiguous subject ranges, one context each.

The subjects of Algorithm 2 are independent except for sums over all of them
(Algorithm 3's mode-1 and mode-2 MTTKRPs, W^TW and the loss terms), so a
collection can be split into contiguous subject ranges with balanced
non-zero counts, one library context per range.  Each context loads only its
own slices and calls an exchange hook (p2_set_exchange in include/p2.h) that
sums its partial results with the other shards'; H and V are then solved
identically on every shard, and each shard keeps the W rows of its subjects.

Exchanges provided here (each sums a device buffer of doubles in place):

* ``TorchExchange``: torch.distributed all_reduce on the device buffer,
  enqueued on the library's stream (NCCL: one process per GPU);
* ``HostExchange``: copy to the host, torch.distributed all_reduce of a CPU
  tensor (gloo, any transport that reduces host memory), copy back;
* ``LocalExchange``: several contexts in one process (for instance several
  shards on one GPU), each driven by its own host thread; the host sums the
  shards' buffers in shard order.

Argument marshalling only: every sum over subjects inside a shard runs in the
library's kernels; the hooks move and add the shards' partial sums.
"""
from __future__ import annotations

import ctypes
import threading
from dataclasses import dataclass

import numpy as np

EXCHANGE_FN = ctypes.CFUNCTYPE(ctypes.c_int, ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p,
                               ctypes.c_void_p)


@dataclass
class SubjectRange:
    """Subjects k0 .. k1-1 of a collection as CSR arrays (the layout
    p2_load_slices takes), offsets rebased to zero."""
    K: int
    J: int
    subj_ptr: np.ndarray
    row_ptr: np.ndarray
    col: np.ndarray
    val: np.ndarray
    k0: int = 0


def plan_shards(subj_ptr, row_ptr, n_shards):
    """Cut points k_0 = 0 < ... < k_n = K of n_shards contiguous subject
    ranges with nearly equal non-zero counts (a range may be empty when there
    are fewer subjects than shards)."""
    subj_ptr = np.asarray(subj_ptr, np.int64)
    row_ptr = np.asarray(row_ptr, np.int64)
    K = len(subj_ptr) - 1
    n = int(n_shards)
    if n < 1:
        raise ValueError("n_shards must be >= 1")
    nnz_at = row_ptr[subj_ptr]                         # non-zeros before subject k
    total = int(nnz_at[-1])
    cuts = [0]
    for i in range(1, n):
        k = int(np.searchsorted(nnz_at, total * i / n, side="left"))
        cuts.append(min(max(k, cuts[-1]), K))
    cuts.append(K)
    return cuts


def subject_range(X, k0, k1):
    """Subjects k0 .. k1-1 of X (any object with K, J, subj_ptr, row_ptr, col, val)."""
    sp = np.asarray(X.subj_ptr, np.int64)
    rp = np.asarray(X.row_ptr, np.int64)
    r0, r1 = int(sp[k0]), int(sp[k1])
    n0, n1 = int(rp[r0]), int(rp[r1])
    return SubjectRange(int(k1 - k0), int(X.J), np.ascontiguousarray(sp[k0:k1 + 1] - r0),
                        np.ascontiguousarray(rp[r0:r1 + 1] - n0),
                        np.ascontiguousarray(np.asarray(X.col)[n0:n1], dtype=np.int32),
                        np.ascontiguousarray(np.asarray(X.val)[n0:n1], dtype=np.float32), int(k0))


def shards(X, n_shards):
    """The n_shards SubjectRange pieces of X (plan_shards' cut points)."""
    cuts = plan_shards(X.subj_ptr, X.row_ptr, n_shards)
    return [subject_range(X, a, b) for a, b in zip(cuts[:-1], cuts[1:])]


def _device_tensor(ptr, count):
    """A float64 CUDA tensor viewing `count` doubles at device address ptr."""
    import torch

    class _View:
        pass

    v = _View()
    v.__cuda_array_interface__ = {"shape": (int(count),), "typestr": "<f8",
                                  "data": (int(ptr), False), "version": 2}
    return torch.as_tensor(v, device=torch.device("cuda", torch.cuda.current_device()))


def host_allreduce_(arr, group=None):
    """Sum a float64 host array in place over the ranks of a torch.distributed
    group (gloo or any backend that reduces CPU tensors)."""
    import torch
    import torch.distributed as dist
    t = torch.from_numpy(arr)
    dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
    return arr


class _Hook:
    """Wraps a Python exchange(ptr, count, stream) as the C callback; an
    exception becomes a non-zero return (the library call then fails with
    P2_EEXCHANGE) and is kept in .error."""

    def __init__(self, fn):
        self.fn = fn
        self.error = None

        def cb(buf, count, stream, user):
            try:
                fn(int(buf or 0), int(count), int(stream or 0))
                return 0
            except BaseException as e:   # noqa: BLE001 - reported through the return code
                self.error = e
                return 1

        self.c_fn = EXCHANGE_FN(cb)


class TorchExchange:
    """all_reduce(SUM) of the device buffer over a torch.distributed group,
    enqueued on the library's stream (so the library's later kernels on that
    stream see the sum)."""

    def __init__(self, group=None):
        self.group = group

    def __call__(self, ptr, count, stream):
        import torch
        import torch.distributed as dist
        t = _device_tensor(ptr, count)
        with torch.cuda.stream(torch.cuda.ExternalStream(stream)):
            dist.all_reduce(t, op=dist.ReduceOp.SUM, group=self.group)


class HostExchange:
    """The device buffer through the host: synchronise the library's stream,
    copy to the host, host_allreduce_, copy back on that stream."""

    def __init__(self, group=None):
        self.group = group

    def __call__(self, ptr, count, stream):
        import torch
        s = torch.cuda.ExternalStream(stream)
        t = _device_tensor(ptr, count)
        s.synchronize()
        host = t.cpu().numpy().copy()
        host_allreduce_(host, self.group)
        with torch.cuda.stream(s):
            t.copy_(torch.from_numpy(host))
        s.synchronize()


class LocalExchange:
    """n shards in one process, each context driven by its own host thread:
    exchange i deposits shard i's buffer, waits for the others, and every
    shard receives the same sum, added on the host in shard order."""

    def __init__(self, n):
        self.n = int(n)
        self.parts = [None] * self.n
        self.barrier = threading.Barrier(self.n)
        self.timeout = 600.0

    def hook(self, i):
        def fn(ptr, count, stream):
            import torch
            s = torch.cuda.ExternalStream(stream)
            t = _device_tensor(ptr, count)
            s.synchronize()
            self.parts[i] = t.cpu().numpy().copy()
            self.barrier.wait(self.timeout)
            total = self.parts[0].copy()
            for p in self.parts[1:]:
                total += p
            self.barrier.wait(self.timeout)       # every shard has read the parts
            with torch.cuda.stream(s):
                t.copy_(torch.from_numpy(total))
            s.synchronize()
        return fn

    def abort(self):
        self.barrier.abort()
