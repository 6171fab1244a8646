"""Host logic: the seeded generator and the multi-rank bench aggregation (gloo)."""
import os

import numpy as np
import pytest

import synth


def test_generator_is_deterministic_and_follows_the_recipe():
    a = synth.generate("c63m", K=4000)
    b = synth.generate("c63m", K=4000)
    for x, y in ((a.subj_ptr, b.subj_ptr), (a.row_ptr, b.row_ptr), (a.col, b.col), (a.val, b.val)):
        assert np.array_equal(x, y)
    I = np.diff(a.subj_ptr)
    assert I.min() >= 1 and I.max() <= 100 and abs(I.mean() - 50.5) < 2.0
    per_row = np.diff(a.row_ptr)
    assert per_row.min() >= 1 and abs(per_row.mean() - 1.25) < 0.02
    for r in range(0, a.n_rows, 997):                          # distinct, sorted columns
        c = a.col[a.row_ptr[r]:a.row_ptr[r + 1]]
        assert np.all(np.diff(c) > 0)
    assert a.col.min() >= 0 and a.col.max() < a.J
    assert np.all(a.val >= 1) and np.all(a.val == np.round(a.val))
    counts = np.sort(np.bincount(a.col, minlength=a.J))[::-1]
    assert 0.12 < counts[0] / a.nnz < 0.19                      # Zipf(1.1) head over 5,000 ranks


def test_prefix_of_a_workload_is_the_smaller_workload():
    big = synth.generate("tiny", K=150)
    small = synth.generate("tiny", K=60)
    assert np.array_equal(big.subj_ptr[:61], small.subj_ptr)
    assert np.array_equal(big.col[:small.nnz], small.col)


def test_init_factors_exact_in_fp32():
    H, V, W = synth.init_factors(5, 30, 40, seed=9)
    for A in (H, V, W):
        assert A.dtype == np.float32 and A.min() >= 0 and A.max() < 1
        assert np.array_equal(A.astype(np.float64) * 2.0 ** 24, np.round(A.astype(np.float64) * 2.0 ** 24))


def _rank(rank, world, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    t = bench.max_over_ranks(10.0 + rank, dist)
    q.put((rank, t, bench.job_throughput(1000, 4, t, world)))
    dist.destroy_process_group()


def test_bench_aggregation_over_two_gloo_ranks():
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 29500 + (os.getpid() % 1000)
    ps = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    res = [q.get(timeout=120) for _ in ps]
    for p in ps:
        p.join(timeout=60)
    assert all(p.exitcode == 0 for p in ps)
    for rank, t, v in res:
        assert t == 11.0                                     # max over ranks
        assert abs(v - 2 * 1000 * 4 / 0.011) < 1e-6          # both replicas' work / slowest time
