"""Host logic: the seeded generator, the multi-rank bench aggregation (gloo) and
the bench's clock record."""
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


class _FakeSampler:
    def terminate(self):
        pass

    def wait(self, timeout=None):
        pass

    def poll(self):
        return None


def _bench_module():
    import importlib.util
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    spec = importlib.util.spec_from_file_location("bench_mod", os.path.join(root, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


@pytest.mark.parametrize("lines,skip,want", [
    # two samples inside the timed region: the idle one before it is ignored
    (["0, 1500, 2070, 300, 0x0, Not Active, Not Active, Not Active, Not Active",
      "0, 2070, 2070, 900, 0x4, Not Active, Not Active, Not Active, Active",
      "0, 2060, 2070, 950, 0x0, Not Active, Not Active, Not Active, Not Active"], 1,
     dict(sm_mhz=2065.0, samples=2, in_timed_region=True, reasons=["sw_power_cap"])),
    # none inside: the last earlier sample is reported, flagged as such
    (["0, 1500, 2070, 300, 0x0, Not Active, Not Active, Not Active, Not Active"], 1,
     dict(sm_mhz=1500.0, samples=1, in_timed_region=False, reasons=[])),
    # a thermal slowdown inside the region is reported
    (["0, 2070, 2070, 300, 0x0, Not Active, Not Active, Not Active, Not Active",
      "0, 1800, 2070, 1300, 0x20, Not Active, Active, Not Active, Not Active"], 1,
     dict(sm_mhz=1800.0, samples=1, in_timed_region=True, reasons=["hw_thermal_slowdown"])),
])
def test_clock_record_counts_only_samples_in_the_timed_region(tmp_path, lines, skip, want):
    """bench.py's clock record: nvidia-smi lines written before the timed
    region starts are skipped (unless no later line exists)."""
    bench = _bench_module()
    c = bench.ClockSampler(0)
    c.path = str(tmp_path / "clocks.csv")
    with open(c.path, "w") as f:
        f.write("\n".join(lines) + "\n")
    c.proc, c.fh, c.skip = _FakeSampler(), open(os.devnull, "w"), skip
    got = c.stop()
    for k, v in want.items():
        assert got[k] == v, (k, got)
