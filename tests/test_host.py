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


def test_plan_shards_balances_nonzeros_and_covers_every_subject():
    from paper_1703_04219_gb300 import shard
    X = synth.generate("c63m", K=5000)
    for n in (1, 2, 3, 7):
        cuts = shard.plan_shards(X.subj_ptr, X.row_ptr, n)
        assert cuts[0] == 0 and cuts[-1] == X.K and len(cuts) == n + 1
        assert all(a <= b for a, b in zip(cuts, cuts[1:]))
        nnz = [int(X.row_ptr[X.subj_ptr[b]] - X.row_ptr[X.subj_ptr[a]])
               for a, b in zip(cuts, cuts[1:])]
        assert sum(nnz) == X.nnz
        biggest = int(np.diff(X.row_ptr[X.subj_ptr]).max())     # one subject's non-zeros
        assert max(nnz) - min(nnz) <= 2 * biggest, (n, nnz)
    parts = shard.shards(X, 3)
    assert sum(p.K for p in parts) == X.K
    for p in parts:                                           # the ranges reassemble X
        k = p.k0
        assert np.array_equal(p.col, X.col[X.row_ptr[X.subj_ptr[k]]:
                                           X.row_ptr[X.subj_ptr[k + p.K]]])
        assert p.subj_ptr[0] == 0 and p.row_ptr[0] == 0 and p.row_ptr[-1] == len(p.col)
    tiny = shard.plan_shards(np.array([0, 2, 3]), np.arange(4), 4)   # more shards than subjects
    assert tiny[0] == 0 and tiny[-1] == 2 and len(tiny) == 5


def _shard_rank(rank, world, port, q):
    """One shard of the subject-sharded iteration, with the oracle's
    per-subject functions standing in for the library's kernels: the shard's
    partial M1, W^TW and M2 are summed with host_allreduce_ (gloo) exactly
    where a sharded context calls its exchange hook."""
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from oracle import parafac2 as P
    from paper_1703_04219_gb300 import shard
    X = synth.generate("tiny", K=120)
    R = 4
    H0, V0, W0 = (a.astype(np.float64) for a in synth.init_factors(R, X.J, X.K, seed=8))
    cuts = shard.plan_shards(X.subj_ptr, X.row_ptr, world)
    rng_ = shard.subject_range(X, cuts[rank], cuts[rank + 1])
    part = synth.Slices(rng_.K, rng_.J, rng_.subj_ptr, rng_.row_ptr, rng_.col, rng_.val)
    W = W0[cuts[rank]:cuts[rank + 1]]
    blocks = P.all_blocks(part)
    cols = [c for _, c in blocks]
    Ys = [P.form_y(P.procrustes_q(Xc, c, H0, V0, W[k]), Xc) for k, (Xc, c) in enumerate(blocks)]
    stats = np.concatenate([P.mttkrp_spartan(Ys, cols, H0, V0, W, 1).ravel(), (W.T @ W).ravel()])
    shard.host_allreduce_(stats)
    M1, WtW = stats[:R * R].reshape(R, R), stats[R * R:].reshape(R, R)
    H, _ = P.normalize_columns(M1 @ P.pinv_sym(WtW * (V0.T @ V0)))
    M2 = np.ascontiguousarray(P.mttkrp_spartan(Ys, cols, H, V0, W, 2))
    shard.host_allreduce_(M2)
    q.put((rank, M1, WtW, M2))
    dist.destroy_process_group()


def test_sharded_exchange_over_two_gloo_ranks():
    """Two ranks (gloo, CPU) each hold one nnz-balanced subject range; after
    the exchanges both hold the unsharded iteration's M1, W^TW and M2."""
    import multiprocessing as mp
    from oracle import parafac2 as P
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 30500 + (os.getpid() % 1000)
    ps = [ctx.Process(target=_shard_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    got = []
    import queue
    while len(got) < 2:
        try:
            got.append(q.get(timeout=5))
        except queue.Empty:
            assert all(p.is_alive() or p.exitcode == 0 for p in ps), [p.exitcode for p in ps]
    res = sorted(got, key=lambda t: t[0])
    for p in ps:
        p.join(timeout=60)
    assert all(p.exitcode == 0 for p in ps)
    X = synth.generate("tiny", K=120)
    H0, V0, W0 = (a.astype(np.float64) for a in synth.init_factors(4, X.J, X.K, seed=8))
    ref = P.als_iteration(P.all_blocks(X), H0, V0, W0)
    for _, M1, WtW, M2 in res:
        assert np.allclose(M1, ref["M1"], rtol=1e-12, atol=1e-12 * np.abs(ref["M1"]).max())
        assert np.allclose(WtW, W0.T @ W0, rtol=1e-12)
        assert np.allclose(M2, ref["M2"], rtol=1e-12, atol=1e-12 * np.abs(ref["M2"]).max())
    assert np.array_equal(res[0][3], res[1][3])           # every rank holds the same sum


@pytest.mark.parametrize("R,split,name_has,wname,traffic_key", [
    (10, True, "k_polar_reg<MODE 1>", "c63m", "k_polar_reg_split"),
    (10, False, "k_polar_reg (double-word", "c63m", "k_polar_reg"),
    (40, True, "k_polar_grp<MODE 1>", "c250m", "k_polar_split"),
])
def test_roofline_names_the_procrustes_kernels_that_ran(R, split, name_has, wname, traffic_key):
    """bench.py's roofline for a Procrustes-dominated step: the kernel group
    named after the split or fused form that ran, the achieved rate =
    algorithmic flops / phase time against the derived double-word peak, and
    DRAM traffic only from a profiles/traffic.json entry of that group whose
    sources hash matches (else null)."""
    import types
    bench = _bench_module()
    X = types.SimpleNamespace(K=1000, n_rows=50000, nnz=60000)
    phase = {"procrustes": 5.0, "beta_mode2": 1.0, "alpha_mode3_w_gram": 1.0,
             "subject_stats_mode1": 0.1, "h_solve": 0.1, "v_solve": 0.1, "fit": 0.1}
    flops = 1e10
    roof, sparse = bench.roofline(X, R, phase, flops, wname, split=split)
    assert name_has in roof["kernel"] and roof["bound"] == "alu"
    assert roof["achieved"] == pytest.approx(flops / 5e-3 / 1e12)
    assert roof["frac"] == pytest.approx(roof["achieved"] / bench.DW_PEAK_TFLOPS)
    assert roof["traffic"] == bench._traffic(traffic_key, wname)
    assert set(sparse) == {"beta_mode2", "alpha_mode3_w_gram"}
