"""Benchmark: PARAFAC2-ALS iterations (SPARTan formulation) on GB300.

One step = one full ALS iteration of Algorithm 2 (Q-step for every subject,
the three MTTKRPs of Algorithm 3, the H/V/W solves and the fit) over the
whole synthetic collection, replayed from a CUDA graph with the data
resident in HBM.  Prints one JSON line (rank 0).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--workload c63m]
  python bench.py --impl reference ...   # the FP64 CPU oracle on a bounded sample

Multi-GPU: the path has per-iteration reductions over all subjects, and no
run here uses more than one GPU, so N ranks run N independent replicas of
the workload (weak scaling); the only cross-rank step is the timing barrier.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

# the oracle's per-subject numpy work runs single-threaded; state it, do not vary it
os.environ.setdefault("OPENBLAS_NUM_THREADS", "1")
os.environ.setdefault("MKL_NUM_THREADS", "1")

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "PARAFAC2-ALS s/iter & nnz/s, 63M-500M nnz, R=10/40; HBM roofline fraction"
UNIT = "nnz/s"
FP64_PEAK_TFLOPS = 1.25        # GB300 FP64 (nominal; measured 1.19 with an FMA loop)
# The Procrustes step runs in double-word (float-float) arithmetic on the FP32
# pipe: 152 SMs x 128 FP32 lanes x 2.07 GHz = 40.3e12 FP32 instructions/s,
# and a double-word multiply-accumulate (product with its error terms, TwoSum,
# low-part update) is 12 of them, i.e. 2 flops per 12 instructions.
DW_INSTR_PER_FMA = 12
DW_PEAK_TFLOPS = 152 * 128 * 2.07e9 * 2 / DW_INSTR_PER_FMA / 1e12
PHASES = ("h_solve", "beta_mode2", "v_solve", "alpha_mode3_w_gram", "procrustes",
          "subject_stats_mode1", "fit")


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def _workload_desc(w, X):
    if w.planted_rank > 0:
        return (f"{w.name}: K={w.K:,} subjects, J={w.J:,}, planted PARAFAC2 X_k = Q_k H S_k V^T "
                f"(rank {w.planted_rank}, {w.dense_rows} dense rows) kept with p={w.keep_p:g}, "
                f"empty rows dropped (mean I_k {X.n_rows / max(X.K, 1):.1f}), R={w.R}, "
                f"nnz={X.nnz:,}")
    cols = "uniform" if w.col_mode == 0 else f"Zipf({w.zipf_s}) via seeded permutation"
    return (f"{w.name}: K={w.K:,} subjects, J={w.J:,}, I_k~U{{{w.imin}..{w.imax}}}, "
            f"Poisson({w.lam})+1 nnz/row, {cols} columns, values 1+Poisson(1), "
            f"R={w.R}, nnz={X.nnz:,}")


def _bytes_model(X, R):
    """Algorithmic HBM bytes per launch of each kernel group: the streamed
    format of X (u16 column + f32 value per non-zero, u16 row length, two
    int64 offsets per subject) plus the per-subject state each pass must read
    or write (T_k f32 R x R, packed Gram f64, W and M3 rows)."""
    K, N, nnz = X.K, X.n_rows, X.nnz
    P = R * (R + 1) // 2
    xb = 6 * nnz + 2 * N + 16 * (K + 1)          # u16 col + f32 val, u16 row length, 2 int64 offsets
    return {
        "beta_mode2": xb + K * (4 * R * R + 4 * R),
        "alpha_mode3_w_gram": xb + K * (4 * R * R + 8 * P + 8 * R),
        "procrustes": K * (8 * P + 4 * R + 4 * R * R),
        "subject_stats_mode1": K * (4 * R * R + 4 * P + 8 * R),
    }


class ClockSampler:
    """nvidia-smi clock/throttle samples during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id):
        self.gpu_id = str(gpu_id)
        self.proc = None
        self.path = None
        self.skip = 0

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(prefix="clocks_", suffix=".csv")
            os.close(fd)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "50", "-i", self.gpu_id], stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def _lines(self):
        try:
            with open(self.path) as f:
                return sum(1 for ln in f if ln.endswith("\n"))
        except OSError:
            return 0

    def mark_region_start(self, timeout=3.0):
        """Wait (bounded) for the sampler's first line, then remember how many
        lines precede the timed region so that only later samples count."""
        if self.proc is None:
            return
        t0 = time.time()
        while self._lines() == 0 and time.time() - t0 < timeout and self.proc.poll() is None:
            time.sleep(0.01)
        self.skip = self._lines()

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        sm, mx, reasons = [], [], set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        with open(self.path) as f:
            lines = [ln for ln in f if ln.endswith("\n")]
        # samples taken during the timed region; the last earlier one if none
        in_region = len(lines) > self.skip
        lines = lines[self.skip:] if in_region else lines[max(self.skip - 1, 0):self.skip]
        for line in lines:
            p = [x.strip() for x in line.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                mx.append(float(p[2]))
            except ValueError:
                continue
            for n, v in zip(names, p[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        os.unlink(self.path)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "samples": len(sm),
                "in_timed_region": in_region, "reasons": sorted(reasons)}


def _dist():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def max_over_ranks(x, dist, device="cpu"):
    """Largest value of x over all ranks (the slowest rank sets the job time)."""
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(nnz_per_rank, steps, ms_total_max, world):
    """Whole-job nnz/s: every rank processed its replica; time is the max over ranks."""
    return world * nnz_per_rank * steps / (ms_total_max / 1e3)


# sources that define each kernel whose DRAM traffic profiles/traffic.json records
TRAFFIC_SOURCES = {
    "k_polar_reg": ("p2_dw.cuh", "p2_num.cuh", "p2_eig_dw.cuh", "p2_polar.cu", "p2_polar.cuh"),
    "k_polar_split": ("p2_dw.cuh", "p2_num.cuh", "p2_polar.cu", "p2_polar.cuh",
                      "p2_polar_grp.cu", "p2_polar_grp.cuh", "p2_polar_grp_launch.cuh"),
    "k_polar_reg_split": ("p2_dw.cuh", "p2_num.cuh", "p2_eig_dw.cuh", "p2_polar.cu",
                          "p2_polar.cuh", "p2_polar_grp.cuh"),
}


def traffic_sources_sha1(kernel):
    """SHA-1 of the sources that define `kernel` (in a fixed order)."""
    h = hashlib.sha1()
    csrc = os.path.join(ROOT, "paper_1703_04219_gb300", "csrc")
    for name in TRAFFIC_SOURCES[kernel]:
        with open(os.path.join(csrc, name), "rb") as g:
            h.update(g.read())
    return h.hexdigest()


def _traffic(kernel, workload):
    """DRAM bytes per launch from the committed ncu summary, if the kernel's
    sources are the ones the counters were taken on."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as f:
            d = json.load(f)
        ent = d.get(workload, {}).get(kernel)
        if ent and ent.get("sources_sha1") == traffic_sources_sha1(kernel):
            return ent["dram_bytes_per_launch"]
    except Exception:
        pass
    return None


def prefix(X, n):
    """The first n subjects of X (array slices; no arithmetic)."""
    import synth
    r1 = int(X.subj_ptr[n])
    e1 = int(X.row_ptr[r1])
    return synth.Slices(int(n), X.J, X.subj_ptr[:n + 1].copy(), X.row_ptr[:r1 + 1].copy(),
                        X.col[:e1].copy(), X.val[:e1].copy())


def host_cores():
    return len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()


def _pooled_sample_time(X, n, H0, V0, W0, cores):
    """Seconds of one oracle iteration over the first n subjects, on `cores`
    worker processes (loading the workers is not timed)."""
    from oracle.pool import OraclePool
    Xs = prefix(X, n)
    with OraclePool(Xs, cores) as pool:
        t = time.perf_counter()
        pool.iteration(H0, V0, W0[:n])
        return time.perf_counter() - t, Xs.nnz, pool.n_workers


def cpu_baseline(w, X, H0, V0, W0, target_s=15.0):
    """The FP64 oracle, as it stands, on all host cores (one worker process per
    core over contiguous subject chunks, oracle.pool) on a bounded prefix of
    the same workload, sized for about target_s seconds of one iteration."""
    cores = host_cores()
    n_pilot = int(min(X.K, max(2000, 250 * cores)))
    dt, nnz, _ = _pooled_sample_time(X, n_pilot, H0, V0, W0, cores)
    n = int(min(X.K, max(n_pilot, n_pilot * target_s / max(dt, 1e-3))))
    dt, nnz, used = _pooled_sample_time(X, n, H0, V0, W0, cores)
    return {"value": nnz / dt, "unit": UNIT, "cores": used, "kind": "oracle",
            "host_cores": cores,
            "sample": f"first {n:,} subjects of {w.name} ({nnz:,} nnz), 1 iteration, "
                      f"{dt:.1f} s, numpy FP64, {used} worker processes (one per host core) "
                      f"over contiguous subject chunks"}


def run_reference(args, w):
    """--impl reference: the FP64 oracle on all host cores (oracle.pool), a
    bounded prefix of the workload per step."""
    world, rank, _ = _dist()
    if rank != 0:
        return 0
    import synth
    from oracle.pool import OraclePool
    X = synth.generate(w)
    H0, V0, W0 = synth.init_factors(w.R, X.J, X.K, seed=w.seed)
    cores = host_cores()
    # size the per-step sample so that (warmup + steps) steps take ~2 minutes
    n_pilot = int(min(X.K, max(2000, 250 * cores)))
    dt, _, _ = _pooled_sample_time(X, n_pilot, H0, V0, W0, cores)
    budget = 120.0 / max(args.steps + args.warmup, 1)
    n = int(min(X.K, max(n_pilot, n_pilot * budget / max(dt, 1e-3))))
    Xs = prefix(X, n)
    times = []
    with OraclePool(Xs, cores) as pool:
        H, V, Wk = (np.asarray(a, np.float64) for a in (H0, V0, W0[:n]))
        for i in range(args.warmup + args.steps):
            t = time.perf_counter()
            out = pool.iteration(H, V, Wk)
            dt = time.perf_counter() - t
            H, V, Wk = out["H"], out["V"], out["W"]
            if i >= args.warmup:
                times.append(dt)
        used = pool.n_workers
    step = statistics.mean(times)
    value = Xs.nnz / step
    sample = (f"first {n:,} subjects of {w.name} ({Xs.nnz:,} nnz) per step, numpy FP64, "
              f"{used} worker processes (one per host core) over contiguous subject chunks")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 0,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": step * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": _workload_desc(w, X), "sample_subjects": n,
                       "sample_nnz": int(Xs.nnz)},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": used, "kind": "oracle",
                             "host_cores": cores, "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def roofline(X, R, phase_ms, flops, wname, split=True):
    """Roofline of the dominant kernel group and the sparse passes' GB/s
    (split: whether the Procrustes step ran split into its three kernels)."""
    dom = max(phase_ms, key=phase_ms.get)
    bmodel = _bytes_model(X, R)
    hbm_peak, hbm_src = _peaks()
    if dom == "procrustes":
        ach = flops / (phase_ms[dom] / 1e3) / 1e12
        if R <= 12 and split:
            kname = ("split double-word Procrustes step: k_polar_reg<MODE 1> (M, Householder, "
                     "one lane per subject), k_qr_record (QR, one lane per subject), "
                     "k_polar_reg<MODE 2> (rotations applied, T_k)")
            tkey = "k_polar_reg_split"
        elif R <= 12:
            kname = "k_polar_reg (double-word Procrustes, one lane per subject)"
            tkey = "k_polar_reg"
        else:
            kname = ("split double-word Procrustes step: k_polar_grp<MODE 1> (Householder, a "
                     "group of 8 or 16 lanes per subject), k_qr_record (QR, one lane per "
                     "subject), k_polar_grp<MODE 2> (rotations applied, T_k)")
            tkey = "k_polar_split"
        roof = {"kernel": kname, "bound": "alu",
                "achieved": ach, "peak": DW_PEAK_TFLOPS, "unit": "TFLOP/s",
                "frac": ach / DW_PEAK_TFLOPS,
                "peak_source": "derived: FP32 pipe 152 SMs x 128 lanes x 2.07 GHz, "
                f"{DW_INSTR_PER_FMA} FP32 instructions per double-word multiply-add",
                "vs_fp64_nominal": ach / FP64_PEAK_TFLOPS,
                "algorithmic_flops_per_launch": flops,
                "traffic": _traffic(tkey, wname)}
    else:
        by = bmodel.get(dom, 0)
        ach = by / (phase_ms[dom] / 1e3) / 1e9
        roof = {"kernel": dom, "bound": "hbm", "achieved": ach, "peak": hbm_peak, "unit": "GB/s",
                "frac": ach / hbm_peak, "peak_source": hbm_src,
                "algorithmic_bytes_per_launch": by, "traffic": _traffic(dom, wname)}
    sparse = {}
    for k in ("beta_mode2", "alpha_mode3_w_gram"):
        gbs = bmodel[k] / (phase_ms[k] / 1e3) / 1e9 if phase_ms[k] > 0 else None
        sparse[k] = {"ms": phase_ms[k], "algorithmic_GBps": gbs,
                     "hbm_frac": gbs / hbm_peak if gbs else None}
    return roof, sparse


def tc_m_on(R, fp64_procrustes, tensor_core_m):
    """Whether the library forms the Procrustes step's M on the tensor cores
    (opt-in, 13 <= R <= 48)."""
    if fp64_procrustes or not 13 <= R <= 48:
        return False
    return bool(tensor_core_m)


def measure_workload(X, w, precision, steps, warmup, device, gpu_id, fp64_procrustes=False,
                     nonneg=False, tuning=None, tensor_core_m=None):
    """One workload timed like the headline (graph replays, CUDA events on the
    library's stream, phase events, clocks sampled in the timed region)."""
    import torch
    import paper_1703_04219_gb300 as p2
    R = w.R
    H0, V0, W0 = synth_init(w, X)
    stream = torch.cuda.Stream()
    m = p2.Parafac2(R, device=device, stream=stream.cuda_stream, timing=True,
                    precision=precision, fp64_procrustes=fp64_procrustes, nonneg=nonneg,
                    tensor_core_m=tensor_core_m)
    if tuning:
        m.set_tuning(**tuning)
    m.load(X)
    m.init(H0, V0, W0)
    for _ in range(warmup):
        m.iterate(1, want_fit=False)
    stream.synchronize()
    clocks = ClockSampler(gpu_id)
    t = timed_steps(m, stream, steps, None, clocks)
    fit, _ = m.fit()
    tune = m.tuning()
    m.close()
    ms = t["ms_total"] / steps
    roof, sparse = roofline(X, R, t["phase_ms"], t["flops"], w.name,
                            split=tune.get("procrustes_split") == 1)
    if tune.get("procrustes_split") == 0 and R > 12 and roof.get("bound") == "alu":
        roof["kernel"] = "k_polar_grp (fused double-word Procrustes, 8 or 16 lanes per subject)"
        roof["traffic"] = None
    if fp64_procrustes:
        roof = fp64_roofline(R, t["phase_ms"], t["flops"])
    return {"workload": _workload_desc(w, X), "precision": precision,
            "procrustes": "fp64" if fp64_procrustes else "double-word", "tuning": tune,
            "m_on_tensor_cores": tc_m_on(R, fp64_procrustes, tensor_core_m),
            "nonneg": bool(nonneg),
            "storage": "V and P_k bfloat16" if precision == "bf16" else "float",
            "steps": steps, "warmup": warmup, "s_per_iter": ms / 1e3,
            "value": X.nnz / (ms / 1e3), "unit": UNIT, "fit_after_steps": fit,
            "phase_ms": t["phase_ms"], "sparse_passes": sparse, "roofline": roof,
            "gpu_launches": t["launches"], "clocks": t["clocks"]}


def fp64_roofline(R, phase_ms, flops):
    """Roofline of the FP64 arm of the Procrustes step, against the FP64 pipe."""
    ach = flops / (phase_ms["procrustes"] / 1e3) / 1e12
    return {"kernel": ("k_polar_reg" if R <= 12 else "k_polar_grp") + " (FP64 arm)",
            "bound": "alu", "achieved": ach, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
            "frac": ach / FP64_PEAK_TFLOPS, "peak_source": "GB300 FP64 nominal",
            "algorithmic_flops_per_launch": flops, "traffic": None}


def synth_init(w, X):
    import synth
    return synth.init_factors(w.R, X.J, X.K, seed=w.seed)


def run_r40(args, device, gpu_id):
    """Table 1's R = 40 column: the 250M-non-zero workload in FP32 (split
    Procrustes step; for comparison M formed on the tensor cores, and the
    fused kernel), with bfloat16
    storage and with the FP64 arm of the Procrustes step, the
    555M-non-zero workload in FP32, and the paper's own configuration
    (planted 500M-non-zero workload, non-negative S_k and V)."""
    import synth
    out = {}
    steps = max(1, min(args.steps, 5))
    for name, precs in (("c250m", ("fp32", "tc", "fused", "bf16", "fp64p")), ("c555m", ("fp32",))):
        w = synth.WORKLOADS[name]
        X = synth.generate(w)
        for prec in precs:
            if prec == "fp64p" and args.no_fp64:
                continue
            key = {"fp64p": f"{name}_fp64_procrustes",
                   "tc": f"{name}_fp32_m_on_tensor_cores",
                   "fused": f"{name}_fp32_fused_procrustes"}.get(prec, f"{name}_{prec}")
            out[key] = measure_workload(X, w, prec if prec in ("fp32", "bf16") else "fp32",
                                        min(steps, 3) if prec == "fp64p" else steps,
                                        args.warmup, device, gpu_id,
                                        fp64_procrustes=prec == "fp64p",
                                        tuning={"procrustes_split": 0} if prec == "fused" else None,
                                        tensor_core_m=True if prec == "tc" else None)
        del X
    if not args.no_nonneg:
        # the paper's configuration: planted workload, non-negative S_k and V
        w = synth.WORKLOADS["p500m"]
        X = synth.generate(w)
        out["p500m_nonneg"] = measure_workload(X, w, "fp32", min(steps, 3), args.warmup, device,
                                               gpu_id, nonneg=True)
        del X
    return out


def _gpu_id(local):
    import torch
    props = torch.cuda.get_device_properties(local)
    gpu_id = getattr(props, "uuid", None)
    if gpu_id is None:
        return local
    return str(gpu_id) if str(gpu_id).startswith("GPU-") else f"GPU-{gpu_id}"


def run_p2(args, w):
    import torch
    world, rank, local = _dist()
    torch.cuda.set_device(local)
    pg = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
        pg = dist
    import synth
    import paper_1703_04219_gb300 as p2

    X = synth.generate(w)
    R = w.R
    H0, V0, W0 = synth.init_factors(R, X.J, X.K, seed=w.seed)
    stream = torch.cuda.Stream()
    m = p2.Parafac2(R, device=local, stream=stream.cuda_stream, timing=True,
                    tensor_core_m=args.tensor_core_m)
    if args.procrustes_split is not None:
        m.set_tuning(procrustes_split=args.procrustes_split)
    m.load(X)
    m.init(H0, V0, W0)
    for _ in range(args.warmup):
        m.iterate(1, want_fit=False)
    stream.synchronize()

    gpu_id = _gpu_id(local)
    clocks = ClockSampler(gpu_id)
    t = timed_steps(m, stream, args.steps, pg, clocks)
    ms_total, clk, launches = t["ms_total"], t["clocks"], t["launches"]
    phase_ms = t["phase_ms"]
    fit, loss = m.fit()
    if pg:
        ms_total = max_over_ranks(ms_total, pg, device="cuda")
    ms_step = ms_total / args.steps
    value = job_throughput(X.nnz, args.steps, ms_total, world)

    roof, sparse = roofline(X, R, phase_ms, t["flops"], w.name,
                            split=m.tuning()["procrustes_split"] == 1)

    # end-to-end through the public API from pinned host buffers
    e2e = None
    if not args.no_e2e:
        e2e = run_e2e(m, X, H0, V0, W0, args.e2e_steps, world, pg)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        cpu = cpu_baseline(w, X, H0, V0, W0)
    m.close()
    bf16 = None
    if not args.no_bf16:
        bf16 = time_precision(X, R, H0, V0, W0, "bf16", args.steps, args.warmup, local)
    fp64p = None
    if rank == 0 and world == 1 and not args.no_fp64:
        fp64p = measure_workload(X, w, "fp32", args.steps, args.warmup, local, gpu_id,
                                 fp64_procrustes=True)
    nonneg = None
    if not args.no_nonneg and R <= 16:
        nonneg = time_precision(X, R, H0, V0, W0, "fp32", args.steps, args.warmup, local,
                                nonneg=True)
    r40 = None
    if rank == 0 and world == 1 and not args.no_r40:
        r40 = run_r40(args, local, gpu_id)
    serving = None
    if rank == 0 and not args.no_serve:
        serving = {"fp32": run_serving(precision="fp32"), "bf16": run_serving(precision="bf16")}
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_step, "s_per_iter": ms_step / 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32 storage and SpMM (Gram: error-free f32 pairs), double-word (f32 pair) "
                     "Procrustes, f64 R x R solves", "data": "synthetic",
            "config": {"workload": _workload_desc(w, X), "K": X.K, "J": X.J, "R": R,
                       "nnz": int(X.nnz), "rows": int(X.n_rows),
                       "l2": "inputs larger than L2: X (~6 B/nnz) streamed twice per step",
                       "parallelism": f"replicas x{world}" if world > 1 else "single GPU",
                       "graph": True, "fit_after_steps": fit},
            "phase_ms": phase_ms, "sparse_passes": sparse, "roofline": roof,
            "gpu_launches": launches, "clocks": clk, "e2e": e2e, "cpu_baseline": cpu,
            "bf16_storage": bf16, "fp64_procrustes": fp64p, "nonneg": nonneg, "r40": r40,
            "serving": serving}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if pg:
        pg.destroy_process_group()
    return 0


def timed_steps(m, stream, steps, pg=None, clocks=None):
    """Time `steps` graph replays with CUDA events on the library's stream
    (barrier + synchronize on both sides).  After each step the phase events
    recorded inside the graph are read (p2_stats), so the per-kernel times are
    averages over the timed region."""
    import torch
    st0 = m.stats()
    phase_sum = {k: 0.0 for k in PHASES}
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    if clocks:
        clocks.start()
        clocks.mark_region_start()
    if pg:
        pg.barrier()
    torch.cuda.synchronize()
    ev0.record(stream)
    for _ in range(steps):
        m.iterate(1, want_fit=False)
        st = m.stats()                  # synchronises the stream; reads this step's phase events
        for k in PHASES:
            phase_sum[k] += st["phase_ms"].get(k, 0.0)
    ev1.record(stream)
    ev1.synchronize()
    torch.cuda.synchronize()
    if pg:
        pg.barrier()
    ms_total = ev0.elapsed_time(ev1)
    clk = clocks.stop() if clocks else None
    st1 = m.stats()
    return {"ms_total": ms_total, "phase_ms": {k: v / steps for k, v in phase_sum.items()},
            "launches": st1["kernel_launches"] - st0["kernel_launches"],
            "flops": (st1["polar_fp64_flops"] - st0["polar_fp64_flops"]) / steps, "clocks": clk}


def time_precision(X, R, H0, V0, W0, precision, steps, warmup, device, nonneg=False):
    """The same workload and timing with another storage precision, or in the
    non-negative variant (Section 5.1)."""
    import torch
    import paper_1703_04219_gb300 as p2
    stream = torch.cuda.Stream()
    m = p2.Parafac2(R, device=device, stream=stream.cuda_stream, timing=True, precision=precision,
                    nonneg=nonneg)
    m.load(X)
    m.init(H0, V0, W0)
    for _ in range(warmup):
        m.iterate(1, want_fit=False)
    stream.synchronize()
    t = timed_steps(m, stream, steps)
    fit, _ = m.fit()
    m.close()
    ms = t["ms_total"] / steps
    return {"ms_per_step": ms, "value": X.nnz / (ms / 1e3), "unit": UNIT,
            "fit_after_steps": fit, "phase_ms": t["phase_ms"],
            "storage": "V and P_k bfloat16" if precision == "bf16" else "float",
            "nonneg": bool(nonneg)}


def run_serving(rate=50000.0, horizon_s=2.0, n_iter=5, n_slots=4, seed=5, precision="fp32"):
    """Serving pattern: new subjects projected onto a fixed model (H 40x40,
    V 5000x40) by the continuous-batching server; Poisson arrivals at `rate`
    for `horizon_s` seconds.  The model comes from two ALS iterations on a
    20,000-subject slice of the 250M-nnz generator (R = 40)."""
    from dataclasses import replace
    import synth
    import paper_1703_04219_gb300 as p2
    from paper_1703_04219_gb300.serve import Server, requests_from_slices
    wt = synth.WORKLOADS["c250m"].scaled(20000)
    Xt = synth.generate(wt)
    R = wt.R
    H0, V0, W0 = synth.init_factors(R, Xt.J, Xt.K, seed=wt.seed)
    model = p2.Parafac2(R, precision=precision)
    model.load(Xt)
    model.init(H0, V0, W0)
    model.iterate(2)
    ws = synth.WORKLOADS["serve"]
    n_req = int(rate * horizon_s)
    req = synth.generate(replace(ws, K=n_req, seed=ws.seed))
    reqs = requests_from_slices(req, rate_per_s=rate, seed=seed)
    max_subjects = 4096
    # admission by device memory: 2% of the free device memory for the slots'
    # scratch, capacities from the requests' mean shape (rows, non-zeros per row)
    srv = Server(model, n_slots=n_slots, max_subjects=max_subjects, n_iter=n_iter,
                 memory_fraction=0.02,
                 shape=(float(req.n_rows / req.K), float(req.nnz / max(req.n_rows, 1))))
    warm = requests_from_slices(req.take(list(range(min(512, n_req)))), rate_per_s=1e9, seed=seed)
    srv.run(warm)                      # first launches, allocator
    _, st = srv.run(reqs)
    srv.close()
    model.close()
    st.update({"precision": precision, "rate_per_s": rate, "horizon_s": horizon_s,
               "n_iter": n_iter, "slots": n_slots,
               "R": R, "mean_rows": float(req.n_rows / req.K), "mean_nnz": float(req.nnz / req.K)})
    return st


def run_e2e(m, X, H0, V0, W0, steps, world, pg):
    """Per step: p2_load_slices from pinned host memory + p2_init + one iteration
    + the fit read back (device -> host)."""
    import torch
    import paper_1703_04219_gb300 as p2
    arrs = [X.subj_ptr, X.row_ptr, X.col, X.val]
    pinned = [torch.from_numpy(np.ascontiguousarray(a)).pin_memory() for a in arrs]
    fac = [torch.from_numpy(np.ascontiguousarray(a)).pin_memory() for a in (H0, V0, W0)]
    h2d = sum(t.numel() * t.element_size() for t in pinned + fac)
    times = []
    for i in range(steps + 1):
        torch.cuda.synchronize()
        if pg:
            pg.barrier()
        t = time.perf_counter()
        p2.p2_load_slices(m.ctx, X.K, X.J, *pinned, location=0)
        lib = p2.lib
        rc = lib.p2_init(m.ctx, p2._ptr(fac[0]), p2._ptr(fac[1]), p2._ptr(fac[2]))
        p2._check(rc, "p2_init")
        fit = m.iterate(1, want_fit=True)
        dt = time.perf_counter() - t
        if i > 0:                      # first one warms the allocator
            times.append(dt)
    step = statistics.mean(times)
    if pg:
        step = max_over_ranks(step, pg, device="cuda")
    return {"value": world * X.nnz / step, "unit": UNIT, "s_per_step": step,
            "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": 8,
            "step": "p2_load_slices (host, pinned) + p2_init + p2_iterate(1) + fit read-back",
            "fit": fit}


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="p2", choices=["p2", "reference"])
    ap.add_argument("--workload", default="c63m")
    ap.add_argument("--K", type=int, default=None, help="override the number of subjects")
    ap.add_argument("--e2e-steps", type=int, default=2)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-serve", action="store_true")
    ap.add_argument("--no-bf16", action="store_true")
    ap.add_argument("--no-nonneg", action="store_true", help="skip the non-negative variant line")
    ap.add_argument("--no-fp64", action="store_true",
                    help="skip the FP64 arm of the Procrustes step")
    ap.add_argument("--no-r40", action="store_true",
                    help="skip the R = 40 workloads (250M nnz FP32 and bfloat16, 555M nnz)")
    ap.add_argument("--tensor-core-m", choices=["auto", "on", "off"], default="auto",
                    help="form the Procrustes step's M on the tensor cores (auto: the "
                         "library's default, off)")
    ap.add_argument("--procrustes-split", choices=["auto", "on", "off"], default="auto",
                    help="headline workload: the Procrustes step split into its Householder, "
                         "QR-recording and rotation kernels, or fused (auto: the library's "
                         "default, on)")
    args = ap.parse_args(argv)
    args.tensor_core_m = {"auto": None, "on": True, "off": False}[args.tensor_core_m]
    args.procrustes_split = {"auto": None, "on": 1, "off": 0}[args.procrustes_split]
    if args.warmup < 3:
        args.warmup = 3
    import synth
    w = synth.WORKLOADS[args.workload]
    if args.K:
        w = w.scaled(args.K)
    if args.impl == "reference":
        return run_reference(args, w)
    return run_p2(args, w)


if __name__ == "__main__":
    sys.exit(main())
