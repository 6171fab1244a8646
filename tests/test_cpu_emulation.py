"""The library's CUDA kernels run on the CPU emulator (tests/cpu_emu) under
AddressSanitizer: one ALS iteration at R = 5 and R = 10 (lane-per-subject
Procrustes; at R = 5 also from a start with two equal columns of V and W, whose
singular Gram-Hadamard products send the pseudo-inverses down their Jacobi
path), at R = 13 and R = 40 (grouped Procrustes, eight and sixteen lanes
per subject), at R = 20 (a rank outside the compiled list: generic kernels), at R = 10
and R = 40 with the FP64 arm of the Procrustes step, at R = 5 with bfloat16
storage and in the non-negative variant, a projection of new
subjects, U_k = Q_k H for a range of subjects, the seeded initialisation
with the stopping rule, the rational start (subspace iteration in FP64), and
the tensor-core formation of the Procrustes step's M (tcgen05 MMAs emulated
from the shared-memory descriptors).
Every device buffer and every block's shared memory is a heap block of its
exact size, so an out-of-bounds access by any kernel aborts the run; the
results must also match the FP64 oracle.  No GPU involved."""
import json
import os
import shutil
import subprocess
import sys

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
EMU = os.path.join(HERE, "cpu_emu")

CASES = {
    "iterate_r5": ["iterate", "tiny", "24", "5"],
    "iterate_r10": ["iterate", "tiny", "24", "10"],
    "iterate_r13": ["iterate", "tiny", "16", "13"],
    "iterate_r40": ["iterate", "tiny", "16", "40"],
    "iterate_r20": ["iterate", "c250m", "12", "20"],     # outside the rank-compiled list
    "iterate_r5_bf16": ["iterate", "tiny", "24", "5", "bf16"],
    "iterate_r5_nonneg": ["iterate", "tiny", "24", "5", "nonneg"],
    "iterate_r17_nonneg": ["iterate", "tiny", "24", "17", "nonneg"],
    "iterate_r10_fp64": ["iterate", "tiny", "24", "10", "fp64"],
    "iterate_r5_dupcols": ["iterate", "tiny", "24", "5", "dupcols"],
    "iterate_r40_fp64": ["iterate", "tiny", "16", "40", "fp64"],
    "project_r12": ["project", "12", "3"],
    "project_r8_nonneg": ["project", "8", "3", "nonneg"],
    "getu_r5": ["getu", "5", "3", "17"],
    "seed_r4": ["seed", "4", "987654321"],
    "rational_r3": ["rational", "3", "12"],
    "shard_r6": ["shard", "6", "20"],
    "split_r5": ["split", "5", "40"],
    "split_r10": ["split", "10", "24"],
    "split_r12": ["split", "12", "16"],
    "split_r13": ["split", "13", "12"],
    "split_r40": ["split", "40", "8"],
    "tc_r40": ["tc", "40", "8"],
    "tc_r13": ["tc", "13", "16"],
    "blocks_r6": ["blocks", "6", "40"],
}


def _asan_runtime():
    if shutil.which("g++") is None:
        return None
    r = subprocess.run(["g++", "-print-file-name=libasan.so"], capture_output=True, text=True)
    path = r.stdout.strip()
    return path if os.path.isabs(path) and os.path.exists(path) else None


@pytest.fixture(scope="module")
def emulated_runs():
    asan = _asan_runtime()
    if asan is None:
        pytest.skip("g++ with AddressSanitizer is not available")
    sys.path.insert(0, EMU)
    import build_emu
    build_emu.build()
    env = dict(os.environ, LD_PRELOAD=asan, EMU_NSM="1",
               ASAN_OPTIONS="detect_leaks=0:abort_on_error=1")
    procs = {name: subprocess.Popen([sys.executable, os.path.join(EMU, "run_case.py")] + args,
                                    env=env, stdout=subprocess.PIPE, stderr=subprocess.PIPE,
                                    text=True)
             for name, args in CASES.items()}
    out = {}
    for name, p in procs.items():
        try:
            so, se = p.communicate(timeout=900)
        except subprocess.TimeoutExpired:
            p.kill()
            so, se = p.communicate()
        out[name] = (p.returncode, so, se)
    return out


def _result(runs, name):
    rc, so, se = runs[name]
    assert rc == 0, f"{name} failed (rc {rc}):\n{se[-3000:]}"
    assert "AddressSanitizer" not in se, se[-3000:]
    return json.loads(so.strip().splitlines()[-1])


@pytest.mark.parametrize("name", ["iterate_r5", "iterate_r10", "iterate_r13", "iterate_r40",
                                  "iterate_r20", "iterate_r10_fp64", "iterate_r40_fp64",
                                  "iterate_r5_dupcols"])
def test_emulated_iteration_is_in_bounds_and_matches_oracle(emulated_runs, name):
    err = _result(emulated_runs, name)
    for key in ("M1", "M2", "M3", "H", "V", "W"):
        assert err[key] < 1e-5, (key, err[key])
    assert err["fit"] < 1e-4


def test_emulated_bf16_storage_is_in_bounds_and_within_3e3(emulated_runs):
    err = _result(emulated_runs, "iterate_r5_bf16")
    for key in ("M1", "M2", "M3", "H", "V", "W"):
        assert err[key] < 3e-3, (key, err[key])
    assert err["fit"] < 1e-4


@pytest.mark.parametrize("name", ["project_r12", "project_r8_nonneg"])
def test_emulated_projection_is_in_bounds_and_matches_oracle(emulated_runs, name):
    err = _result(emulated_runs, name)
    assert err["S_max"] < 1e-4


def test_emulated_get_U_is_in_bounds_and_matches_oracle(emulated_runs):
    err = _result(emulated_runs, "getu_r5")
    assert err["rows"] > 0
    assert err["U"] < 1e-5, err


def test_emulated_seeded_init_and_stopping_rule(emulated_runs):
    out = _result(emulated_runs, "seed_r4")
    assert out["init_equal"] == 1.0
    assert out["n"] == 3 and out["fit"] == out["fit_fixed"]
    assert out["n_loose"] == 2


@pytest.mark.parametrize("name", ["iterate_r5_nonneg", "iterate_r17_nonneg"])
def test_emulated_nonneg_iteration_is_in_bounds_and_matches_oracle(emulated_runs, name):
    """Section 5.1's non-negative variant: row-wise NNLS for V and W (one
    lane per row at R = 5, one warp per row at R = 17)."""
    err = _result(emulated_runs, name)
    assert err["neg"] == 0.0
    for key in ("M1", "M2", "M3", "H", "V", "W"):
        assert err[key] < 1e-5, (key, err[key])
    assert err["fit"] < 1e-4



def test_emulated_rational_start_is_in_bounds_and_matches_oracle(emulated_runs):
    """H = I, W = 1, V orthonormal and near the leading eigenvectors of
    sum_k X_k^T X_k after 12 products (the product in several column
    passes), the first iteration from that start against the oracle, and a
    rank-deficient input converging to an orthonormal completion."""
    out = _result(emulated_runs, "rational_r3")
    assert out["n"] == 12 and out["H_eye"] == 1.0 and out["W_one"] == 1.0
    assert out["orth"] < 1e-6 and out["sin2"] < 5e-4, out
    for key in ("H1", "V1", "W1"):
        assert out[key] < 1e-5, (key, out[key])
    assert out["fit"] < 1e-4
    assert 1 <= out["def_n"] < 50, out
    assert out["def_orth"] < 1e-6 and out["def_lead"] < 1e-6, out
    assert out["def_fit_finite"] == 1.0
    assert out["einval"] == 1.0 and out["still_iterates"] == 1.0


def test_emulated_sharded_context_is_in_bounds_and_matches(emulated_runs):
    """The subject-sharded code path (p2_set_exchange): a hook that doubles
    every exchanged buffer stands for two shards holding the same subjects,
    against one context on the collection stacked twice."""
    out = _result(emulated_runs, "shard_r6")
    assert out["calls_ok"] == 1.0, out
    for key in ("H", "V", "W", "M2"):
        assert out[key] < 1e-5, (key, out[key])
    assert out["fit"] < 1e-6


@pytest.mark.parametrize("name", ["split_r5", "split_r10", "split_r12", "split_r13", "split_r40"])
def test_emulated_split_procrustes_equals_fused(emulated_runs, name):
    """The split Procrustes step (Householder kernel, one-lane QR recorder,
    rotation-applying kernel) and its fused fallback give the fused kernel's
    results bit for bit, within bounds."""
    assert _result(emulated_runs, name)["bitwise"] == 1.0


@pytest.mark.parametrize("name", ["tc_r40", "tc_r13"])
def test_emulated_tensor_core_m(emulated_runs, name):
    """M of the Procrustes step formed on the (emulated) tensor cores: in
    bounds, the split step, the fused kernel and the fallback bitwise equal
    to each other, T_k close to the double-word formation's, and the factors
    within 1e-5 of the oracle."""
    out = _result(emulated_runs, name)
    assert out["tc_paths_bitwise"] == 1.0, out
    for path in ("tc", "tc_fused", "tc_fallback"):
        assert out[f"{path}_T0_vs_dw"] < 1e-4, out
        for f in ("W", "V", "H"):
            assert out[f"{path}_{f}"] < 1e-5, (path, f, out)


def test_emulated_mode2_row_blocks_are_in_bounds_and_match(emulated_runs):
    """The mode-2 pass over many row blocks (1 KiB of P rows each) against a
    single block and the oracle."""
    out = _result(emulated_runs, "blocks_r6")
    assert out["M2_blocks"] < 1e-12 and out["V_blocks"] < 1e-6, out
    assert out["M2"] < 1e-5 and out["V"] < 1e-5, out
    assert out["fit"] < 1e-9
