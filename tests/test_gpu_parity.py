"""GPU path (through the C ABI) against the FP64 oracle on the same seeded inputs.

Tolerances: factors and MTTKRPs within relative Frobenius 1e-5 of the FP64
oracle for the FP32 path, fit within 1e-4 after a fixed number of
iterations.  The one-step tests start both sides from the same FP32-exact
state, so they isolate kernel error from ALS trajectory divergence.
"""
import numpy as np
import pytest

import synth
from oracle import parafac2 as P
from tests.helpers import rel_fro, slices_from_dense

pytestmark = pytest.mark.gpu

TOL = 1e-5
FIT_TOL = 1e-4


@pytest.fixture(scope="module")
def p2():
    import paper_1703_04219_gb300 as mod
    return mod


def _one_step(p2, X, R, seed, **kw):
    H0, V0, W0 = synth.init_factors(R, X.J, X.K, seed=seed)
    with p2.Parafac2(R, **kw) as m:
        m.load(X)
        m.init(H0, V0, W0)
        fit = m.iterate(1)
        H, V, W = m.factors()
        M = {n: m.mttkrp(n) for n in (1, 2, 3)}
    blocks = P.all_blocks(X)
    ref = P.als_iteration(blocks, H0.astype(np.float64), V0.astype(np.float64),
                          W0.astype(np.float64))
    nx2 = P.norm_x_sq(blocks)
    return dict(fit=fit, H=H, V=V, W=W, M=M, ref=ref, ref_fit=P.fit_from_loss(ref["loss"], nx2))


@pytest.mark.parametrize("name,K,R", [("tiny", 200, 5), ("tiny", 200, 1), ("tiny", 97, 8),
                                      ("c63m", 3000, 10), ("c250m", 400, 40),
                                      ("tiny", 150, 13), ("tiny", 120, 16), ("c250m", 300, 24),
                                      ("tiny", 60, 64), ("c555m", 150, 40),
                                      # ranks outside the compiled list: the generic kernels
                                      ("c250m", 300, 20), ("c250m", 200, 33)])
def test_one_step_parity(p2, name, K, R):
    X = synth.generate(name, K=K)
    out = _one_step(p2, X, R, seed=11)
    ref = out["ref"]
    for mode, key in ((1, "M1"), (2, "M2"), (3, "M3")):
        assert rel_fro(out["M"][mode], ref[key]) < TOL, (key, rel_fro(out["M"][mode], ref[key]))
    for key in ("H", "V", "W"):
        assert rel_fro(out[key], ref[key]) < TOL, (key, rel_fro(out[key], ref[key]))
    assert abs(out["fit"] - out["ref_fit"]) < FIT_TOL


@pytest.mark.parametrize("name,K,R", [("tiny", 200, 5), ("c63m", 3000, 10), ("c250m", 400, 40),
                                      ("c250m", 300, 20), ("tiny", 150, 13)])
def test_fp64_procrustes_one_step_parity(p2, name, K, R):
    """The opt-in FP64 arm of the Procrustes step (p2_options.fp64_procrustes:
    the same Householder + QR eigen-decomposition and T_k formation in FP64 on
    the FP64 pipe) against the oracle, at the FP32 tolerances."""
    X = synth.generate(name, K=K)
    out = _one_step(p2, X, R, seed=11, fp64_procrustes=True)
    ref = out["ref"]
    for mode, key in ((1, "M1"), (2, "M2"), (3, "M3")):
        assert rel_fro(out["M"][mode], ref[key]) < TOL, (key, rel_fro(out["M"][mode], ref[key]))
    for key in ("H", "V", "W"):
        assert rel_fro(out[key], ref[key]) < TOL, (key, rel_fro(out[key], ref[key]))
    assert abs(out["fit"] - out["ref_fit"]) < FIT_TOL


def test_tiny_ten_iterations(p2):
    """The tiny workload (K=200, J=100, R=5), 10 iterations from the same start."""
    X = synth.generate("tiny")
    R = 5
    H0, V0, W0 = synth.init_factors(R, X.J, X.K, seed=20170314)
    with p2.Parafac2(R) as m:
        m.load(X)
        m.init(H0, V0, W0)
        fits = [m.iterate(1) for _ in range(10)]
        H, V, W = m.factors()
    ref = P.parafac2_als(X, H0, V0, W0, n_iter=10)
    ref_fits = [h["fit"] for h in ref["history"]]
    assert max(abs(a - b) for a, b in zip(fits, ref_fits)) < FIT_TOL
    for key, got in (("H", H), ("V", V), ("W", W)):
        assert rel_fro(got, ref[key]) < 1e-4, (key, rel_fro(got, ref[key]))


def test_graph_and_eager_agree_bitwise(p2):
    X = synth.generate("c63m", K=1500)
    R = 10
    H0, V0, W0 = synth.init_factors(R, X.J, X.K, seed=3)
    outs = []
    for graph in (True, False, True):
        with p2.Parafac2(R, use_graph=graph) as m:
            m.load(X)
            m.init(H0, V0, W0)
            m.iterate(3)
            outs.append(m.factors())
    for a, b in zip(outs[0], outs[1]):
        assert np.array_equal(a, b)
    for a, b in zip(outs[0], outs[2]):
        assert np.array_equal(a, b)


def test_edge_cases_empty_rows_and_small_subjects(p2):
    rng = np.random.default_rng(0)
    J, R = 12, 4
    mats = []
    for k in range(30):
        I = int(rng.integers(1, 7))
        m = rng.random((I, J)) * (rng.random((I, J)) < 0.4)
        if k % 5 == 0:
            m[0, :] = 0.0                      # an empty row
        if k % 7 == 0:
            m = np.vstack([m, 2.0 * m[:1]])    # proportional rows: rank deficient
        mats.append(m)
    X = slices_from_dense(mats, J)
    out = _one_step(p2, X, R, seed=5)
    ref = out["ref"]
    for key in ("H", "V", "W"):
        assert rel_fro(out[key], ref[key]) < TOL, (key, rel_fro(out[key], ref[key]))


def test_invalid_input_rejected(p2):
    X = synth.generate("tiny", K=10)
    with p2.Parafac2(3) as m:
        bad = X.col.copy()
        bad[0] = X.J + 5
        with pytest.raises(p2.P2Error) as ei:
            p2.p2_load_slices(m.ctx, X.K, X.J, X.subj_ptr, X.row_ptr, bad, X.val)
        assert ei.value.code == p2.P2_EINVAL
        badv = X.val.copy()
        badv[3] = np.nan
        with pytest.raises(p2.P2Error):
            p2.p2_load_slices(m.ctx, X.K, X.J, X.subj_ptr, X.row_ptr, X.col, badv)
        with pytest.raises(p2.P2Error) as ei:
            p2.p2_iterate(m.ctx, 1)
        assert ei.value.code == p2.P2_ESTATE


def test_stats_and_phase_timing(p2):
    """p2_stats: phase events inside the captured graph, launch and FP64 counters."""
    X = synth.generate("c63m", K=800)
    R = 10
    H0, V0, W0 = synth.init_factors(R, X.J, X.K, seed=2)
    with p2.Parafac2(R, timing=True) as m:
        m.load(X)
        m.init(H0, V0, W0)
        s0 = m.stats()
        m.iterate(2, want_fit=False)
        s1 = m.stats()
    assert s1["iterations"] == 2
    assert s1["kernel_launches"] > s0["kernel_launches"]
    assert set(s1["phase_ms"]) == set(p2.PHASES)
    assert all(v > 0 for v in s1["phase_ms"].values()), s1["phase_ms"]
    assert s1["polar_fp64_flops"] > s0["polar_fp64_flops"] > 0


@pytest.mark.parametrize("name,K,R", [("tiny", 200, 5), ("c63m", 2000, 10), ("c250m", 300, 40)])
def test_get_U_matches_oracle(p2, name, K, R):
    """U_k = Q_k H (Algorithm 2's ENSURE output) for a range of subjects, with
    Q_k the oracle's Procrustes factor (Section 3.2) for the factors the
    library returns.  Q_k is formed from the FP32 T_k, whose rounding is
    amplified by cond(A_k): each subject is held to max(1e-5, 8 eps32 cond)."""
    X = synth.generate(name, K=K)
    H0, V0, W0 = synth.init_factors(R, X.J, X.K, seed=5)
    with p2.Parafac2(R) as m:
        m.load(X)
        m.init(H0, V0, W0)
        m.iterate(2)
        H, V, W = m.factors()
        k0, k1 = K // 3, min(K, K // 3 + 40)
        U = m.U(k0, k1)
        assert m.U().shape == (X.n_rows, R)
        assert m.U(k1, k1).shape == (0, R)
    H, V, W = (a.astype(np.float64) for a in (H, V, W))
    eps32 = 2.0 ** -24
    row = 0
    for k in range(k0, k1):
        Xc, cols = P.subject_block(X, k)
        n = Xc.shape[0]
        got = U[row:row + n]
        row += n
        ref = P.assemble_u([P.procrustes_q(Xc, cols, H, V, W[k])], H)[0]
        if n == 0 or not np.any(ref):
            assert np.all(got == 0) if n else True
            continue
        A = (Xc @ V[cols]) * W[k] @ H.T
        sv = np.linalg.svd(A, compute_uv=False)
        sv = sv[sv > 1e-5 * sv[0]]
        bound = max(1e-5, 8 * eps32 * sv[0] / sv[-1])
        assert rel_fro(got, ref) < bound, (k, rel_fro(got, ref), bound)
    assert row == U.shape[0]


def test_seeded_init_and_stopping_rule(p2):
    """p2_init without factors draws the same H, V, W as the input generator
    for the context's seed; p2_iterate_until stops on the fit change and its
    fit equals that of a fixed-count run of the same length (bitwise: the
    iteration is deterministic)."""
    X = synth.generate("c63m", K=2000)
    with p2.Parafac2(10, seed=123) as m:
        m.load(X)
        m.init()
        H, V, W = m.factors()
        n, fit = m.iterate_until(60, 1e-6)
    H0, V0, W0 = synth.init_factors(10, X.J, X.K, seed=123)
    assert np.array_equal(H, H0) and np.array_equal(V, V0) and np.array_equal(W, W0)
    assert 2 <= n <= 60
    with p2.Parafac2(10) as m:
        m.load(X)
        m.init(H0, V0, W0)
        assert m.iterate(n) == fit


@pytest.mark.parametrize("name,K,R", [("tiny", 200, 5), ("c63m", 3000, 10), ("c63m", 1500, 16),
                                      ("ptiny", 50, 5), ("p63m", 2000, 10),
                                      # one warp per row above R = 16
                                      ("c250m", 400, 24), ("c250m", 400, 40), ("p500m", 300, 40),
                                      ("tiny", 120, 64)])
def test_nonneg_one_step_parity(p2, name, K, R):
    """Section 5.1's variant (non-negative S_k and V): one iteration from the
    same FP32-exact start against the oracle's Lawson-Hanson solves, with the
    lane-per-row NNLS kernel (R <= 16) and the warp-per-row one (R > 16)."""
    X = synth.generate(name, K=K)
    H0, V0, W0 = synth.init_factors(R, X.J, X.K, seed=3)
    with p2.Parafac2(R, nonneg=True) as m:
        m.load(X)
        m.init(H0, V0, W0)
        fit = m.iterate(1)
        H, V, W = m.factors()
        M = {n: m.mttkrp(n) for n in (1, 2, 3)}
    blocks = P.all_blocks(X)
    ref = P.als_iteration(blocks, H0.astype(np.float64), V0.astype(np.float64),
                          W0.astype(np.float64), nonneg=True)
    assert np.all(V >= 0) and np.all(W >= 0)
    for mode, key in ((1, "M1"), (2, "M2"), (3, "M3")):
        assert rel_fro(M[mode], ref[key]) < TOL, (key, rel_fro(M[mode], ref[key]))
    for key, v in (("H", H), ("V", V), ("W", W)):
        assert rel_fro(v, ref[key]) < TOL, (key, rel_fro(v, ref[key]))
    assert abs(fit - P.fit_from_loss(ref["loss"], P.norm_x_sq(blocks))) < FIT_TOL


def test_nonneg_ten_iterations_and_limits(p2):
    X = synth.generate("tiny", K=200)
    R = 5
    H0, V0, W0 = synth.init_factors(R, X.J, X.K, seed=4)
    with p2.Parafac2(R, nonneg=True) as m:
        m.load(X)
        m.init(H0, V0, W0)
        fit = m.iterate(10)
        _, V, W = m.factors()
    ref = P.parafac2_als(X, H0, V0, W0, n_iter=10, nonneg=True)
    assert abs(fit - ref["history"][-1]["fit"]) < FIT_TOL
    assert np.all(V >= 0) and np.all(W >= 0)
    with pytest.raises(p2.P2Error):
        p2.Parafac2(65, nonneg=True)


def test_nonneg_ten_iterations_r40(p2):
    """Ten non-negative iterations at R = 40 (warp-per-row NNLS, warm-started
    passive sets carried across iterations) against the oracle's fits."""
    X = synth.generate("c250m", K=300)
    R = 40
    H0, V0, W0 = synth.init_factors(R, X.J, X.K, seed=6)
    with p2.Parafac2(R, nonneg=True) as m:
        m.load(X)
        m.init(H0, V0, W0)
        fits = [m.iterate(1) for _ in range(10)]
        _, V, W = m.factors()
    ref = P.parafac2_als(X, H0, V0, W0, n_iter=10, nonneg=True)
    assert max(abs(a - h["fit"]) for a, h in zip(fits, ref["history"])) < FIT_TOL
    assert np.all(V >= 0) and np.all(W >= 0)


@pytest.mark.parametrize("name,K,R,precision", [("tiny", 200, 5, "fp32"), ("c63m", 2000, 10, "fp32"),
                                                ("c250m", 300, 40, "fp32"), ("c63m", 2000, 10, "bf16")])
def test_rational_start_matches_oracle(p2, name, K, R, precision):
    """p2_init_eig: H = I, W = 1 and V = the oracle's leading eigenvectors of
    sum_k X_k^T X_k (within 1e-5, or 3e-3 with bfloat16 storage of V); one
    iteration from the stored start against the oracle's iteration from the
    same state."""
    X = synth.generate(name, K=K)
    blocks = P.all_blocks(X)
    _, Vref, _, _ = P.rational_start(blocks, X.K, X.J, R)
    bf16 = precision == "bf16"
    with p2.Parafac2(R, precision=precision) as m:
        m.load(X)
        n = m.init_eig(max_iter=2000, tol=1e-10)
        H, V, W = m.factors()
        fit = m.iterate(1)
        H1, V1, W1 = m.factors()
    assert 1 <= n < 2000
    assert np.array_equal(H, np.eye(R, dtype=np.float32))
    assert np.all(W == 1.0)
    assert rel_fro(V, Vref) < (3e-3 if bf16 else TOL), rel_fro(V, Vref)
    if bf16:
        return
    ref = P.als_iteration(blocks, np.eye(R), V.astype(np.float64), np.ones((X.K, R)))
    for key, got in (("H", H1), ("V", V1), ("W", W1)):
        assert rel_fro(got, ref[key]) < TOL, (key, rel_fro(got, ref[key]))
    assert abs(fit - P.fit_from_loss(ref["loss"], P.norm_x_sq(blocks))) < FIT_TOL


def test_rational_start_rank_deficient_and_limits(p2):
    """sum_k X_k^T X_k of rank 3 with R = 5: the leading three columns match
    the oracle, the other two complete an orthonormal V; J < R and bad
    arguments are rejected with P2_EINVAL."""
    rng = np.random.default_rng(5)
    mats = []
    for _ in range(40):
        d = np.zeros((6, 30))
        d[:, [2, 7, 19]] = rng.uniform(0.5, 2.0, (6, 3))
        mats.append(d)
    X = slices_from_dense(mats, J=30)
    _, Vref, _, _ = P.rational_start(P.all_blocks(X), X.K, X.J, 5)
    with p2.Parafac2(5) as m:
        m.load(X)
        n = m.init_eig(max_iter=500, tol=1e-10)
        _, V, _ = m.factors()
        fit = m.iterate(2)
        for bad in ((0, 1e-6), (10, -1.0)):
            with pytest.raises(p2.P2Error) as ei:
                m.init_eig(*bad)
            assert ei.value.code == p2.P2_EINVAL
    V = V.astype(np.float64)
    assert n < 500
    assert np.abs(V.T @ V - np.eye(5)).max() < 1e-6
    assert rel_fro(V[:, :3], Vref[:, :3]) < TOL
    assert np.isfinite(fit)
    narrow = slices_from_dense([rng.uniform(0.5, 1.0, (3, 4)) for _ in range(5)], J=4)
    with p2.Parafac2(5) as m:
        m.load(narrow)
        with pytest.raises(p2.P2Error) as ei:
            m.init_eig()
        assert ei.value.code == p2.P2_EINVAL
