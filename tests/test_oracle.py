"""Pins of the FP64 oracle against facts fixed by the paper and by mathematics.

Each test would fail on a plausible slip inside the oracle (a dropped W
factor, a transposed H, a wrong unfolding, a missing normalisation, a wrong
polar factor or pseudo-inverse).
"""
import json
import os

import numpy as np
import pytest
import scipy.linalg

import synth
from oracle import parafac2 as P
from oracle import bruteforce as BF
from tests.helpers import (slices_from_dense, rel_fro, random_orthonormal,
                           planted_parafac2, tucker_congruence)

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "worked_examples.json")


def _random_state(rng, K, J, R, imax=6, density=0.5):
    mats = []
    for k in range(K):
        I = int(rng.integers(1, imax + 1))
        m = rng.random((I, J)) * (rng.random((I, J)) < density)
        for i in range(I):                # keep every row non-empty
            if not m[i].any():
                m[i, rng.integers(J)] = 1.0 + rng.random()
        mats.append(m)
    X = slices_from_dense(mats, J)
    H = rng.standard_normal((R, R))
    V = rng.random((J, R))
    W = rng.random((K, R)) + 0.1
    return X, H, V, W


# ---------------------------------------------------------------- Algorithm 3
@pytest.mark.parametrize("seed,R", [(0, 3), (1, 4), (2, 1), (3, 5)])
def test_mttkrp_matches_textbook_unfolding(seed, R):
    """Algorithm 3 equals Y_(n)(KR) on the materialised Y (Eqs. mttkrp1/2/3)."""
    rng = np.random.default_rng(seed)
    K, J = 7, 9
    X, H, V, W = _random_state(rng, K, J, R)
    blocks = P.all_blocks(X)
    Qs = [P.procrustes_q(Xc, cols, H, V, W[k]) for k, (Xc, cols) in enumerate(blocks)]
    Ys = [P.form_y(Qs[k], blocks[k][0]) for k in range(K)]
    colsets = [c for _, c in blocks]
    Y = BF.materialize_y(blocks, Qs, R, J)
    for mode in (1, 2, 3):
        got = P.mttkrp_spartan(Ys, colsets, H, V, W, mode)
        ref = BF.mttkrp(Y, H, V, W, mode)
        assert rel_fro(got, ref) < 1e-12, mode


def test_mttkrp_index_forms():
    """Element formulas: M1[r,s]=sum Y[r,j,k]V[j,s]W[k,s], M2[j,s]=sum Y[r,j,k]H[r,s]W[k,s],
    M3[k,s]=sum H[r,s]Y[r,j,k]V[j,s]."""
    rng = np.random.default_rng(11)
    K, J, R = 4, 5, 3
    X, H, V, W = _random_state(rng, K, J, R)
    blocks = P.all_blocks(X)
    Qs = [random_orthonormal(rng, Xc.shape[0], R) if Xc.shape[0] >= R else
          random_orthonormal(rng, R, Xc.shape[0]).T for Xc, _ in blocks]
    Ys = [P.form_y(Qs[k], blocks[k][0]) for k in range(K)]
    Y = BF.materialize_y(blocks, Qs, R, J)
    colsets = [c for _, c in blocks]
    M1 = np.einsum("rjk,js,ks->rs", Y, V, W)
    M2 = np.einsum("rjk,rs,ks->js", Y, H, W)
    M3 = np.einsum("rs,rjk,js->ks", H, Y, V)
    assert rel_fro(P.mttkrp_spartan(Ys, colsets, H, V, W, 1), M1) < 1e-12
    assert rel_fro(P.mttkrp_spartan(Ys, colsets, H, V, W, 2), M2) < 1e-12
    assert rel_fro(P.mttkrp_spartan(Ys, colsets, H, V, W, 3), M3) < 1e-12


# ---------------------------------------------------------------- Q-step
def test_procrustes_polar_closed_form_and_orthonormality():
    """Q_k is the polar factor of A_k = X_k V S_k H^T: Q_k (A^T A)^{1/2} = A,
    Q^T Q = I when I_k >= R (full rank), Q Q^T = I when I_k < R."""
    rng = np.random.default_rng(5)
    R, J = 4, 10
    for I in (1, 2, 3, 4, 7, 12):
        Xc = rng.random((I, J)) + 0.05
        cols = np.arange(J)
        H = rng.standard_normal((R, R))
        V = rng.random((J, R))
        w = rng.random(R) + 0.2
        Q = P.procrustes_q(Xc, cols, H, V, w)
        A = Xc @ V @ np.diag(w) @ H.T
        if I >= R:
            assert np.abs(Q.T @ Q - np.eye(R)).max() < 1e-12
            S = scipy.linalg.sqrtm(A.T @ A).real
            assert rel_fro(Q @ S, A) < 1e-10
        else:
            assert np.abs(Q @ Q.T - np.eye(I)).max() < 1e-12
            S = scipy.linalg.sqrtm(A @ A.T).real      # A = (A A^T)^{1/2} Q
            assert rel_fro(S @ Q, A) < 1e-10


def test_procrustes_beats_random_orthonormal():
    """No other column-orthonormal Q gives a lower ||X_k - Q H S_k V^T|| (Section 3.2)."""
    rng = np.random.default_rng(6)
    R, J, I = 3, 8, 6
    Xc = rng.random((I, J))
    cols = np.arange(J)
    H = rng.standard_normal((R, R))
    V = rng.random((J, R))
    w = rng.random(R) + 0.1
    B = H @ np.diag(w) @ V.T
    Q = P.procrustes_q(Xc, cols, H, V, w)
    best = np.linalg.norm(Xc - Q @ B)
    for _ in range(500):
        Qr = random_orthonormal(rng, I, R)
        assert np.linalg.norm(Xc - Qr @ B) >= best - 1e-12


def test_procrustes_rank1_special_case():
    """R = 1: the polar factor of a column a is a / ||a||."""
    rng = np.random.default_rng(7)
    Xc = rng.random((5, 6))
    cols = np.arange(6)
    H = np.array([[-1.7]])
    V = rng.random((6, 1))
    w = np.array([0.8])
    a = Xc @ V * w[0] * H[0, 0]
    Q = P.procrustes_q(Xc, cols, H, V, w)
    assert rel_fro(Q, a / np.linalg.norm(a)) < 1e-13


def test_procrustes_rank_deficient_is_partial_isometry():
    """Proportional rows give rank(A_k) < R: Q_k is the partial isometry on range(A_k)."""
    rng = np.random.default_rng(8)
    R, J = 3, 6
    base = rng.random((1, J))
    Xc = np.vstack([base, 2.0 * base, rng.random((1, J))])     # rank 2
    cols = np.arange(J)
    H = rng.standard_normal((R, R))
    V = rng.random((J, R))
    w = rng.random(R) + 0.1
    Q = P.procrustes_q(Xc, cols, H, V, w)
    sv = np.linalg.svd(Q, compute_uv=False)
    assert np.allclose(sorted(sv), [0.0, 1.0, 1.0], atol=1e-10)
    A = Xc @ V @ np.diag(w) @ H.T
    # Q maps onto range(A) and Q^T A is symmetric positive semidefinite
    QtA = Q.T @ A
    assert np.abs(QtA - QtA.T).max() < 1e-10
    assert np.linalg.eigvalsh((QtA + QtA.T) / 2).min() > -1e-10


def test_procrustes_zero_slice():
    Xc = np.zeros((2, 3))
    Q = P.procrustes_q(Xc, np.arange(3), np.eye(2), np.ones((3, 2)), np.ones(2))
    assert np.all(Q == 0)


# ---------------------------------------------------------------- solves
def test_sweep_solves_equal_least_squares():
    """Each CP-ALS update of Algorithm 1 is the least-squares factor on the explicit KR."""
    rng = np.random.default_rng(9)
    K, J, R = 6, 7, 3
    X, H, V, W = _random_state(rng, K, J, R)
    blocks = P.all_blocks(X)
    Qs = [P.procrustes_q(Xc, cols, H, V, W[k]) for k, (Xc, cols) in enumerate(blocks)]
    Ys = [P.form_y(Qs[k], blocks[k][0]) for k in range(K)]
    Y = BF.materialize_y(blocks, Qs, R, J)
    colsets = [c for _, c in blocks]
    H1, V1, W1, *_ = P.cp_als_sweep(Ys, colsets, H, V, W)
    Href = BF.ls_factor(Y, H, V, W, 1)
    Href = Href / np.linalg.norm(Href, axis=0)
    assert rel_fro(H1, Href) < 1e-10
    Vref = BF.ls_factor(Y, H1, V, W, 2)
    Vref = Vref / np.linalg.norm(Vref, axis=0)
    assert rel_fro(V1, Vref) < 1e-10
    Wref = BF.ls_factor(Y, H1, V1, W, 3)
    assert rel_fro(W1, Wref) < 1e-10
    assert np.allclose(np.linalg.norm(H1, axis=0), 1.0)
    assert np.allclose(np.linalg.norm(V1, axis=0), 1.0)


# ---------------------------------------------------------------- loss / fit
def test_surrogate_loss_closed_form_and_exact():
    """L~ (per-k sum) = ||X||^2 - 2<W,M3> + 1^T(W^TW*H^TH*V^TV)1, and L~ = L when
    every Q_k has orthonormal columns."""
    rng = np.random.default_rng(10)
    K, J, R = 5, 8, 3
    mats = [rng.random((int(rng.integers(R, R + 4)), J)) for _ in range(K)]
    X = slices_from_dense(mats, J)
    H = rng.standard_normal((R, R))
    V = rng.random((J, R))
    W = rng.random((K, R)) + 0.1
    blocks = P.all_blocks(X)
    out = P.als_iteration(blocks, H, V, W, want_exact=True)
    H1, V1, W1, M3 = out["H"], out["V"], out["W"], out["M3"]
    closed = (P.norm_x_sq(blocks) - 2.0 * np.sum(W1 * M3)
              + np.sum((W1.T @ W1) * (H1.T @ H1) * (V1.T @ V1)))
    assert abs(out["loss"] - closed) <= 1e-10 * P.norm_x_sq(blocks)
    assert abs(out["loss"] - out["loss_exact"]) <= 1e-10 * P.norm_x_sq(blocks)


def test_loss_nonincreasing_tiny_workload():
    """Section 3.2: a single CP-ALS iteration after the Q-step decreases the objective."""
    X = synth.generate("tiny", K=60)
    R = 5
    H0, V0, W0 = synth.init_factors(R, X.J, X.K, seed=1)
    res = P.parafac2_als(X, H0, V0, W0, n_iter=12)
    losses = [h["loss"] for h in res["history"]]
    nx2 = res["norm_x_sq"]
    for a, b in zip(losses, losses[1:]):
        assert b <= a + 1e-10 * nx2
    assert losses[-1] < losses[0]


# ---------------------------------------------------------------- whole iteration
def test_worked_examples_golden():
    with open(GOLDEN) as f:
        data = json.load(f)
    for ex in data["examples"]:
        X = slices_from_dense([np.array(m, float) for m in ex["X"]], ex["J"])
        blocks = P.all_blocks(X)
        out = P.als_iteration(blocks, np.array(ex["H0"], float), np.array(ex["V0"], float),
                              np.array(ex["W0"], float))
        for k, Q in enumerate(ex["Q"]):
            assert np.allclose(out["Qs"][k], Q, atol=1e-12), ex["name"]
        for key in ("M1", "M2", "M3", "H", "V", "W"):
            assert np.allclose(out[key], np.array(ex[key], float), atol=1e-12), (ex["name"], key)
        nx2 = P.norm_x_sq(blocks)
        assert abs(out["loss"] - ex["loss"]) < 1e-10 * nx2
        assert abs(P.fit_from_loss(out["loss"], nx2) - ex["fit"]) < 1e-6


def test_cp_special_case_fits_exactly():
    """A CP tensor (U_k = U for every k) is an exact PARAFAC2 model (Sections 2.2, 3.1):
    from the best of five random starts the loss reaches round-off."""
    rng = np.random.default_rng(12)
    K, J, R, I = 12, 8, 2, 5
    U = rng.standard_normal((I, R))
    V = rng.standard_normal((J, R))
    W = rng.uniform(0.1, 2.0, (K, R))
    X = slices_from_dense([U @ np.diag(W[k]) @ V.T for k in range(K)], J)
    blocks = P.all_blocks(X)
    best = np.inf
    for s in range(5):
        r2 = np.random.default_rng(100 + s)
        res = P.parafac2_als(X, r2.random((R, R)), r2.random((J, R)), r2.random((K, R)), 400,
                             blocks=blocks)
        best = min(best, res["history"][-1]["loss"] / res["norm_x_sq"])
        if best < 1e-12:
            break
    assert best < 1e-10


@pytest.mark.parametrize("w_sparse", [False, True])
def test_planted_recovery(w_sparse):
    """PARAFAC2 is unique for K >= 4 (Section 3.1): planted noiseless data is fitted
    exactly and V, W are recovered up to permutation, scale and sign."""
    rng = np.random.default_rng(13 if not w_sparse else 14)
    K, J, R, I = 8, 9, 2, 5
    Xs, Ht, Vt, Wt = planted_parafac2(rng, K, J, R, I, w_sparse=w_sparse)
    X = slices_from_dense(Xs, J)
    blocks = P.all_blocks(X)
    best = None
    for s in range(8):                      # best of several random starts (ALS has local minima)
        r2 = np.random.default_rng(200 + s)
        res = P.parafac2_als(X, r2.random((R, R)), r2.random((J, R)), r2.random((K, R)), 600,
                             blocks=blocks)
        if best is None or res["history"][-1]["loss"] < best["history"][-1]["loss"]:
            best = res
        if best["history"][-1]["loss"] / best["norm_x_sq"] < 1e-13:
            break
    assert best["history"][-1]["loss"] / best["norm_x_sq"] < 1e-10
    assert tucker_congruence(best["V"], Vt) > 0.9999
    if w_sparse:
        # a subject with a single active component fixes that entry of W only up to sign
        assert tucker_congruence(np.abs(best["W"]), np.abs(Wt)) > 0.9999
    else:
        assert tucker_congruence(best["W"], Wt) > 0.9999


def test_invariances_subject_and_column_permutation_and_scaling():
    X = synth.generate("tiny", K=30)
    R = 3
    H0, V0, W0 = synth.init_factors(R, X.J, X.K, seed=2)
    base = P.parafac2_als(X, H0, V0, W0, n_iter=3)
    rng = np.random.default_rng(0)
    # subjects permuted -> W rows permuted
    perm = rng.permutation(X.K)
    Xp = X.take(perm)
    res = P.parafac2_als(Xp, H0, V0, W0[perm], n_iter=3)
    assert rel_fro(res["W"], base["W"][perm]) < 1e-10
    assert rel_fro(res["V"], base["V"]) < 1e-10
    # columns permuted -> V rows permuted
    cperm = rng.permutation(X.J)              # new column id of old column j is cperm[j]
    mats = []
    for k in range(X.K):
        Xc, cols = P.subject_block(X, k)
        full = np.zeros((Xc.shape[0], X.J))
        full[:, cperm[cols]] = Xc
        mats.append(full)
    Xq = slices_from_dense(mats, X.J)
    V0q = np.empty_like(V0)
    V0q[cperm] = V0
    res = P.parafac2_als(Xq, H0, V0q, W0, n_iter=3)
    assert rel_fro(res["V"][cperm], base["V"]) < 1e-10
    assert rel_fro(res["W"], base["W"]) < 1e-10
    # X scaled by c -> W scaled by c, fit unchanged
    Xs = type(X)(X.K, X.J, X.subj_ptr, X.row_ptr, X.col, (X.val * 4.0).astype(np.float32))
    res = P.parafac2_als(Xs, H0, V0, W0, n_iter=3)
    assert rel_fro(res["W"], 4.0 * base["W"]) < 1e-10
    assert abs(res["history"][-1]["fit"] - base["history"][-1]["fit"]) < 1e-10


# ---------------------------------------------------------------- projection (serving)
def test_projection_recovers_planted_weights():
    """With the true (H, V) of noiseless planted data, projecting a subject from s = 1
    converges to that subject's W row (the model is exact and unique, Section 3.1)."""
    rng = np.random.default_rng(21)
    K, J, R, I = 6, 9, 3, 7
    Xs, Ht, Vt, Wt = planted_parafac2(rng, K, J, R, I)
    X = slices_from_dense(Xs, J)
    for k in range(K):
        Xc, cols = P.subject_block(X, k)
        s, Q = P.project_subject(Xc, cols, Ht, Vt, n_iter=200)
        assert np.allclose(s, Wt[k], rtol=1e-6, atol=1e-8), (k, s, Wt[k])
        assert np.allclose(Q @ Ht @ np.diag(s) @ Vt[cols].T, Xc, atol=1e-8)


def test_projection_step_is_the_least_squares_row():
    """One s-update equals argmin_s ||Y - H diag(s) V^T||_F on the explicit Khatri-Rao
    (mode-3 solve of Algorithm 1 for a single subject)."""
    rng = np.random.default_rng(22)
    J, R = 8, 3
    Xc = rng.random((6, J))
    cols = np.arange(J)
    H = rng.standard_normal((R, R))
    V = rng.random((J, R))
    s0 = rng.random(R) + 0.5
    s1, _ = P.project_subject(Xc, cols, H, V, n_iter=1, s0=s0)
    Q = P.procrustes_q(Xc, cols, H, V, s0)
    Y = Q.T @ Xc                                            # R x J
    KR = BF.khatri_rao(V, H)                                # row r + R j
    ref, *_ = np.linalg.lstsq(KR, Y.T.reshape(-1), rcond=None)
    assert rel_fro(s1, ref) < 1e-10


# ---------------------------------------------------------------- non-negative variant
@pytest.mark.parametrize("n,seed", [(1, 0), (2, 1), (5, 2), (10, 3), (10, 4), (40, 5)])
def test_nnls_gram_matches_scipy_and_kkt(n, seed):
    """nnls_gram solves min_{x>=0} ||y - Bx||^2 from A = B^T B and b = B^T y:
    it must equal scipy's NNLS (a separate Lawson-Hanson implementation) on
    the factored problem min ||U x - U^{-T} b|| (A = U^T U), and satisfy the
    KKT conditions x >= 0, w = b - A x <= 0 where x = 0, w = 0 where x > 0."""
    import scipy.optimize
    rng = np.random.default_rng(seed)
    B = rng.standard_normal((3 * n + 2, n))
    B[:, : max(1, n // 3)] *= 1e-2                      # some conditioning
    A = B.T @ B
    b = B.T @ rng.standard_normal(3 * n + 2)
    x = P.nnls_gram(A, b)
    U = scipy.linalg.cholesky(A, lower=False)
    ref, _ = scipy.optimize.nnls(U, scipy.linalg.solve_triangular(U, b, trans="T"))
    assert np.linalg.norm(x - ref) <= 1e-9 * max(np.linalg.norm(ref), 1e-300)
    w = b - A @ x
    scale = np.abs(b).max() + np.abs(A).max() * np.abs(x).max()
    assert np.all(x >= 0)
    assert np.all(w[x == 0] <= 1e-10 * scale)
    assert np.all(np.abs(w[x > 0]) <= 1e-10 * scale)


def test_nnls_gram_interior_and_boundary_cases():
    """A positive unconstrained solution is returned as is; b < 0 gives 0; a
    diagonal A decouples into max(b_i, 0) / A_ii."""
    rng = np.random.default_rng(9)
    B = rng.standard_normal((20, 6))
    A = B.T @ B
    x0 = rng.random(6) + 0.5
    assert np.allclose(P.nnls_gram(A, A @ x0), x0, rtol=1e-12, atol=0)
    assert np.all(P.nnls_gram(A, -np.ones(6)) == 0.0)       # x = 0 meets the KKT conditions
    Ad = np.diag(rng.random(6) + 1.0)
    bd = rng.standard_normal(6)
    assert np.allclose(P.nnls_gram(Ad, bd), np.maximum(bd, 0) / np.diag(Ad), rtol=1e-14, atol=0)


def test_nonneg_iteration_keeps_sign_and_decreases_loss():
    """Section 5.1's variant: V and W stay non-negative and every block update
    is an exact minimisation, so the surrogate loss never increases."""
    X = synth.generate("tiny", K=60)
    R = 5
    H0, V0, W0 = synth.init_factors(R, X.J, X.K, seed=1)
    res = P.parafac2_als(X, H0, V0, W0, n_iter=10, nonneg=True)
    assert np.all(res["V"] >= 0) and np.all(res["W"] >= 0)
    losses = [h["loss"] for h in res["history"]]
    nx2 = res["norm_x_sq"]
    for a, b in zip(losses, losses[1:]):
        assert b <= a + 1e-10 * nx2


def _dense_stack(X):
    """The stacked dense N x J matrix of the collection (FP32 values as FP64)."""
    rows = []
    for k in range(X.K):
        Xc, cols = P.subject_block(X, k)
        D = np.zeros((Xc.shape[0], X.J))
        D[:, cols] = Xc
        rows.append(D)
    return np.vstack(rows)


def test_rational_start_equals_right_singular_vectors():
    """V of the rational start = the leading right singular vectors of the
    stacked X (an SVD of X, not the eigen-solver of sum_k X_k^T X_k the
    oracle uses), its eigenvalues the squared singular values; H = I, W = 1;
    each column's entry of largest magnitude is positive."""
    rng = np.random.default_rng(3)
    mats = []
    for _ in range(9):
        I = int(rng.integers(2, 7))
        mats.append(rng.uniform(0.1, 1.0, (I, 12)) * (rng.uniform(size=(I, 12)) < 0.5))
    X = slices_from_dense(mats, J=12)
    R = 4
    H, V, W, lam = P.rational_start(P.all_blocks(X), X.K, X.J, R)
    _, sv, Vt = np.linalg.svd(_dense_stack(X))
    ref = Vt[:R].T.copy()
    for r in range(R):
        j = int(np.argmax(np.abs(ref[:, r])))
        ref[:, r] *= np.sign(ref[j, r])
    assert np.abs(V - ref).max() < 1e-10
    assert np.allclose(lam[:R], sv[:R] ** 2, rtol=1e-10)
    assert np.array_equal(H, np.eye(R)) and np.array_equal(W, np.ones((X.K, R)))
    for r in range(R):
        assert V[np.argmax(np.abs(V[:, r])), r] > 0


def test_rational_start_closed_form_for_orthogonal_columns():
    """One non-zero per row: the columns of the stacked X are orthogonal, so
    sum_k X_k^T X_k is diagonal with the column sums of squares, and V is the
    unit vectors of the R columns with the largest sums, in that order."""
    rng = np.random.default_rng(8)
    J, R = 15, 5
    mats = []
    for _ in range(6):
        I = int(rng.integers(3, 9))
        D = np.zeros((I, J))
        D[np.arange(I), rng.integers(0, J, I)] = rng.uniform(0.5, 3.0, I)
        mats.append(D)
    X = slices_from_dense(mats, J=J)
    ss = (_dense_stack(X) ** 2).sum(axis=0)
    top = np.argsort(-ss, kind="stable")[:R]
    _, V, _, lam = P.rational_start(P.all_blocks(X), X.K, X.J, R)
    assert np.abs(V - np.eye(J)[:, top]).max() < 1e-12
    assert np.allclose(lam[:R], ss[top], rtol=1e-12)


def test_assemble_u_reconstructs_planted_slices():
    """U_k = Q_k H (Algorithm 2, after the loop) on planted noiseless data
    X_k = Q_k H S_k V^T: with the true H, V, W the Procrustes step returns the
    planted Q_k, so the assembled U_k must reproduce every slice as
    U_k S_k V^T (to the FP32 rounding of the stored values) and satisfy
    U_k^T U_k = H^T H (Q_k has orthonormal columns).  A transposed H, or H
    applied on the wrong side, fails both."""
    rng = np.random.default_rng(31)
    K, J, R, I = 6, 9, 3, 5
    Xs, H, V, W = planted_parafac2(rng, K, J, R, I)
    X = slices_from_dense(Xs, J)
    blocks = P.all_blocks(X)
    Qs = [P.procrustes_q(Xc, cols, H, V, W[k]) for k, (Xc, cols) in enumerate(blocks)]
    Us = P.assemble_u(Qs, H)
    for k, (Xc, cols) in enumerate(blocks):
        Xk = np.zeros((I, J))
        Xk[:, cols] = Xc
        assert Us[k].shape == (I, R)
        assert np.linalg.norm(Us[k] @ np.diag(W[k]) @ V.T - Xk) <= 1e-6 * np.linalg.norm(Xk)
        assert np.abs(Us[k].T @ Us[k] - H.T @ H).max() <= 1e-10 * np.abs(H.T @ H).max()


@pytest.mark.parametrize("nonneg", [False, True])
def test_pooled_iteration_equals_serial_oracle(nonneg):
    """oracle.pool runs the same per-subject functions over subject chunks in
    worker processes; only the order of the FP64 sums over subjects differs,
    so two iterations agree with parafac2.parafac2_als to round-off."""
    from oracle.pool import OraclePool
    X = synth.generate("tiny", K=200)
    R = 5
    H0, V0, W0 = synth.init_factors(R, X.J, X.K, seed=9)
    ref = P.parafac2_als(X, H0, V0, W0, n_iter=2, nonneg=nonneg)
    with OraclePool(X, n_workers=3) as pool:
        assert pool.n_workers == 3
        got = pool.parafac2_als(H0, V0, W0, n_iter=2, nonneg=nonneg)
    for key in ("H", "V", "W"):
        assert rel_fro(got[key], ref[key]) < 1e-12, key
    for key in ("M1", "M2", "M3"):
        assert rel_fro(got["last"][key], ref["last"][key]) < 1e-12, key
    for a, b in zip(got["history"], ref["history"]):
        assert abs(a["fit"] - b["fit"]) < 1e-13
    assert abs(got["norm_x_sq"] - ref["norm_x_sq"]) <= 1e-13 * ref["norm_x_sq"]
