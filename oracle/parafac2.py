"""FP64 CPU oracle of SPARTan's PARAFAC2-ALS iteration.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path imports this module:
only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline /
reference arm may call it.  It shares no code with the CUDA path.

It is written to be checked against the paper by eye, not to be fast:
per-subject Python loops, FP64 numpy arithmetic, library primitives (SVD,
matrix product, symmetric pseudo-inverse) used as single steps.  Every
function cites the passage it follows (Perros et al., "SPARTan: Scalable
PARAFAC2 for Large & Sparse Data", KDD 2017, arXiv:1703.04219).

Readings of points the paper leaves open (each also listed in the design
notes of the repository):

* Rank cut of the Procrustes SVD (Algorithm 2, "truncated SVD at rank R"):
  singular values sigma_i <= RANK_RTOL * sigma_1 are treated as zero, so when
  I_k < R or X_k V S_k H^T is rank deficient Q_k is the partial isometry
  Z_r P_r^T over the kept singular pairs; Q_k = 0 when sigma_1 = 0.
* "P_k Sigma_k Z_k" (Section 3.2) is read as P_k Sigma_k Z_k^T, with
  Q_k = Z_k P_k^T, i.e. the polar factor of A_k = X_k V S_k H^T.
* One CP-ALS sweep (Algorithm 1 body) in the order H, V, W.  H and V get unit
  2-norm columns and their norms are dropped; W is not normalised, so it
  carries lambda and S_k = diag(W(k,:)) keeps the model scale.
* Moore-Penrose pseudo-inverses of the R x R Gram-Hadamard products drop
  eigenvalues <= R * 2^-52 * lambda_max.
* Non-negative variant (Section 5.1 constrains {S_k} and V): the V and W
  solves become row-wise non-negative least squares with the same Gram-
  Hadamard products; H stays unconstrained.  The loss below is unchanged.
* Loss: the surrogate L~ = sum_k ||X_k||^2 - 2<Y_k, H S_k V^T> + ||H S_k V^T||^2
  (the objective of Section 3.2's CP step plus the constant ||X_k||^2 -
  ||Q_k^T X_k||^2), fit = 1 - sqrt(max(L~, 0)) / ||X||_F.  The exact
  sum_k ||X_k - Q_k H S_k V^T||^2 is available for diagnostics.
"""
from __future__ import annotations

import numpy as np

RANK_RTOL = 1e-5
EPS64 = 2.0 ** -52


# --------------------------------------------------------------------------
# data access: X_k restricted to its non-zero columns (Section 3.3,
# "Structured sparsity"; Section 4.1: Y_k has R c_k non-zeros located in the
# non-zero columns of X_k)
# --------------------------------------------------------------------------
def subject_block(slices, k):
    """Dense FP64 block of X_k on its c_k non-empty columns, and those columns."""
    rp, col, val = slices.subject(k)
    cols = np.unique(col)
    I = len(rp) - 1
    Xc = np.zeros((I, len(cols)), dtype=np.float64)
    pos = np.searchsorted(cols, col)
    for i in range(I):
        Xc[i, pos[rp[i]:rp[i + 1]]] = val[rp[i]:rp[i + 1]].astype(np.float64)
    return Xc, cols


def all_blocks(slices):
    return [subject_block(slices, k) for k in range(slices.K)]


# --------------------------------------------------------------------------
# Q-step: orthogonal Procrustes (Section 3.2, Eq. for min ||X_k - Q_k H S_k V^T||,
# Algorithm 2 first inner loop)
# --------------------------------------------------------------------------
def procrustes_q(Xc, cols, H, V, w, rank_rtol=RANK_RTOL):
    """Q_k from the SVD of H S_k V^T X_k^T = P_k Sigma_k Z_k^T, Q_k = Z_k P_k^T."""
    B = H @ np.diag(w) @ V[cols].T @ Xc.T          # R x I_k
    P, sig, Zt = np.linalg.svd(B, full_matrices=False)
    I = Xc.shape[0]
    R = H.shape[0]
    if sig.size == 0 or sig[0] <= 0.0:
        return np.zeros((I, R))
    keep = sig > rank_rtol * sig[0]
    Z = Zt[keep].T                                  # I_k x r
    return Z @ P[:, keep].T                         # I_k x R


def form_y(Q, Xc):
    """Y_k = Q_k^T X_k on X_k's non-zero columns (Algorithm 2, second inner loop)."""
    return Q.T @ Xc                                  # R x c_k


# --------------------------------------------------------------------------
# SPARTan MTTKRPs on {Y_k} (Section 4.2, Algorithm 3)
# --------------------------------------------------------------------------
def mttkrp_spartan(Ys, colsets, H, V, W, mode):
    """Algorithm 3 for mode n = 1, 2 or 3; Y_k given on its non-zero columns."""
    R = H.shape[0]
    J = V.shape[0]
    K = W.shape[0]
    if mode == 1:
        # M1 = sum_k (Y_k V) * 1 W(k,:)  (Eq. mttkrp1_2 with mttkrp1_3)
        M = np.zeros((R, R))
        for k in range(K):
            temp = Ys[k] @ V[colsets[k]]
            for r in range(R):
                temp[r, :] = temp[r, :] * W[k, :]
            M += temp
        return M
    if mode == 2:
        # M2 = sum_k Y_k^T (W ⊙ H)-block; row j of block k: (Y_k(:,j)^T H) * W(k,:)  (Eq. mttkrp2_3)
        M = np.zeros((J, R))
        for k in range(K):
            temp = np.zeros((J, R))
            for t, j in enumerate(colsets[k]):
                temp[j, :] = (Ys[k][:, t] @ H) * W[k, :]
            M += temp
        return M
    if mode == 3:
        # M3(k,:) = dot(H, Y_k V), column-wise inner products  (Eq. mttkrp3_row_wise)
        M = np.zeros((K, R))
        for k in range(K):
            YV = Ys[k] @ V[colsets[k]]
            M[k, :] = np.sum(H * YV, axis=0)
        return M
    raise ValueError("mode must be 1, 2 or 3")


# --------------------------------------------------------------------------
# one CP-ALS sweep (Algorithm 1 body) on the implicit tensor Y
# --------------------------------------------------------------------------
def pinv_sym(A):
    """Moore-Penrose pseudo-inverse of a symmetric PSD R x R matrix."""
    R = A.shape[0]
    return np.linalg.pinv(A, rcond=R * EPS64, hermitian=True)


def normalize_columns(A):
    """Unit 2-norm columns; a zero column stays zero.  Returns (A_n, norms)."""
    n = np.sqrt(np.sum(A * A, axis=0))
    safe = np.where(n > 0.0, n, 1.0)
    return A / safe, n


def nnls_gram(A, b):
    """argmin_{x >= 0} ||y - B x||^2 given only A = B^T B (symmetric positive
    definite) and b = B^T y, i.e. argmin_{x >= 0} x^T A x / 2 - b^T x.

    The active-set method of Lawson and Hanson ("Solving Least Squares
    Problems", 1974, Chapter 23, algorithm NNLS), with each least-squares
    subproblem on the passive set P solved through its normal equations
    A_PP z_P = b_P.  The minimiser is unique for positive definite A.
    """
    n = b.shape[0]
    scale = max(float(np.max(np.abs(b))), float(np.max(np.abs(A))), 1e-300)
    tol = 64 * n * EPS64 * scale
    x = np.zeros(n)
    P = np.zeros(n, dtype=bool)
    w = b - A @ x
    for _ in range(3 * n + 1):
        if P.all() or not np.any(w[~P] > tol):
            break
        j = int(np.argmax(np.where(P, -np.inf, w)))
        P[j] = True
        while True:
            idx = np.flatnonzero(P)
            z = np.zeros(n)
            z[idx] = np.linalg.solve(A[np.ix_(idx, idx)], b[idx])
            if np.all(z[idx] > 0):
                x = z
                break
            neg = idx[z[idx] <= 0]
            alpha = np.min(x[neg] / (x[neg] - z[neg]))
            x = x + alpha * (z - x)
            P &= x > 0
            x[~P] = 0.0
        w = b - A @ x
    return x


def nnls_rows(M, A):
    """Row-wise non-negative solves: row i of the result is nnls_gram(A, M[i])."""
    return np.stack([nnls_gram(A, M[i]) for i in range(M.shape[0])]) if M.shape[0] else \
        np.zeros_like(M)


def cp_als_sweep(Ys, colsets, H, V, W, nonneg=False):
    """H <- M1 (W^TW * V^TV)^+, normalise; V <- M2 (W^TW * H^TH)^+, normalise;
    W <- M3 (V^TV * H^TH)^+ (Algorithm 1, lines 3-7, with U = H).

    nonneg: Section 5.1's variant with non-negative {S_k} and V: the V and W
    updates become, row by row, the non-negative least-squares problems with
    the same Gram-Hadamard products (nnls_gram); H stays unconstrained."""
    M1 = mttkrp_spartan(Ys, colsets, H, V, W, 1)
    H = M1 @ pinv_sym((W.T @ W) * (V.T @ V))
    H, _ = normalize_columns(H)
    M2 = mttkrp_spartan(Ys, colsets, H, V, W, 2)
    A2 = (W.T @ W) * (H.T @ H)
    V = nnls_rows(M2, A2) if nonneg else M2 @ pinv_sym(A2)
    V, _ = normalize_columns(V)
    M3 = mttkrp_spartan(Ys, colsets, H, V, W, 3)
    A3 = (V.T @ V) * (H.T @ H)
    W = nnls_rows(M3, A3) if nonneg else M3 @ pinv_sym(A3)
    return H, V, W, M1, M2, M3


# --------------------------------------------------------------------------
# loss / fit (objective of Section 3.2)
# --------------------------------------------------------------------------
def surrogate_loss(blocks, Ys, H, V, W):
    """L~ = sum_k ||X_k||^2 - 2 <Y_k, H S_k V^T> + ||H S_k V^T||^2, term by term."""
    total = 0.0
    for k, (Xc, cols) in enumerate(blocks):
        HSVt = H @ np.diag(W[k]) @ V.T                 # R x J
        total += np.sum(Xc * Xc) - 2.0 * np.sum(Ys[k] * HSVt[:, cols]) + np.sum(HSVt * HSVt)
    return total


def exact_loss(blocks, Qs, H, V, W):
    """sum_k ||X_k - Q_k H S_k V^T||_F^2 over all J columns."""
    total = 0.0
    J = V.shape[0]
    for k, (Xc, cols) in enumerate(blocks):
        Xfull = np.zeros((Xc.shape[0], J))
        Xfull[:, cols] = Xc
        D = Xfull - Qs[k] @ H @ np.diag(W[k]) @ V.T
        total += np.sum(D * D)
    return total


def norm_x_sq(blocks):
    return float(sum(np.sum(Xc * Xc) for Xc, _ in blocks))


def fit_from_loss(loss, nx2):
    return 1.0 - np.sqrt(max(loss, 0.0)) / np.sqrt(nx2)


# --------------------------------------------------------------------------
# PARAFAC2-ALS (Algorithm 2)
# --------------------------------------------------------------------------
def als_iteration(blocks, H, V, W, rank_rtol=RANK_RTOL, want_exact=False, nonneg=False):
    """One pass of Algorithm 2's loop body: Q-step, Y, one CP-ALS sweep, S_k."""
    K = len(blocks)
    Qs = [procrustes_q(Xc, cols, H, V, W[k], rank_rtol) for k, (Xc, cols) in enumerate(blocks)]
    Ys = [form_y(Qs[k], blocks[k][0]) for k in range(K)]
    colsets = [cols for _, cols in blocks]
    H, V, W, M1, M2, M3 = cp_als_sweep(Ys, colsets, H, V, W, nonneg)
    out = dict(H=H, V=V, W=W, M1=M1, M2=M2, M3=M3, Qs=Qs, Ys=Ys,
               loss=surrogate_loss(blocks, Ys, H, V, W))
    if want_exact:
        out["loss_exact"] = exact_loss(blocks, Qs, H, V, W)
    return out


def parafac2_als(slices, H0, V0, W0, n_iter, rank_rtol=RANK_RTOL, blocks=None,
                 want_exact=False, nonneg=False):
    """Run n_iter iterations of Algorithm 2 from (H0, V0, W0) in FP64.

    Returns the final factors and the per-iteration loss/fit history.
    """
    if blocks is None:
        blocks = all_blocks(slices)
    H = np.asarray(H0, np.float64)
    V = np.asarray(V0, np.float64)
    W = np.asarray(W0, np.float64)
    nx2 = norm_x_sq(blocks)
    hist = []
    last = None
    for _ in range(n_iter):
        last = als_iteration(blocks, H, V, W, rank_rtol, want_exact, nonneg)
        H, V, W = last["H"], last["V"], last["W"]
        rec = dict(loss=last["loss"], fit=fit_from_loss(last["loss"], nx2))
        if want_exact:
            rec["loss_exact"] = last["loss_exact"]
        hist.append(rec)
    return dict(H=H, V=V, W=W, history=hist, last=last, norm_x_sq=nx2)


# --------------------------------------------------------------------------
# projection of a new subject onto a fixed model (serving): Algorithm 2's
# Q-step and Algorithm 1's W update (mode-3 MTTKRP, Eq. mttkrp3_row_wise,
# times (V^TV * H^TH)^+) applied to one subject with H and V held fixed
# --------------------------------------------------------------------------
def project_subject(Xc, cols, H, V, n_iter, rank_rtol=RANK_RTOL, s0=None, nonneg=False):
    """Alternate Q <- Procrustes(X, H, V, diag(s)) and s <- coldot(H, Q^T X V) G3^+,
    starting from s = 1 (or s0), n_iter times; return s and the Q for the final s.
    nonneg: the model's non-negative variant, s = nnls_gram(G3, coldot(...))."""
    R = H.shape[0]
    s = np.ones(R) if s0 is None else np.asarray(s0, np.float64)
    G3 = (V.T @ V) * (H.T @ H)
    G3p = pinv_sym(G3)
    for _ in range(n_iter):
        Q = procrustes_q(Xc, cols, H, V, s, rank_rtol)
        Y = form_y(Q, Xc)
        m3 = np.sum(H * (Y @ V[cols]), axis=0)
        s = nnls_gram(G3, m3) if nonneg else m3 @ G3p
    return s, procrustes_q(Xc, cols, H, V, s, rank_rtol)


# --------------------------------------------------------------------------
# rational start (the paper leaves Algorithm 2's "Initialize H, V, {S_k}"
# open; reading: Kiers, ten Berge & Bro 1999's start H = I, S_k = I and V
# the R leading eigenvectors of sum_k X_k^T X_k)
# --------------------------------------------------------------------------
def rational_start(blocks, K, J, R):
    """H = I, W = 1 (S_k = I), V = the R leading eigenvectors of sum_k X_k^T X_k,
    in decreasing order of eigenvalue, each column's entry of largest magnitude
    positive (lowest row on ties).  The J x J matrix is formed densely."""
    G = np.zeros((J, J))
    for Xc, cols in blocks:
        G[np.ix_(cols, cols)] += Xc.T @ Xc
    lam, U = np.linalg.eigh(G)
    V = U[:, ::-1][:, :R].copy()
    for r in range(R):
        j = int(np.argmax(np.abs(V[:, r])))
        if V[j, r] < 0:
            V[:, r] = -V[:, r]
    return np.eye(R), V, np.ones((K, R)), lam[::-1]


def assemble_u(Qs, H):
    """U_k = Q_k H (Algorithm 2, after the loop)."""
    return [Q @ H for Q in Qs]
