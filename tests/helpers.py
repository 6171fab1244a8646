"""Small helpers shared by the tests (no PARAFAC2 arithmetic here)."""
from __future__ import annotations

import numpy as np

from synth import Slices


def slices_from_dense(mats, J=None):
    """Stack dense I_k x J matrices into the CSR collection format (zeros dropped)."""
    mats = [np.asarray(m, dtype=np.float64) for m in mats]
    if J is None:
        J = mats[0].shape[1]
    subj = [0]
    rp = [0]
    cols, vals = [], []
    for m in mats:
        for row in m:
            nz = np.nonzero(row)[0]
            cols.extend(nz.tolist())
            vals.extend(row[nz].tolist())
            rp.append(len(cols))
        subj.append(subj[-1] + m.shape[0])
    return Slices(len(mats), J, np.asarray(subj, np.int64), np.asarray(rp, np.int64),
                  np.asarray(cols, np.int32), np.asarray(vals, np.float32))


def rel_fro(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    d = np.linalg.norm(a - b)
    n = np.linalg.norm(b)
    return d / n if n > 0 else d


def random_orthonormal(rng, n, r):
    q, _ = np.linalg.qr(rng.standard_normal((n, r)))
    return q


def planted_parafac2(rng, K, J, R, I, w_sparse=False):
    """Noiseless planted X_k = Q_k H S_k V^T with random orthonormal Q_k (I x R)."""
    H = rng.standard_normal((R, R))
    V = rng.standard_normal((J, R))
    W = rng.uniform(0.2, 2.0, (K, R))
    if w_sparse:
        W = W * (rng.random((K, R)) > 0.3)
        W[:, 0] += 0.5
    Xs = []
    for k in range(K):
        Q = random_orthonormal(rng, I, R)
        Xs.append(Q @ H @ np.diag(W[k]) @ V.T)
    return Xs, H, V, W


def tucker_congruence(A, B):
    """Best column-matched |congruence| between factor matrices (greedy matching)."""
    An = A / np.linalg.norm(A, axis=0)
    Bn = B / np.linalg.norm(B, axis=0)
    C = np.abs(An.T @ Bn)
    R = C.shape[0]
    used = set()
    worst = 1.0
    for r in np.argsort(-C.max(axis=1)):
        cands = [(C[r, s], s) for s in range(R) if s not in used]
        best, s = max(cands)
        used.add(s)
        worst = min(worst, best)
    return worst


def near_dependent_start(R, J, K, seed, delta=1e-3):
    """Seeded uniform start (synth.init_factors) whose V has its second column
    equal to the first plus delta times Gaussian noise, rounded to FP32.  Every
    Z_k = X_k V then has two nearly dependent columns, so most subjects' A_k =
    Z_k S_k H^T have condition numbers of 1e3 to 1e5 (inside the 1e-5 rank cut
    of the Procrustes step)."""
    import synth
    H0, V0, W0 = synth.init_factors(R, J, K, seed=seed)
    V0 = V0.copy()
    rng = np.random.default_rng(seed + 1)
    V0[:, 1] = (V0[:, 0].astype(np.float64) + delta * rng.standard_normal(J)).astype(np.float32)
    return H0, V0, W0
