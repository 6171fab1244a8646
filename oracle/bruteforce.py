"""Brute-force checker for the oracle's MTTKRPs and solves.

TEST INFRASTRUCTURE ONLY (same rules as ``oracle/parafac2.py``).

It materialises the dense intermediate tensor Y (R x J x K) with frontal
slices Y_k = Q_k^T X_k (Algorithm 2), unfolds it (mode-n matricization as in
Section 2.1 / Kolda & Bader 2009: the mode-n fibres become columns, earlier
modes varying fastest), builds the Khatri-Rao products explicitly and forms
the textbook MTTKRPs Y_(n) (· ⊙ ·) of Eqs. mttkrp1, mttkrp2 and mttkrp3
(Section 4.2) and the CP-ALS least-squares solves of Algorithm 1 by a
QR-based least-squares routine.  No step follows Algorithm 3's per-subject
reformulation, so agreement with the oracle pins it.
"""
from __future__ import annotations

import numpy as np


def materialize_y(blocks, Qs, R, J):
    """Dense Y (R x J x K) with Y(:, :, k) = Q_k^T X_k."""
    K = len(blocks)
    Y = np.zeros((R, J, K))
    for k, (Xc, cols) in enumerate(blocks):
        Y[:, cols, k] = Qs[k].T @ Xc
    return Y


def unfold(Y, mode):
    """Mode-n matricization of a 3-way array (modes 1, 2, 3)."""
    R, J, K = Y.shape
    if mode == 1:      # R x (J K): column j + J k
        return Y.transpose(0, 2, 1).reshape(R, K * J)
    if mode == 2:      # J x (R K): column r + R k
        return Y.transpose(1, 2, 0).reshape(J, K * R)
    if mode == 3:      # K x (R J): column r + R j
        return Y.transpose(2, 1, 0).reshape(K, J * R)
    raise ValueError(mode)


def khatri_rao(A, B):
    """Column-wise Kronecker product A ⊙ B; row (a, b) sits at a * rows(B) + b."""
    nA, R = A.shape
    nB, R2 = B.shape
    assert R == R2
    return np.einsum("ar,br->abr", A, B).reshape(nA * nB, R)


def mttkrp(Y, H, V, W, mode):
    """Y_(1)(W ⊙ V), Y_(2)(W ⊙ H) or Y_(3)(V ⊙ H)."""
    if mode == 1:
        return unfold(Y, 1) @ khatri_rao(W, V)
    if mode == 2:
        return unfold(Y, 2) @ khatri_rao(W, H)
    if mode == 3:
        return unfold(Y, 3) @ khatri_rao(V, H)
    raise ValueError(mode)


def ls_factor(Y, H, V, W, mode):
    """argmin_F || Y_(n) - F (KR)^T ||_F by least squares on the explicit KR."""
    if mode == 1:
        KR = khatri_rao(W, V)
    elif mode == 2:
        KR = khatri_rao(W, H)
    else:
        KR = khatri_rao(V, H)
    sol, *_ = np.linalg.lstsq(KR, unfold(Y, mode).T, rcond=None)
    return sol.T
