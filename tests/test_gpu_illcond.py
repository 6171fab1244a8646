"""Procrustes step (Section 3.2) on ill-conditioned subjects, through the C ABI.

The start's V has two nearly dependent columns (tests/helpers.py,
near_dependent_start), so most A_k = X_k V S_k H^T have condition numbers of
1e3 to 1e5.  The GPU's Q_k = X_k V T_k^T must match the oracle's polar factor
within 1e-6 + 1e-8 cond(A_k) per subject: the FP32 storage of T_k allows
~6e-8 cond(A_k), while a Gram accumulated in plain FP32 gives ~6e-8
cond(A_k)^2 and fails the bound for most subjects (the CPU emulation in
tests/test_gram_sensitivity.py shows both on this fixture).  This pins the
error-free Gram of the alpha pass and the double-word eigen-decomposition on
the lane kernel (R = 5, 10) and the grouped kernel (R = 40), and the FP64
arm of the Procrustes step at R = 10 and 40, after the first Q-step
(p2_init) and after one iteration.
"""
import numpy as np
import pytest

import synth
from oracle import parafac2 as P
from tests.helpers import near_dependent_start, rel_fro

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def p2():
    import paper_1703_04219_gb300 as mod
    return mod


def _check(X, H, V, W, T):
    H, V, W = (a.astype(np.float64) for a in (H, V, W))
    conds, worst = [], 0.0
    for k in range(X.K):
        Xc, cols = P.subject_block(X, k)
        Q_ref = P.procrustes_q(Xc, cols, H, V, W[k])
        Q_gpu = Xc @ V[cols] @ T[k].astype(np.float64).T
        A = Xc @ V[cols] @ np.diag(W[k]) @ H.T
        sv = np.linalg.svd(A, compute_uv=False)
        if sv.size == 0 or sv[0] == 0.0:
            assert not np.any(Q_gpu)
            continue
        kept = sv[sv > 1e-5 * sv[0]]
        cond = kept[0] / kept[-1]
        conds.append(cond)
        err = rel_fro(Q_gpu, Q_ref)
        worst = max(worst, err / (1e-6 + 1e-8 * cond))
        assert err < 1e-6 + 1e-8 * cond, (k, err, cond)
    return np.asarray(conds), worst


@pytest.mark.parametrize("name,K,R,fp64", [("tiny", 200, 5, False), ("c63m", 300, 10, False),
                                           ("c250m", 150, 40, False), ("c63m", 300, 10, True),
                                           ("c250m", 150, 40, True)])
def test_ill_conditioned_procrustes_matches_oracle(p2, name, K, R, fp64):
    X = synth.generate(name, K=K)
    H0, V0, W0 = near_dependent_start(R, X.J, X.K, seed=11)
    with p2.Parafac2(R, fp64_procrustes=fp64) as m:
        m.load(X)
        m.init(H0, V0, W0)
        T0 = m.procrustes()
        m.iterate(1)
        H1, V1, W1 = m.factors()
        T1 = m.procrustes()
    conds, _ = _check(X, H0, V0, W0, T0)
    assert np.mean(conds >= 1e3) > 0.5, np.median(conds)
    _check(X, H1, V1, W1, T1)
