"""The paper-shaped planted workloads of the input generator (Section 5,
"Synthetic Data": dense slices X_k = Q_k H S_k V^T sparsified uniformly,
empty rows dropped): every kept entry equals the planted model's value,
Q_k has orthonormal columns, and the statistics match the paper's (mean I_k
46.9 at 63M non-zeros, 99.3 at 500M; 100 (1 - exp(-J p)) in expectation)."""
import numpy as np
import pytest

import synth


def test_planted_entries_equal_the_model():
    w = synth.WORKLOADS["ptiny"]
    X = synth.generate(w)
    D, Rp = w.dense_rows, w.planted_rank
    assert X.n_rows == X.K * D                       # J p = 10: no row of ptiny is empty
    for k in range(X.K):
        H, V, s, v = synth.planted_factors(w, k)
        Q = (np.eye(D) - 2.0 * np.outer(v, v))[:, :Rp]
        assert np.allclose(Q.T @ Q, np.eye(Rp), atol=1e-12)
        Xd = Q @ H.astype(np.float64) @ np.diag(s.astype(np.float64)) @ V.T.astype(np.float64)
        rp, col, val = X.subject(k)
        for i in range(D):
            c = col[rp[i]:rp[i + 1]]
            assert np.all(np.diff(c) > 0)
            assert np.allclose(val[rp[i]:rp[i + 1]], Xd[i, c].astype(np.float32), rtol=1e-6,
                               atol=1e-7 * np.abs(Xd).max())


@pytest.mark.parametrize("name,K,paper_mean_ik", [("p63m", 20000, 46.9), ("p500m", 4000, 99.3)])
def test_planted_statistics_match_the_paper(name, K, paper_mean_ik):
    w = synth.WORKLOADS[name]
    X = synth.generate(w.scaled(K))
    mean_ik = X.n_rows / X.K
    expected = w.dense_rows * (1.0 - np.exp(-w.J * w.keep_p))
    assert abs(mean_ik - expected) < 0.01 * expected
    assert abs(mean_ik - paper_mean_ik) < 0.01 * paper_mean_ik
    assert abs(X.nnz / X.K - w.dense_rows * w.J * w.keep_p) < 0.02 * w.dense_rows * w.J * w.keep_p
    # determinism: the same seed draws the same slices
    Y = synth.generate(w.scaled(K))
    assert np.array_equal(X.col, Y.col) and np.array_equal(X.val, Y.val)
