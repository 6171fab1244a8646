"""Mode 2 in fixed point (p2_options.mode2_fixed_point, R <= 16), through the
C ABI: every non-zero's term x P_k(i, r) rounded at a per-component scale 2^S_r
taken from a bound on every column's sum, added with 64-bit integer atomics
(exact, so the order of the additions does not matter).

* one-step parity against the FP64 oracle (M2, V, W, fit) with it on and
  off, at R = 1, 5, 10, 16;
* the two agree to far below the FP32 rounding of the terms (1e-7);
* repeated runs and graph replay against eager launches are bitwise equal
  (integer sums in any order);
* values spanning 30 orders of magnitude across subjects: the bound keeps
  every partial sum in range (no error flag) and M2 still matches the oracle.
"""
import numpy as np
import pytest

import synth
from oracle import parafac2 as P
from tests.helpers import rel_fro

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def p2():
    import paper_1703_04219_gb300 as mod
    return mod


def _run(p2, X, R, fx, seed=11, n=1, **kw):
    H0, V0, W0 = synth.init_factors(R, X.J, X.K, seed=seed)
    with p2.Parafac2(R, mode2_fixed_point=fx, **kw) as m:
        m.load(X)
        m.init(H0, V0, W0)
        fit = m.iterate(n)
        return dict(fit=fit, M2=m.mttkrp(2), F=m.factors(), init=(H0, V0, W0))


@pytest.mark.parametrize("name,K,R", [("c63m", 3000, 10), ("c63m", 2000, 16), ("tiny", 200, 5),
                                      ("tiny", 200, 1)])
def test_fixed_point_mode2_matches_oracle_and_kahan(p2, name, K, R):
    X = synth.generate(name, K=K)
    on = _run(p2, X, R, True)
    off = _run(p2, X, R, False)
    H0, V0, W0 = on["init"]
    blocks = P.all_blocks(X)
    ref = P.als_iteration(blocks, H0.astype(np.float64), V0.astype(np.float64),
                          W0.astype(np.float64))
    assert rel_fro(on["M2"], ref["M2"]) < 1e-5
    for a, key in zip(on["F"], ("H", "V", "W")):
        assert rel_fro(a, ref[key]) < 1e-5, key
    assert abs(on["fit"] - P.fit_from_loss(ref["loss"], P.norm_x_sq(blocks))) < 1e-4
    assert rel_fro(on["M2"], off["M2"]) < 1e-7


def test_fixed_point_mode2_is_deterministic(p2):
    X = synth.generate("c63m", K=4000)
    runs = [_run(p2, X, 10, True, n=3, use_graph=g) for g in (True, True, False)]
    for r in runs[1:]:
        assert np.array_equal(r["M2"], runs[0]["M2"])
        for a, b in zip(r["F"], runs[0]["F"]):
            assert np.array_equal(a, b)
        assert r["fit"] == runs[0]["fit"]


def test_fixed_point_mode2_wide_value_range(p2):
    X = synth.generate("c63m", K=1500)
    scale = np.ones(X.nnz, np.float32)
    rng = np.random.default_rng(3)
    for k in range(X.K):                  # whole subjects scaled by 1e-15 .. 1e15
        a, b = X.row_ptr[X.subj_ptr[k]], X.row_ptr[X.subj_ptr[k + 1]]
        scale[a:b] = np.float32(10.0 ** rng.integers(-15, 16))
    Xs = synth.Slices(X.K, X.J, X.subj_ptr, X.row_ptr, X.col, (X.val * scale).astype(np.float32))
    on = _run(p2, Xs, 8, True)
    H0, V0, W0 = on["init"]
    ref = P.als_iteration(P.all_blocks(Xs), H0.astype(np.float64), V0.astype(np.float64),
                          W0.astype(np.float64))
    assert rel_fro(on["M2"], ref["M2"]) < 1e-5
