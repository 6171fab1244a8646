"""Parity on 1% subject subsamples of the full workloads, through the C ABI.

K = 10,000 subjects (the first 10,000 of each workload's seed stream) of the
63M-non-zero workload at R = 10 and of the 250M- and 555M-non-zero workloads
at R = 40 (Table 1's R = 10 and R = 40 columns), against the FP64 oracle run
over subject chunks in worker processes (oracle.pool, the unchanged
per-subject functions of Algorithms 2 and 3):

* one step from the same FP32 start: M1, M2, M3, H, V and W within relative
  Frobenius 1e-5 (FP32 storage) or 3e-3 (bfloat16 storage of V and P_k, from
  a start bfloat16 represents exactly), fit within 1e-4;
* ten iterations from the same start (FP32 storage): the fit within 1e-4 of
  the oracle's after every iteration.

The measured errors are printed (pytest -s shows them).
"""
import numpy as np
import pytest

import synth
from oracle import parafac2 as P
from oracle.pool import OraclePool
from tests.helpers import rel_fro

pytestmark = pytest.mark.gpu

K_SUB = 10_000
FIT_TOL = 1e-4


@pytest.fixture(scope="module")
def p2():
    import paper_1703_04219_gb300 as mod
    return mod


@pytest.fixture(scope="module")
def pools():
    cache = {}

    def get(name):
        if name not in cache:
            X = synth.generate(name, K=K_SUB)
            cache[name] = (X, OraclePool(X))
        return cache[name]

    yield get
    for _, pool in cache.values():
        pool.close()


def bf16_round(a):
    u = np.ascontiguousarray(a, dtype=np.float32).view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) >> 16 << 16
    return u.astype(np.uint32).view(np.float32).reshape(np.shape(a))


@pytest.mark.parametrize("name,R,precision", [("c63m", 10, "fp32"), ("c250m", 40, "fp32"),
                                              ("c555m", 40, "fp32"), ("c250m", 40, "bf16")])
def test_subsample_one_step_parity(p2, pools, name, R, precision):
    X, pool = pools(name)
    H0, V0, W0 = synth.init_factors(R, X.J, X.K, seed=11)
    if precision == "bf16":
        V0 = bf16_round(V0)
    with p2.Parafac2(R, precision=precision) as m:
        m.load(X)
        m.init(H0, V0, W0)
        fit = m.iterate(1)
        H, V, W = m.factors()
        M = {n: m.mttkrp(n) for n in (1, 2, 3)}
    ref = pool.iteration(H0, V0, W0)
    tol = 3e-3 if precision == "bf16" else 1e-5
    errs = {}
    for mode, key in ((1, "M1"), (2, "M2"), (3, "M3")):
        errs[key] = rel_fro(M[mode], ref[key])
    for key, v in (("H", H), ("V", V), ("W", W)):
        errs[key] = rel_fro(v, ref[key])
    errs["fit"] = abs(fit - P.fit_from_loss(ref["loss"], pool.norm_x_sq))
    print(f"\n{name} K={X.K} R={R} {precision} one-step errors: " +
          ", ".join(f"{k} {v:.2e}" for k, v in errs.items()))
    for key in ("M1", "M2", "M3", "H", "V", "W"):
        assert errs[key] < tol, (key, errs[key])
    assert errs["fit"] < FIT_TOL


@pytest.mark.parametrize("name,R", [("c63m", 10), ("c250m", 40), ("c555m", 40)])
def test_subsample_ten_iterations_fit(p2, pools, name, R):
    X, pool = pools(name)
    H0, V0, W0 = synth.init_factors(R, X.J, X.K, seed=12)
    with p2.Parafac2(R) as m:
        m.load(X)
        m.init(H0, V0, W0)
        fits = [m.iterate(1) for _ in range(10)]
        H, V, W = m.factors()
    ref = pool.parafac2_als(H0, V0, W0, n_iter=10)
    ref_fits = [h["fit"] for h in ref["history"]]
    diffs = [abs(a - b) for a, b in zip(fits, ref_fits)]
    print(f"\n{name} K={X.K} R={R} ten iterations: max fit difference {max(diffs):.2e}, "
          f"final fit {fits[-1]:.6f} (oracle {ref_fits[-1]:.6f}); factors after ten: " +
          ", ".join(f"{k} {rel_fro(v, ref[k]):.2e}" for k, v in (("H", H), ("V", V), ("W", W))))
    assert max(diffs) < FIT_TOL, diffs
