"""The split Procrustes step (p2_tuning.procrustes_split): a Householder
kernel stores Q_h and the tridiagonal, a one-lane-per-subject kernel runs
the QR iteration and records its Givens rotations, and a third kernel
applies them to Q_h and forms T_k; subjects whose rotations exceed the
record are finished by the fused kernel.  The arithmetic and its order are
the fused kernel's, so T_k, the factors and the MTTKRPs must be the same
bit for bit, with and without the fallback (a small record capacity), for
the lane-per-subject kernel (R <= 12) and the grouped kernel's
rank-compiled and generic instances (R > 12)."""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def p2():
    import paper_1703_04219_gb300 as mod
    return mod


@pytest.mark.parametrize("name,K,R", [("c250m", 3000, 40), ("c250m", 1500, 24),
                                      ("tiny", 150, 13), ("c250m", 800, 20), ("tiny", 80, 64),
                                      ("c63m", 5000, 10), ("tiny", 300, 5), ("c63m", 700, 12),
                                      ("tiny", 100, 2)])
def test_split_procrustes_is_bitwise_the_fused_kernel(p2, name, K, R):
    X = synth.generate(name, K=K)
    H0, V0, W0 = synth.init_factors(R, X.J, X.K, seed=23)
    outs = []
    for tune in (dict(procrustes_split=1), dict(procrustes_split=0),
                 dict(procrustes_split=1, split_record_cap=R * 4)):
        with p2.Parafac2(R) as m:
            m.set_tuning(**tune)
            m.load(X)
            m.init(H0, V0, W0)
            T0 = m.procrustes()
            fits = [m.iterate(1) for _ in range(2)]
            st = m.stats()
            outs.append(dict(T0=T0, T=m.procrustes(), F=m.factors(), M1=m.mttkrp(1),
                             fits=fits, flops=st["polar_fp64_flops"]))
    ref = outs[0]
    for o in outs[1:]:
        assert np.array_equal(o["T0"], ref["T0"]) and np.array_equal(o["T"], ref["T"])
        for a, b in zip(o["F"], ref["F"]):
            assert np.array_equal(a, b)
        assert np.array_equal(o["M1"], ref["M1"]) and o["fits"] == ref["fits"]
        assert o["flops"] == ref["flops"]


def test_autotuner_keeps_results_and_uses_its_cache(p2, tmp_path):
    """p2_options.autotune times the launch choices at the first iteration
    (split or fused Procrustes step, subject bins) and keeps the fastest;
    the results equal the untuned context's bit for bit, the choice is
    appended to the cache file, and a second context reads it from there."""
    X = synth.generate("c250m", K=4000)
    R = 40
    H0, V0, W0 = synth.init_factors(R, X.J, X.K, seed=29)
    cache = str(tmp_path / "tune.jsonl")
    outs, notes, tunes = [], [], []
    for kw in (dict(), dict(autotune=True, tune_cache=cache), dict(autotune=True, tune_cache=cache)):
        with p2.Parafac2(R, **kw) as m:
            m.load(X)
            m.init(H0, V0, W0)
            fit = m.iterate(2)
            outs.append((fit,) + m.factors())
            notes.append(m.tuning_note())
            tunes.append(m.tuning())
    for o in outs[1:]:
        assert o[0] == outs[0][0]
        for a, b in zip(o[1:], outs[0][1:]):
            assert np.array_equal(a, b)
    assert notes[0] == "" and notes[1].startswith("timed") and notes[2] == "cache"
    assert tunes[1] == tunes[2]
    lines = open(cache).read().strip().splitlines()
    assert len(lines) == 1 and '"key": "R=40' in lines[0]
