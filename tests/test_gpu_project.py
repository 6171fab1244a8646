"""Projection of new subjects onto a fitted model (serving) against the oracle."""
import numpy as np
import pytest

import synth
from oracle import parafac2 as P
from tests.helpers import rel_fro

pytestmark = pytest.mark.gpu

EPS32 = 2.0 ** -24


@pytest.fixture(scope="module")
def p2():
    import paper_1703_04219_gb300 as mod
    return mod


def _model(p2, R, K=400, iters=3):
    X = synth.generate("c63m", K=K)
    H0, V0, W0 = synth.init_factors(R, X.J, X.K, seed=31)
    m = p2.Parafac2(R)
    m.load(X)
    m.init(H0, V0, W0)
    m.iterate(iters)
    return m


def _requests(n, seed_shift=0):
    w = synth.WORKLOADS["serve"]
    from dataclasses import replace
    return synth.generate(replace(w, K=n, seed=w.seed + seed_shift))


@pytest.mark.parametrize("R,n_iter,tol", [(10, 1, 1e-5), (10, 8, 1e-4), (8, 5, 1e-4)])
def test_projection_matches_oracle(p2, R, n_iter, tol):
    m = _model(p2, R)
    H, V, _ = m.factors()
    req = _requests(40)
    with p2.Projector(m, 64, 10_000, 100_000) as pj:
        S, T = pj.project(req, n_iter=n_iter, want_T=True)
    m.close()
    H64, V64 = H.astype(np.float64), V.astype(np.float64)
    ref_S = np.zeros_like(S, dtype=np.float64)
    for k in range(req.K):
        Xc, cols = P.subject_block(req, k)
        s, Q = P.project_subject(Xc, cols, H64, V64, n_iter)
        ref_S[k] = s
        # Q from the GPU transform: Q = X V T^T (on X's non-zero columns).  FP32
        # storage of Z = X V perturbs a polar factor by ~eps32 * sigma_1 / sigma_min,
        # so the per-subject bound scales with the conditioning of A = X V S H^T.
        Qg = Xc @ V64[cols] @ T[k].astype(np.float64).T
        sg = S[k].astype(np.float64)                  # the Q-step the GPU took at its own s
        Q = P.procrustes_q(Xc, cols, H64, V64, sg)
        A = Xc @ V64[cols] @ np.diag(sg) @ H64.T
        sv = np.linalg.svd(A, compute_uv=False)
        kept = sv[sv > 1e-5 * sv[0]] if sv.size and sv[0] > 0 else sv[:0]
        if kept.size:
            cond = kept[0] / kept[-1]
            assert rel_fro(Qg, Q) < 1e-5 + 1e-6 * cond, (k, rel_fro(Qg, Q), cond)
    # Per subject, the error of s scales with the conditioning of A_k = X V S H^T:
    # Z = X V, T and G are FP32, i.e. A_k is perturbed by ~eps32 ||A_k||, and the
    # orthogonal polar factor moves by ||dQ|| <= 2 ||dA|| / sigma_min (first-order
    # perturbation of the polar decomposition), so each projection step adds up to
    # ~2 eps32 cond(A_k) relative error and the bound allows 4 eps32 cond(A_k) per
    # step.  Well-conditioned subjects must meet the FP32 tolerance.
    well = []
    for k in range(req.K):
        Xc, cols = P.subject_block(req, k)
        A0 = Xc @ V64[cols] @ H64.T                       # s = 1 at the first step
        sv = np.linalg.svd(A0, compute_uv=False)
        sv = sv[sv > 1e-5 * sv[0]]
        cond = sv[0] / sv[-1]
        err = rel_fro(S[k], ref_S[k])
        assert err < max(tol, 1e-6) + 4 * EPS32 * cond * n_iter, (k, err, cond)
        if cond < 100:
            well.append(k)
    assert len(well) >= 5
    assert rel_fro(S[well], ref_S[well]) < tol, rel_fro(S[well], ref_S[well])


def test_result_is_the_same_alone_and_in_the_mix(p2):
    m = _model(p2, 10)
    req = _requests(60, seed_shift=1)
    with p2.Projector(m, 64, 20_000, 200_000) as pj:
        S_mix = pj.project(req, n_iter=6)
        alone = [pj.project(req.take([k]), n_iter=6)[0] for k in (0, 17, 59)]
    m.close()
    for got, k in zip(alone, (0, 17, 59)):
        assert np.array_equal(got, S_mix[k])


def test_concurrent_projectors_overlap_and_agree(p2):
    torch = pytest.importorskip("torch")
    m = _model(p2, 10)
    a, b = _requests(50, 2), _requests(50, 3)
    with p2.Projector(m, 64, 20_000, 200_000) as pj:
        Sa_ref = pj.project(a, n_iter=5)
        Sb_ref = pj.project(b, n_iter=5)
    s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()
    pa = p2.Projector(m, 64, 20_000, 200_000, stream=s1.cuda_stream)
    pb = p2.Projector(m, 64, 20_000, 200_000, stream=s2.cuda_stream)
    outs = []
    for pj, req in ((pa, a), (pb, b)):
        arrs = [np.ascontiguousarray(x) for x in (req.subj_ptr, req.row_ptr, req.col, req.val)]
        S = np.empty((req.K, 10), np.float32)
        pj.submit(req.K, *arrs, 5, S)
        outs.append((arrs, S))
    pa.sync()
    pb.sync()
    pa.close()
    pb.close()
    m.close()
    assert np.array_equal(outs[0][1], Sa_ref)
    assert np.array_equal(outs[1][1], Sb_ref)


def test_projection_rejects_malformed_requests(p2):
    m = _model(p2, 4, K=50, iters=1)
    req = _requests(5, 4)
    bad = req.col.copy()
    bad[2] = 10 ** 6
    with p2.Projector(m, 8, 2000, 20000) as pj:
        S = np.empty((req.K, 4), np.float32)
        with pytest.raises(p2.P2Error) as ei:
            pj.submit(req.K, req.subj_ptr, req.row_ptr, bad, req.val, 2, S)
        assert ei.value.code == p2.P2_EINVAL
        with pytest.raises(p2.P2Error):
            pj.submit(100, req.subj_ptr, req.row_ptr, req.col, req.val, 2, S)   # over capacity
    m.close()


def test_server_continuous_batching_matches_direct_projection(p2):
    pytest.importorskip("torch")
    from paper_1703_04219_gb300.serve import Server, requests_from_slices
    m = _model(p2, 10)
    req = _requests(300, 5)
    reqs = requests_from_slices(req, rate_per_s=20000.0, seed=1)
    srv = Server(m, n_slots=3, max_subjects=32, max_rows=8000, max_nnz=60000, n_iter=6)
    res, stats = srv.run(reqs)
    srv.close()
    with p2.Projector(m, 400, 60_000, 400_000) as pj:
        S = pj.project(req, n_iter=6)
    m.close()
    assert stats["completed"] + stats["rejected"] == req.K
    assert stats["batches"] >= 3 and stats["p99_ms"] >= stats["p50_ms"] > 0
    for k, s in res.items():
        assert np.array_equal(s, S[k]), k


def test_projection_onto_nonneg_model(p2):
    """A model trained in the non-negative variant (Section 5.1) projects new
    subjects with s >= 0 solved by NNLS; one step from s = 1 against the
    oracle for the well-conditioned subjects, as the other tests."""
    R = 10
    X = synth.generate("c63m", K=400)
    H0, V0, W0 = synth.init_factors(R, X.J, X.K, seed=31)
    with p2.Parafac2(R, nonneg=True) as m:
        m.load(X)
        m.init(H0, V0, W0)
        m.iterate(3)
        H, V, _ = m.factors()
        req = _requests(200)
        with p2.Projector(m, 256, 20_000, 200_000) as pj:
            S = pj.project(req, n_iter=1)
    assert np.all(S >= 0)
    H64, V64 = H.astype(np.float64), V.astype(np.float64)
    good = 0
    for k in range(req.K):
        Xc, cols = P.subject_block(req, k)
        s, _ = P.project_subject(Xc, cols, H64, V64, 1, nonneg=True)
        A = Xc @ V64[cols] @ H64.T
        sv = np.linalg.svd(A, compute_uv=False)
        sv = sv[sv > 1e-5 * sv[0]]
        if sv.size and sv[0] / sv[-1] < 100:
            assert rel_fro(S[k], s) < 1e-4, (k, rel_fro(S[k], s))
            good += 1
    assert good >= 5
