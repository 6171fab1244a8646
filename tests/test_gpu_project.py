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
    """Two projectors on two streams: the same results as one at a time, and
    their device work overlaps.  Both batches (pinned host buffers, so a
    submit only validates and enqueues) are queued behind one gate event that
    a short bounded device sleep delays, so neither starts before both are
    enqueued; CUDA events bracket each batch on its own stream.  The two
    intervals intersect, and the pair finishes in well under the sum of the
    two batches' times run one after the other."""
    torch = pytest.importorskip("torch")
    m = _model(p2, 10)
    a, b = _requests(400, 2), _requests(400, 3)
    n_iter = 10
    pin = lambda x: torch.from_numpy(np.ascontiguousarray(x)).pin_memory()   # noqa: E731
    arrs = {id(r): [pin(x) for x in (r.subj_ptr, r.row_ptr, r.col, r.val)] for r in (a, b)}
    s0, s1, s2 = torch.cuda.Stream(), torch.cuda.Stream(), torch.cuda.Stream()
    pa = p2.Projector(m, 512, 40_000, 400_000, stream=s1.cuda_stream)
    pb = p2.Projector(m, 512, 40_000, 400_000, stream=s2.cuda_stream)
    ev = lambda: torch.cuda.Event(enable_timing=True)   # noqa: E731
    out = lambda r: torch.empty((r.K, 10), dtype=torch.float32).pin_memory()   # noqa: E731

    def run(pj, st, req, S):
        e0, e1 = ev(), ev()
        e0.record(st)
        pj.submit(req.K, *arrs[id(req)], n_iter, S)
        e1.record(st)
        return e0, e1

    Sa_ref, Sb_ref = out(a), out(b)
    for _ in range(2):                                  # warm-up, one at a time
        run(pa, s1, a, Sa_ref)
        pa.sync()
        run(pb, s2, b, Sb_ref)
        pb.sync()
    serial = []
    for _ in range(3):
        ta0, ta1 = run(pa, s1, a, Sa_ref)
        pa.sync()
        tb0, tb1 = run(pb, s2, b, Sb_ref)
        pb.sync()
        serial.append(ta0.elapsed_time(ta1) + tb0.elapsed_time(tb1))
    conc, intersect = [], []
    for _ in range(3):
        Sa, Sb = out(a), out(b)
        torch.cuda.synchronize()
        origin, gate = ev(), torch.cuda.Event()
        origin.record(s0)
        with torch.cuda.stream(s0):
            torch.cuda._sleep(20_000_000)               # ~10 ms: both batches get queued
        gate.record(s0)
        s1.wait_event(gate)
        s2.wait_event(gate)
        ta0, ta1 = run(pa, s1, a, Sa)
        tb0, tb1 = run(pb, s2, b, Sb)
        pa.sync()
        pb.sync()
        a0, a1 = origin.elapsed_time(ta0), origin.elapsed_time(ta1)
        b0, b1 = origin.elapsed_time(tb0), origin.elapsed_time(tb1)
        intersect.append(a0 < b1 and b0 < a1)
        conc.append(max(a1, b1) - min(a0, b0))
        assert torch.equal(Sa, Sa_ref) and torch.equal(Sb, Sb_ref)
    pa.close()
    pb.close()
    m.close()
    print(f"\nserial {min(serial):.3f} ms, concurrent {min(conc):.3f} ms")
    assert all(intersect)
    assert min(conc) < 0.85 * min(serial), (conc, serial)


def test_server_admits_by_device_memory(p2):
    """Slots sized from a device-memory budget (p2_projector_bytes): every
    launched batch fits the slot's capacities, the slot's projector takes no
    more than its share of the budget, a request larger than a slot is
    rejected, and the results equal the direct projection."""
    pytest.importorskip("torch")
    from paper_1703_04219_gb300.serve import Server, requests_from_slices
    m = _model(p2, 10)
    req = _requests(200, 6)
    budget = 3 * p2.p2_projector_bytes(m, 24, 24 * 66, 24 * 66 * 3)
    srv = Server(m, n_slots=3, max_subjects=64, n_iter=4, memory_bytes=budget,
                 shape=(33.0, 3.0), log_batches=True)
    adm = srv.admission
    cap = adm["capacity"]
    assert adm["slot_projector_bytes"] <= adm["slot_bytes"] == budget // 3
    assert p2.p2_projector_bytes(m, cap["subjects"], cap["rows"], cap["nnz"]) <= budget // 3
    reqs = requests_from_slices(req, rate_per_s=20000.0, seed=2)
    big = max(reqs, key=lambda r: r.rows)
    res, stats = srv.run(reqs)
    log = srv.batch_log
    srv.close()
    with p2.Projector(m, 256, 60_000, 400_000) as pj:
        S = pj.project(req, n_iter=4)
    m.close()
    assert stats["completed"] + stats["rejected"] == req.K
    for n, rows, nnz in log:
        assert n <= cap["subjects"] and rows <= cap["rows"] and nnz <= cap["nnz"]
    too_big = [r.rid for r in reqs if r.rows > cap["rows"] or r.nnz > cap["nnz"]]
    assert stats["rejected"] == len(too_big)
    if big.rows > cap["rows"]:
        assert big.rid not in res
    for k, s in res.items():
        assert np.array_equal(s, S[k]), k


def test_projector_bytes_matches_its_allocation(p2):
    torch = pytest.importorskip("torch")
    m = _model(p2, 10, K=100, iters=1)
    want = p2.p2_projector_bytes(m, 5000, 200_000, 2_000_000)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    pj = p2.Projector(m, 5000, 200_000, 2_000_000)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    pj.close()
    m.close()
    used = free0 - free1
    assert want - 4 * 2 ** 20 <= used <= want + 64 * 2 ** 20, (want, used)


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
