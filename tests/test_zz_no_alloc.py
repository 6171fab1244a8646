"""The allocation-free mode-1 entry point (p2_mode1_stats_noalloc).

Callers that cannot allocate device memory at the point of use (inside a
graph capture, in a real-time loop, under a host-managed memory arena) get
mode 1 and W^TW from their own device buffers.  This checks its result
against a host FP64 evaluation of the same sums from the same T, G and W:
M1 = sum_k (T_k G_k) * 1 W(k,:) (Eq. mttkrp1_3 with Y_k V = T_k G_k) and
W^TW, on two calls in a row (the second call reuses the shared fixed
scratch), and that the library's own iteration agrees.
"""
import numpy as np
import pytest

import synth
from tests.helpers import rel_fro

pytestmark = pytest.mark.gpu


def _host_gram(X, V):
    """Packed lower Gram Z_k^T Z_k of Z_k = X_k V for every subject (FP64)."""
    R = V.shape[1]
    P = R * (R + 1) // 2
    il = np.tril_indices(R)
    G = np.zeros((X.K, P))
    V64 = V.astype(np.float64)
    for k in range(X.K):
        rp, col, val = X.subject(k)
        Z = np.zeros((len(rp) - 1, R))
        for i in range(len(rp) - 1):
            a, b = rp[i], rp[i + 1]
            Z[i] = val[a:b].astype(np.float64) @ V64[col[a:b]]
        G[k] = (Z.T @ Z)[il]
    return G


def test_noalloc_mode1_matches_iteration_on_two_calls():
    torch = pytest.importorskip("torch")
    import paper_1703_04219_gb300 as p2
    X = synth.generate("c63m", K=2500)
    R = 10
    H0, V0, W0 = synth.init_factors(R, X.J, X.K, seed=4)
    dev = torch.device("cuda", 0)
    with p2.Parafac2(R) as m:
        m.load(X)
        m.init(H0, V0, W0)
        m.iterate(1)
        _, V, W = m.factors()
        T = m.procrustes()
        G = _host_gram(X, V)
        Td = torch.from_numpy(np.ascontiguousarray(T)).to(dev)
        Gd = torch.from_numpy(G).to(dev)
        Wd = torch.from_numpy(np.ascontiguousarray(W)).to(dev)
        outs = []
        for _ in range(2):
            M1 = torch.full((R, R), float("nan"), dtype=torch.float64, device=dev)
            WtW = torch.full((R, R), float("nan"), dtype=torch.float64, device=dev)
            p2.p2_mode1_stats_noalloc(X.K, R, Td, Gd, Wd, M1, WtW)
            torch.cuda.synchronize()
            outs.append((M1.cpu().numpy(), WtW.cpu().numpy()))
        m.iterate(1)
        M1_ref = m.mttkrp(1)       # mode 1 of the iteration that started from this state
    W64 = W.astype(np.float64)
    T64 = T.astype(np.float64)
    il = np.tril_indices(R)
    M1_host = np.zeros((R, R))
    for k in range(X.K):                       # sum_k (T_k G_k) * 1 w_k^T in FP64
        Gk = np.zeros((R, R))
        Gk[il] = G[k]
        Gk = Gk + np.tril(Gk, -1).T
        M1_host += (T64[k] @ Gk) * W64[k][None, :]
    for M1, WtW in outs:
        assert rel_fro(M1, M1_host) < 1e-5, rel_fro(M1, M1_host)
        assert rel_fro(WtW, W64.T @ W64) < 1e-12
    assert rel_fro(M1_ref, M1_host) < 1e-5, rel_fro(M1_ref, M1_host)
    assert np.array_equal(outs[0][0], outs[1][0])
    assert np.array_equal(outs[0][1], outs[1][1])


def test_noalloc_wrapper_rejects_wrong_buffers():
    """Host arrays, wrong dtypes and wrong sizes are refused before the call."""
    torch = pytest.importorskip("torch")
    import paper_1703_04219_gb300 as p2
    dev = torch.device("cuda", 0)
    K, R = 3, 4
    P_ = R * (R + 1) // 2
    T = torch.zeros((K, R, R), dtype=torch.float32, device=dev)
    G = torch.zeros((K, P_), dtype=torch.float64, device=dev)
    W = torch.zeros((K, R), dtype=torch.float32, device=dev)
    M1 = torch.zeros((R, R), dtype=torch.float64, device=dev)
    for bad in (dict(T=T.cpu()), dict(G=G.float()), dict(W=W[:2]), dict(M1=M1.cpu().numpy()),
                dict(WtW=torch.zeros((R, R + 1), dtype=torch.float64, device=dev))):
        args = dict(T=T, G=G, W=W, M1=M1, WtW=None)
        args.update(bad)
        with pytest.raises(ValueError):
            p2.p2_mode1_stats_noalloc(K, R, **args)


def test_noalloc_rejects_rank_beyond_scratch():
    torch = pytest.importorskip("torch")
    import paper_1703_04219_gb300 as p2
    dev = torch.device("cuda", 0)
    R = 17
    T = torch.zeros((1, R, R), dtype=torch.float32, device=dev)
    G = torch.zeros((1, R * (R + 1) // 2), dtype=torch.float64, device=dev)
    W = torch.zeros((1, R), dtype=torch.float32, device=dev)
    M1 = torch.zeros((R, R), dtype=torch.float64, device=dev)
    with pytest.raises(p2.P2Error) as ei:
        p2.p2_mode1_stats_noalloc(1, R, T, G, W, M1)
    assert ei.value.code == p2.P2_EINVAL
