"""One case on the CPU-emulated library (run in a subprocess with the
AddressSanitizer runtime preloaded).  Prints one JSON line of relative
errors against the FP64 oracle."""
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import paper_1703_04219_gb300 as p2  # noqa: E402
import synth  # noqa: E402
from oracle import parafac2 as P  # noqa: E402
from tests.helpers import rel_fro, slices_from_dense  # noqa: E402

p2.LIB_PATH = os.path.join(HERE, "_build", "libp2emu.so")
p2.lib = p2._load()


def bf16_round(a):
    """Round float32 values to the nearest bfloat16 (ties to even), as float32."""
    u = np.ascontiguousarray(a, dtype=np.float32).view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) >> 16 << 16
    return u.astype(np.uint32).view(np.float32).reshape(np.shape(a))


def iterate_case(name, K, R, precision="fp32"):
    nonneg = precision == "nonneg"
    fp64 = precision == "fp64"                # the FP64 arm of the Procrustes step
    dup = precision == "dupcols"              # singular Gram-Hadamard products
    if nonneg or fp64 or dup:
        precision = "fp32"
    X = synth.generate(name, K=K)
    H0, V0, W0 = synth.init_factors(R, X.J, X.K, seed=11)
    if dup:
        # column 1 of V and W equal to column 0: every R x R Gram-Hadamard
        # product is singular, so the pseudo-inverses take the Jacobi path
        V0[:, 1] = V0[:, 0]
        W0[:, 1] = W0[:, 0]
    if precision == "bf16":                # a start that bfloat16 storage represents exactly
        V0 = bf16_round(V0)
    with p2.Parafac2(R, use_graph=False, precision=precision, nonneg=nonneg,
                     fp64_procrustes=fp64) as m:
        m.load(X)
        m.init(H0, V0, W0)
        fit = m.iterate(1)
        H, V, W = m.factors()
        M = {n: m.mttkrp(n) for n in (1, 2, 3)}
    ref = P.als_iteration(P.all_blocks(X), H0.astype(np.float64), V0.astype(np.float64),
                          W0.astype(np.float64), nonneg=nonneg)
    err = {key: rel_fro(M[mode], ref[key]) for mode, key in ((1, "M1"), (2, "M2"), (3, "M3"))}
    if nonneg:
        err["neg"] = float(min(V.min(), W.min()) < 0)
    err.update({key: rel_fro(v, ref[key]) for key, v in (("H", H), ("V", V), ("W", W))})
    err["fit"] = abs(fit - P.fit_from_loss(ref["loss"], P.norm_x_sq(P.all_blocks(X))))
    return err


def project_case(R, n_req, nonneg=False):
    from dataclasses import replace
    X = synth.generate("c63m", K=30)
    H0, V0, W0 = synth.init_factors(R, X.J, X.K, seed=31)
    with p2.Parafac2(R, use_graph=False, nonneg=nonneg) as m:
        m.load(X)
        m.init(H0, V0, W0)
        m.iterate(1)
        H, V, _ = m.factors()
        w = synth.WORKLOADS["serve"]
        req = synth.generate(replace(w, K=n_req, seed=w.seed))
        with p2.Projector(m, 8, 4000, 40000) as pj:
            S = pj.project(req, n_iter=2)
    errs = []
    for k in range(req.K):
        Xc, cols = P.subject_block(req, k)
        s, _ = P.project_subject(Xc, cols, H.astype(np.float64), V.astype(np.float64), 2,
                                 nonneg=nonneg)
        errs.append(rel_fro(S[k], s))
    return {"S_max": float(max(errs))}


def getu_case(R, k0, k1):
    """U_k = Q_k H for subjects k0 .. k1-1 against the oracle's Procrustes
    factor for the factors the library returns."""
    X = synth.generate("tiny", K=24)
    H0, V0, W0 = synth.init_factors(R, X.J, X.K, seed=11)
    with p2.Parafac2(R, use_graph=False) as m:
        m.load(X)
        m.init(H0, V0, W0)
        m.iterate(1)
        H, V, W = m.factors()
        U = m.U(k0, k1)
    H, V, W = (a.astype(np.float64) for a in (H, V, W))
    refs = []
    for k in range(k0, k1):
        Xc, cols = P.subject_block(X, k)
        refs.append(P.procrustes_q(Xc, cols, H, V, W[k]) @ H)
    ref = np.concatenate(refs, axis=0) if refs else np.zeros((0, R))
    assert U.shape == ref.shape, (U.shape, ref.shape)
    return {"U": rel_fro(U, ref), "rows": float(U.shape[0])}


def seed_case(R, seed):
    """p2_init with no factors draws H, V, W from the context's seed exactly as
    the input generator's init_factors does; p2_iterate_until runs max_iter
    iterations with tol = 0 (reproducing a fixed-count run) and stops after
    the second when every change is within tol."""
    X = synth.generate("tiny", K=24)
    with p2.Parafac2(R, use_graph=False, seed=seed) as m:
        m.load(X)
        m.init()
        H, V, W = m.factors()
        n, fit = m.iterate_until(3, 0.0)
    H0, V0, W0 = synth.init_factors(R, X.J, X.K, seed=seed)
    same = float(np.array_equal(H, H0) and np.array_equal(V, V0) and np.array_equal(W, W0))
    with p2.Parafac2(R, use_graph=False) as m:
        m.load(X)
        m.init(H0, V0, W0)
        fit_fixed = m.iterate(3)
        n_loose, _ = m.iterate_until(10, 10.0)
    return {"init_equal": same, "n": float(n), "fit": fit, "fit_fixed": fit_fixed,
            "n_loose": float(n_loose)}


def rational_case(R, K):
    """p2_init_eig for a fixed 12 products (tol 0) with the product split into
    several column passes: H = I, W = 1, V orthonormal and close to the
    oracle's leading eigenvectors (12 products at this spectrum's rate leave
    a sine of ~1e-3; full convergence is checked on the GPU); one iteration
    from the stored start against the oracle's iteration from the same
    state; and a rank-deficient input (3 non-zero columns of 8, R = 5) whose
    null-space columns are an orthonormal completion."""
    X = synth.generate("tiny", K=K)
    blocks = P.all_blocks(X)
    _, Vref, _, _ = P.rational_start(blocks, X.K, X.J, R)
    # 16 KiB reported free: the product's N x w scratch gets a quarter, so
    # the block's columns go through in several passes (a ragged last one)
    os.environ["EMU_FREE_BYTES"] = "16384"
    with p2.Parafac2(R, use_graph=False) as m:
        m.load(X)
        n = m.init_eig(max_iter=12, tol=0.0)
        H, V, W = m.factors()
        fit = m.iterate(1)
        H1, V1, W1 = m.factors()
        # an argument error leaves the context as it was: it still iterates
        try:
            m.init_eig(max_iter=0)
            einval = 0.0
        except p2.P2Error as e:
            einval = float(e.code == p2.P2_EINVAL)
        still = float(np.isfinite(m.iterate(1)))
    del os.environ["EMU_FREE_BYTES"]
    V64 = V.astype(np.float64)
    ref = P.als_iteration(blocks, np.eye(R), V64, np.ones((X.K, R)))
    nx2 = P.norm_x_sq(blocks)
    sin2 = float(np.sum((V64 - Vref @ (Vref.T @ V64)) ** 2))
    rng = np.random.default_rng(5)
    mats = []
    for _ in range(6):
        d = np.zeros((4, 8))
        d[:, :3] = rng.uniform(0.5, 2.0, (4, 3))
        mats.append(d)
    Xd = slices_from_dense(mats, J=8)
    with p2.Parafac2(5, use_graph=False) as m:
        m.load(Xd)
        nd = m.init_eig(max_iter=50, tol=1e-9)
        _, Vd, _ = m.factors()
        fitd = m.iterate(1)
    _, Vd0, _, _ = P.rational_start(P.all_blocks(Xd), Xd.K, Xd.J, 5)
    Vd = Vd.astype(np.float64)
    return {"n": n, "H_eye": float(np.array_equal(H, np.eye(R, dtype=np.float32))),
            "W_one": float(np.all(W == 1.0)), "orth": float(np.abs(V64.T @ V64 - np.eye(R)).max()),
            "sin2": sin2, "H1": rel_fro(H1, ref["H"]), "V1": rel_fro(V1, ref["V"]),
            "W1": rel_fro(W1, ref["W"]), "fit": abs(fit - P.fit_from_loss(ref["loss"], nx2)),
            "def_n": nd, "def_orth": float(np.abs(Vd.T @ Vd - np.eye(5)).max()),
            "def_lead": rel_fro(Vd[:, :3], Vd0[:, :3]), "def_fit_finite": float(np.isfinite(fitd)),
            "einval": einval, "still_iterates": still}


def tc_case(R, K):
    """The tensor-core formation of M' (p2_options.tensor_core_m: digits of
    8 bits on the emulated tensor core, exact FP32 accumulation) against the
    double-word formation on the FP32 pipe: T_k of the first Q-step and the
    factors after one iteration close to each other and to the oracle, with
    the split step, the fused kernel and the split step's fallback."""
    X = synth.generate("tiny", K=K)
    H0, V0, W0 = synth.init_factors(R, X.J, X.K, seed=41)
    ref = P.als_iteration(P.all_blocks(X), H0.astype(np.float64), V0.astype(np.float64),
                          W0.astype(np.float64))
    out = {}
    runs = {}
    for name, tc, tune in (("dw", False, dict(procrustes_split=1)),
                           ("tc", True, dict(procrustes_split=1)),
                           ("tc_fused", True, dict(procrustes_split=0)),
                           ("tc_fallback", True, dict(procrustes_split=1, split_record_cap=R))):
        with p2.Parafac2(R, use_graph=False, tensor_core_m=tc) as m:
            m.set_tuning(**tune)
            m.load(X)
            m.init(H0, V0, W0)
            T0 = m.procrustes()
            fit = m.iterate(1)
            runs[name] = (T0, fit) + m.factors()
    for name in ("dw", "tc", "tc_fused", "tc_fallback"):
        T0, fit, H, V, W = runs[name]
        out[f"{name}_T0_vs_dw"] = rel_fro(T0, runs["dw"][0])
        out[f"{name}_W"] = rel_fro(W, ref["W"])
        out[f"{name}_V"] = rel_fro(V, ref["V"])
        out[f"{name}_H"] = rel_fro(H, ref["H"])
    out["tc_paths_bitwise"] = float(all(np.array_equal(a, b) for n in ("tc_fused", "tc_fallback")
                                        for a, b in zip(runs["tc"], runs[n])))
    return out


def split_case(R, K):
    """The split Procrustes step (QR recorder) against the fused kernel, and
    with a record capacity small enough that most subjects go to the fused
    fallback: T_k and the factors bitwise equal after one iteration."""
    X = synth.generate("tiny", K=K)
    H0, V0, W0 = synth.init_factors(R, X.J, X.K, seed=17)
    outs = []
    for tune in (dict(procrustes_split=1), dict(procrustes_split=0),
                 dict(procrustes_split=1, split_record_cap=R)):
        with p2.Parafac2(R, use_graph=False) as m:
            m.set_tuning(**tune)
            m.load(X)
            m.init(H0, V0, W0)
            T0 = m.procrustes()
            m.iterate(1)
            outs.append((T0, m.procrustes()) + m.factors())
    same = all(np.array_equal(a, b) for o in outs[1:] for a, b in zip(outs[0], o))
    return {"bitwise": float(same)}


def blocks_case(R, K):
    """The mode-2 pass over many row blocks (a tiny block size) against one
    block: M2, V and the fit equal to round-off (the partial sums are added
    in another order), and both against the oracle."""
    X = synth.generate("tiny", K=K)
    H0, V0, W0 = synth.init_factors(R, X.J, X.K, seed=19)
    outs = []
    for kib in (0, 1):
        with p2.Parafac2(R, use_graph=False) as m:
            m.set_tuning(m2_block_kib=kib)
            m.load(X)
            m.init(H0, V0, W0)
            fit = m.iterate(1)
            outs.append((fit, m.mttkrp(2), m.factors()[1]))
    ref = P.als_iteration(P.all_blocks(X), H0.astype(np.float64), V0.astype(np.float64),
                          W0.astype(np.float64))
    return {"M2_blocks": rel_fro(outs[1][1], outs[0][1]), "V_blocks": rel_fro(outs[1][2], outs[0][2]),
            "M2": rel_fro(outs[1][1], ref["M2"]), "V": rel_fro(outs[1][2], ref["V"]),
            "fit": abs(outs[1][0] - outs[0][0])}


def shard_case(R, K):
    """A context whose exchange hook doubles every buffer (the sum over two
    shards that hold the same subjects) against an unsharded context on the
    collection stacked twice: same H, V and fit, and W rows equal to the
    first copy's.  Exercises the sharded load (column counts, ||X||^2), the
    statistics row and the M2 exchange under AddressSanitizer (device
    buffers are host memory on the emulator)."""
    import ctypes
    X = synth.generate("tiny", K=K)
    X2 = X.take(list(range(K)) + list(range(K)))
    H0, V0, W0 = synth.init_factors(R, X.J, X.K, seed=13)
    calls = []

    def double(ptr, count, stream):
        buf = (ctypes.c_double * count).from_address(ptr)
        a = np.frombuffer(buf, dtype=np.float64)
        a *= 2.0
        calls.append(count)

    with p2.Parafac2(R, use_graph=False) as m:
        m.set_exchange(double)
        m.load(X)
        m.init(H0, V0, W0)
        fit = m.iterate(2)
        H, V, W = m.factors()
        M2 = m.mttkrp(2)
    with p2.Parafac2(R, use_graph=False) as m:
        m.load(X2)
        m.init(H0, V0, np.vstack([W0, W0]))
        fit2 = m.iterate(2)
        H2, V2, W2 = m.factors()
        M22 = m.mttkrp(2)
    P_ = R * R * 2 + 1
    want = [X.J + 1] + [P_, X.J * R, P_, X.J * R, P_]   # load, prologue, 2 x (M2, stats)
    return {"H": rel_fro(H, H2), "V": rel_fro(V, V2), "W": rel_fro(W, W2[:K]),
            "M2": rel_fro(M2, M22), "fit": abs(fit - fit2),
            "calls_ok": float(calls == want)}


if __name__ == "__main__":
    kind = sys.argv[1]
    if kind == "iterate":
        out = iterate_case(sys.argv[2], int(sys.argv[3]), int(sys.argv[4]),
                           sys.argv[5] if len(sys.argv) > 5 else "fp32")
    elif kind == "seed":
        out = seed_case(int(sys.argv[2]), int(sys.argv[3]))
    elif kind == "rational":
        out = rational_case(int(sys.argv[2]), int(sys.argv[3]))
    elif kind == "blocks":
        out = blocks_case(int(sys.argv[2]), int(sys.argv[3]))
    elif kind == "tc":
        out = tc_case(int(sys.argv[2]), int(sys.argv[3]))
    elif kind == "split":
        out = split_case(int(sys.argv[2]), int(sys.argv[3]))
    elif kind == "shard":
        out = shard_case(int(sys.argv[2]), int(sys.argv[3]))
    elif kind == "getu":
        out = getu_case(int(sys.argv[2]), int(sys.argv[3]), int(sys.argv[4]))
    else:
        out = project_case(int(sys.argv[2]), int(sys.argv[3]),
                           len(sys.argv) > 4 and sys.argv[4] == "nonneg")
    print(json.dumps({k: float(v) for k, v in out.items()}), flush=True)
