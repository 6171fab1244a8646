"""Double-word ("float-float") arithmetic and the double-word eigen-decomposition
that the Procrustes kernels run, compiled as plain C++ on the host
(tests/dw_host/dw_check.cpp) and pinned to mathematics that does not involve
them:

* every primitive against the exact rational result of its double-word
  operands (fractions.Fraction), within the normwise bounds of Joldes, Muller
  and Popescu (ACM TOMS 2017) for u = 2^-24, cancellation cases included;
* the Householder + implicit-QR decomposition M = Z diag(d) Z^T of symmetric
  matrices with adversarial spectra (condition numbers to 1e12, clusters,
  exact rank deficiency, diagonal and nearly diagonal inputs with
  sub-diagonals far below the FP32 normal range once squared): it must
  converge, Z must be orthogonal and Z diag(d) Z^T must reproduce M to a few
  2^-44 of ||M||, and d must match LAPACK's FP64 eigenvalues (numpy.linalg.eigvalsh)
  to the same normwise bound (Weyl's inequality);
* the same code compiled for FP64 (the opt-in FP64 arm) to a bound 16x
  tighter.
No GPU involved."""
import os
import shutil
import subprocess
from fractions import Fraction

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_1703_04219_gb300", "csrc")
U2 = Fraction(1, 2 ** 48)


@pytest.fixture(scope="module")
def exe(tmp_path_factory):
    if shutil.which("g++") is None:
        pytest.skip("g++ not available")
    out = str(tmp_path_factory.mktemp("dw") / "dw_check")
    subprocess.run(["g++", "-std=c++17", "-O1", "-ffp-contract=off", "-I", CSRC, "-o", out,
                    os.path.join(HERE, "dw_host", "dw_check.cpp")], check=True)
    return out


def _pair(rng, emin=-40, emax=40):
    """A normalised double-word: random sign and exponent, |l| <= ulp(h)/2."""
    h = np.float32(rng.uniform(1, 2) * 2.0 ** rng.integers(emin, emax) * rng.choice([-1, 1]))
    ulp = float(np.spacing(np.abs(h)))
    lo = np.float32(rng.uniform(-0.5, 0.5) * ulp)
    return float(h), float(lo)


def _fr(p):
    return Fraction(p[0]) + Fraction(p[1])


def _run_ops(exe, lines):
    r = subprocess.run([exe, "ops"], input="\n".join(lines) + "\n", capture_output=True,
                       text=True, check=True)
    return [tuple(float.fromhex(t) for t in ln.split()) for ln in r.stdout.strip().splitlines()]


def _isqrt_frac(x):
    """sqrt of a positive Fraction to ~2^-80 relative (enough to judge 2^-44)."""
    f = float(x)
    s = Fraction(np.sqrt(f))
    for _ in range(3):
        s = (s + x / s) / 2
    return s


def test_primitives_against_exact_rationals(exe):
    rng = np.random.default_rng(5)
    cases = []
    for _ in range(400):
        x, y, z = _pair(rng), _pair(rng), _pair(rng)
        cases.append((x, y, z))
    for _ in range(100):                                  # cancellation: y close to -x
        x = _pair(rng)
        y = (-x[0], float(np.float32(rng.uniform(-0.5, 0.5) * float(np.spacing(np.float32(abs(x[0])))))))
        cases.append((x, y, _pair(rng)))
    ops = ["add", "sub", "mul", "mulf", "sqr", "fma", "div", "sqrt", "rsqrt", "dot2", "acc"]
    lines = []
    for op in ops:
        for x, y, z in cases:
            if op in ("sqrt", "rsqrt"):
                x = (abs(x[0]), x[1] if x[0] > 0 else -x[1])
            lines.append(f"{op} {x[0].hex()} {x[1].hex()} {y[0].hex()} {y[1].hex()} "
                         f"{z[0].hex()} {z[1].hex()}")
    res = _run_ops(exe, lines)
    assert len(res) == len(lines)
    i = 0
    for op in ops:
        for x, y, z in cases:
            if op in ("sqrt", "rsqrt"):
                x = (abs(x[0]), x[1] if x[0] > 0 else -x[1])
            X, Y, Z = _fr(x), _fr(y), _fr(z)
            got = _fr(res[i])
            i += 1
            if op == "add":
                ref, scale, k = X + Y, abs(X) + abs(Y), 4
            elif op == "sub":
                ref, scale, k = X - Y, abs(X) + abs(Y), 4
            elif op == "mul":
                ref, scale, k = X * Y, abs(X * Y), 6
            elif op == "mulf":
                Yh = Fraction(y[0])
                ref, scale, k = X * Yh, abs(X * Yh), 4
            elif op == "sqr":
                ref, scale, k = X * X, X * X, 6
            elif op == "fma":
                ref, scale, k = X * Y + Z, abs(X * Y) + abs(Z), 8
            elif op == "div":
                ref, scale, k = X / Y, abs(X / Y), 16
            elif op == "sqrt":
                ref = _isqrt_frac(X)
                scale, k = ref, 8
            elif op == "rsqrt":
                ref = 1 / _isqrt_frac(X)
                scale, k = ref, 2 ** 6                     # one Newton step from ~2 ulp
            elif op == "dot2":
                ref, scale, k = X * Y + Z * X, abs(X * Y) + abs(Z * X), 8
            else:
                ref, scale, k = Y + X * Y + Z * X, abs(Y) + abs(X * Y) + abs(Z * X), 10
            assert abs(got - ref) <= k * U2 * scale, (op, x, y, z, float(abs(got - ref) / scale))


def _eig(exe, M, mode="eig"):
    n = M.shape[0]
    r = subprocess.run([exe, mode, str(n)], input="\n".join(repr(float(v)) for v in M.ravel()),
                       capture_output=True, text=True, check=True)
    vals = [float(t) for t in r.stdout.split()]
    steps = int(vals[0])
    d = np.array(vals[1:1 + n])
    Z = np.array(vals[1 + n:]).reshape(n, n)
    return steps, d, Z


def _spd(rng, lam):
    n = len(lam)
    Q, _ = np.linalg.qr(rng.standard_normal((n, n)))
    M = (Q * lam) @ Q.T
    M = (M + M.T) / 2
    return M / np.max(np.abs(np.diag(M))) if np.max(np.abs(np.diag(M))) > 0 else M


def _matrices():
    rng = np.random.default_rng(17)
    out = []
    for n in (1, 2, 3, 5, 10, 12, 17, 40):
        out.append((f"uniform{n}", _spd(rng, rng.uniform(0.1, 1.0, n))))
        out.append((f"geometric{n}", _spd(rng, np.geomspace(1.0, 1e-12, n))))
        if n >= 3:
            lam = rng.uniform(0.1, 1.0, n)
            lam[: n // 2] = lam[0]                          # a cluster of multiplicity n/2
            out.append((f"cluster{n}", _spd(rng, lam)))
            lam = rng.uniform(0.1, 1.0, n)
            lam[: n // 2] = 0.0                             # exact rank deficiency
            out.append((f"rankdef{n}", _spd(rng, lam)))
            out.append((f"diagonal{n}", np.diag(rng.uniform(0.1, 1.0, n))))
            for tiny in (1e-21, 1e-25, 1e-30):             # squares below FP32's normal range
                T = np.diag(rng.uniform(0.1, 1.0, n))
                off = tiny * rng.uniform(0.5, 1.0, n - 1)
                T += np.diag(off, -1) + np.diag(off, 1)
                if n >= 5:
                    T[n - 1, 0] = T[0, n - 1] = tiny
                out.append((f"tiny{tiny:g}_{n}", T))
            lam = np.geomspace(1.0, 1e-6, n)                 # geometric with tiny couplings
            T = np.diag(lam) + np.diag(np.full(n - 1, 1e-22), -1) + np.diag(np.full(n - 1, 1e-22), 1)
            out.append((f"gradedtiny{n}", T))
    return out


@pytest.mark.parametrize("name,M", _matrices(), ids=[m[0] for m in _matrices()])
def test_eigen_decomposition_against_lapack(exe, name, M):
    n = M.shape[0]
    steps, d, Z = _eig(exe, M)
    assert steps >= 0, f"{name}: no convergence"
    assert np.all(np.isfinite(d)) and np.all(np.isfinite(Z)), name
    nrm = max(np.abs(np.linalg.eigvalsh(M)).max(), np.finfo(float).tiny)
    bound = 2.0 ** -42 * n
    assert np.abs(Z.T @ Z - np.eye(n)).max() <= bound, (name, np.abs(Z.T @ Z - np.eye(n)).max())
    assert np.abs((Z * d) @ Z.T - M).max() <= bound * nrm, (name, np.abs((Z * d) @ Z.T - M).max())
    ref = np.linalg.eigvalsh(M)
    assert np.abs(np.sort(d) - ref).max() <= bound * nrm, (name, np.abs(np.sort(d) - ref).max())


@pytest.mark.parametrize("name,M", _matrices(), ids=[m[0] for m in _matrices()])
def test_fp64_eigen_decomposition_against_lapack(exe, name, M):
    """The same Householder + QR code compiled for FP64 (the opt-in FP64 arm
    of the Procrustes step): a few 2^-50 n normwise, 16x tighter than the
    double-word bound above."""
    n = M.shape[0]
    steps, d, Z = _eig(exe, M, "eig64")
    assert steps >= 0, f"{name}: no convergence"
    assert np.all(np.isfinite(d)) and np.all(np.isfinite(Z)), name
    nrm = max(np.abs(np.linalg.eigvalsh(M)).max(), np.finfo(float).tiny)
    bound = 2.0 ** -46 * n
    assert np.abs(Z.T @ Z - np.eye(n)).max() <= bound, (name, np.abs(Z.T @ Z - np.eye(n)).max())
    assert np.abs((Z * d) @ Z.T - M).max() <= bound * nrm, (name, np.abs((Z * d) @ Z.T - M).max())
    ref = np.linalg.eigvalsh(M)
    assert np.abs(np.sort(d) - ref).max() <= bound * nrm, (name, np.abs(np.sort(d) - ref).max())
