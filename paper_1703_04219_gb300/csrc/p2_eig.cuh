// Symmetric eigen-decomposition of one small FP64 matrix by one thread.
//
// Used by the Procrustes step (Section 3.2): with one GPU lane per subject,
// the R x R matrix A_k^T A_k is decomposed as Z diag(d) Z^T so that the
// polar factor's pseudo-inverse square root can be formed.
//
// Method (Golub & Van Loan, "Matrix Computations", 4th ed., Algorithms
// 5.1.1, 8.3.1 and 8.3.2): Householder reduction to tridiagonal form with
// backward accumulation of the orthogonal factor, then implicit symmetric QR
// steps with the Wilkinson shift and deflation, rotations accumulated into
// the eigenvector matrix.  Cost ~ (4/3) n^3 + O(n^2) rotations, versus the
// ~6 n^3 per sweep of cyclic Jacobi: FP64 issue slots are the scarce resource
// on this GPU, so the cheaper method wins.
//
// The matrix and vectors are reached through small accessor objects so the
// same code runs on interleaved shared memory (element e of thread t at
// base[e * stride + t]) on the GPU and on plain arrays on the host.
#pragma once

#ifndef P2_HD
#define P2_HD __host__ __device__ __forceinline__
#endif

#include <math.h>
#include <stdint.h>
#include <string.h>

namespace p2 {

struct MatView {
    double *base;
    int stride;
    int n;
    P2_HD double &operator()(int i, int j) const { return base[(size_t)(i * n + j) * stride]; }
};

struct VecView {
    double *base;
    int stride;
    P2_HD double &operator[](int i) const { return base[(size_t)i * stride]; }
};

P2_HD double p2_rsqrt(double x) {
#ifdef __CUDA_ARCH__
    return rsqrt(x);
#else
    return 1.0 / sqrt(x);
#endif
}

// Reduce the symmetric matrix held in the lower triangle of A (n x n) to
// tridiagonal form T = Q^T A Q, then overwrite A with Q (full storage).
// On return d[0..n) is diag(T) and e[0..n-1) its sub-diagonal.  Work space:
// d doubles as the Householder work vector during the reduction, and the
// Householder scalars beta_k are kept in the (unused) upper triangle at
// A(k, k+1) until the backward accumulation consumes them.
// N > 0 fixes n at compile time (n_rt is then ignored).
template <int N>
P2_HD void tridiagonalize(int n_rt, MatView A, VecView d, VecView e) {
    const int n = N > 0 ? N : n_rt;
    VecView t = d;
    for (int k = 0; k + 2 < n; ++k) {
        // Householder vector for x = A[k+1:n, k]
        double sigma = 0.0;
        for (int i = k + 2; i < n; ++i) sigma = fma(A(i, k), A(i, k), sigma);
        double x0 = A(k + 1, k);
        if (sigma == 0.0) {
            A(k, k + 1) = 0.0;      // beta_k
            e[k] = x0;
            continue;
        }
        double mu = sqrt(x0 * x0 + sigma);
        double v0 = (x0 <= 0.0) ? (x0 - mu) : (-sigma / (x0 + mu));
        double v02 = v0 * v0;
        double b = 2.0 * v02 / (sigma + v02);
        double inv_v0 = 1.0 / v0;
        for (int i = k + 2; i < n; ++i) A(i, k) *= inv_v0;     // v = [1, A(k+2:n,k)]
        A(k, k + 1) = b;
        e[k] = mu;
        // p = b * A22 v  (A22 symmetric, lower triangle stored), K = b/2 p^T v
        double pv = 0.0;
        for (int i = k + 1; i < n; ++i) {
            double s = A(i, k + 1);                           // v_{k+1} = 1
            for (int j = k + 2; j < n; ++j) {
                double aij = (j <= i) ? A(i, j) : A(j, i);
                s = fma(aij, A(j, k), s);
            }
            s *= b;
            t[i] = s;
            double vi = (i == k + 1) ? 1.0 : A(i, k);
            pv = fma(s, vi, pv);
        }
        double Kc = 0.5 * b * pv;
        for (int i = k + 1; i < n; ++i) {                      // w = p - K v
            double vi = (i == k + 1) ? 1.0 : A(i, k);
            t[i] = fma(-Kc, vi, t[i]);
        }
        for (int i = k + 1; i < n; ++i) {                      // A22 -= v w^T + w v^T
            double vi = (i == k + 1) ? 1.0 : A(i, k);
            double wi = t[i];
            for (int j = k + 1; j <= i; ++j) {
                double vj = (j == k + 1) ? 1.0 : A(j, k);
                A(i, j) = fma(-vi, t[j], fma(-wi, vj, A(i, j)));
            }
        }
    }
    if (n >= 2) e[n - 2] = A(n - 1, n - 2);
    for (int i = 0; i < n; ++i) d[i] = A(i, i);

    // Backward accumulation Q = P_0 P_1 ... P_{n-3}, in place.
    if (n == 1) {
        A(0, 0) = 1.0;
        return;
    }
    A(n - 1, n - 1) = 1.0;
    A(n - 2, n - 2) = 1.0;
    A(n - 1, n - 2) = 0.0;
    A(n - 2, n - 1) = 0.0;
    for (int k = n - 3; k >= 0; --k) {
        const double b = A(k, k + 1);
        A(k + 1, k + 1) = 1.0;
        for (int j = k + 2; j < n; ++j) {
            A(k + 1, j) = 0.0;
            A(j, k + 1) = 0.0;
        }
        if (b == 0.0) continue;
        for (int c = k + 1; c < n; ++c) {
            double s = A(k + 1, c);
            for (int i = k + 2; i < n; ++i) s = fma(A(i, k), A(i, c), s);
            s *= b;
            A(k + 1, c) -= s;
            for (int i = k + 2; i < n; ++i) A(i, c) = fma(-s, A(i, k), A(i, c));
        }
    }
    A(0, 0) = 1.0;
    for (int j = 1; j < n; ++j) {
        A(0, j) = 0.0;
        A(j, 0) = 0.0;
    }
}

// Binary exponent field of |v| (0 for zero and subnormals).
P2_HD int p2_expo(double v) {
#ifdef __CUDA_ARCH__
    return (__double2hiint(v) >> 20) & 0x7ff;
#else
    uint64_t b;
    memcpy(&b, &v, sizeof b);
    return (int)((b >> 52) & 0x7ff);
#endif
}

// Deflation test of a sub-diagonal entry ev of the tridiagonal, in integer
// arithmetic on binary exponents: negligible when expo(ev) <= expo(max(|d1|,
// |d2|)) - 52 or expo(ev) <= tiny_ex = expo(eps ||T||).  Either condition
// implies |ev| < 2 eps (|d1| + |d2|) or |ev| < 2 eps ||T||, i.e. a backward
// error of the order of the rounding already committed, and the test costs
// no FP64 instruction.
P2_HD bool p2_negligible(double ev, double d1, double d2, int tiny_ex) {
    const int x = p2_expo(ev);
    const int a = p2_expo(d1), b = p2_expo(d2);
    return x == 0 || x <= (a > b ? a : b) - 52 || x <= tiny_ex;
}

// Implicit symmetric QR with Wilkinson shift on the tridiagonal (d, e);
// rotations are accumulated into the columns of Z (n x n).  Returns the
// number of QR steps taken, or -1 if max_steps was exceeded (d then holds
// the current, partly converged, diagonal).  *rotations (if given) is
// incremented by the number of Givens rotations applied.  Each rotation is
// formed from one reciprocal square root: c = x / r, s = -z / r, r = t / sqrt(t)
// with t = x^2 + z^2.
template <int N>
P2_HD int tridiagonal_qr(int n_rt, MatView Z, VecView d, VecView e, int max_steps,
                         int *rotations = nullptr) {
    const int n = N > 0 ? N : n_rt;
    const double eps = 2.220446049250313e-16;
    double anorm = 0.0;
    for (int i = 0; i < n; ++i) {
        double r = fabs(d[i]) + ((i + 1 < n) ? fabs(e[i]) : 0.0) + ((i > 0) ? fabs(e[i - 1]) : 0.0);
        anorm = fmax(anorm, r);
    }
    const int tiny_ex = p2_expo(eps * anorm);
    int steps = 0;
    int q = n - 1;
    while (q > 0) {
        double eq = e[q - 1];
        if (p2_negligible(eq, d[q - 1], d[q], tiny_ex)) {
            e[q - 1] = 0.0;
            --q;
            continue;
        }
        int p = q - 1;
        while (p > 0) {
            if (p2_negligible(e[p - 1], d[p - 1], d[p], tiny_ex)) {
                e[p - 1] = 0.0;
                break;
            }
            --p;
        }
        if (++steps > max_steps) return -1;
        if (rotations) *rotations += q - p;
        // Wilkinson shift from the trailing 2 x 2 block
        double dd = 0.5 * (d[q - 1] - d[q]);
        double h = sqrt(dd * dd + eq * eq);
        double mu = d[q] - eq * eq / (dd + (dd >= 0.0 ? h : -h));
        double x = d[p] - mu;
        double z = e[p];
        for (int k = p; k < q; ++k) {
            const double tt = fma(x, x, z * z);
            double c = 1.0, s = 0.0, r = 0.0;
            if (tt > 0.0) {
                const double ir = p2_rsqrt(tt);
                c = x * ir;
                s = -z * ir;
                r = tt * ir;
            }
            if (k > p) e[k - 1] = r;
            double a = d[k], bb = d[k + 1], g = e[k];
            double cc = c * c, ss = s * s, cs = c * s;
            double cs2g = 2.0 * cs * g;
            d[k] = fma(cc, a, fma(ss, bb, -cs2g));
            d[k + 1] = fma(ss, a, fma(cc, bb, cs2g));
            e[k] = fma(cs, a - bb, (cc - ss) * g);
            if (k + 1 < q) {
                double en = e[k + 1];
                z = -s * en;
                e[k + 1] = c * en;
                x = e[k];
            }
            for (int i = 0; i < n; ++i) {
                double zk = Z(i, k), zk1 = Z(i, k + 1);
                Z(i, k) = fma(c, zk, -s * zk1);
                Z(i, k + 1) = fma(s, zk, c * zk1);
            }
        }
    }
    return steps;
}

}  // namespace p2
