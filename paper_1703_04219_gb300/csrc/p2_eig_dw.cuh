// Symmetric eigen-decomposition of one small matrix by one thread, in
// double-word arithmetic (p2_dw.cuh) or, for the opt-in FP64 arm, in FP64
// (p2_num.cuh): the code is written once for a number type D.
//
// Used by the Procrustes step (Section 3.2): with one GPU lane per subject,
// the R x R matrix A_k^T A_k is decomposed as Z diag(d) Z^T so that the
// polar factor's pseudo-inverse square root can be formed.
//
// Method (Golub & Van Loan, "Matrix Computations", 4th ed., Algorithms
// 5.1.1, 8.3.1 and 8.3.2): Householder reduction to tridiagonal form with
// backward accumulation of the orthogonal factor, then implicit symmetric QR
// steps with the Wilkinson shift and deflation, rotations accumulated into
// the eigenvector matrix.  Both halves are normwise backward stable, so the
// arithmetic's normwise error bounds (a few 2^-48 for double-words, a few
// 2^-53 in FP64) carry over to the decomposition.
//
// The matrix and vectors are reached through accessor objects so the same
// code runs on interleaved shared memory (element e of thread t at
// base[e * stride + t]) on the GPU and on plain arrays on the host.
#pragma once

#include "p2_num.cuh"

namespace p2 {

template <class D = dw>
struct DwMat {
    D *base;
    int stride;
    int n;
    P2_HD D &operator()(int i, int j) const { return base[(size_t)(i * n + j) * stride]; }
};

template <class D = dw>
struct DwVec {
    D *base;
    int stride;
    P2_HD D &operator[](int i) const { return base[(size_t)i * stride]; }
};

// Reduce the symmetric matrix held in the lower triangle of A (n x n) to
// tridiagonal form T = Q^T A Q, then overwrite A with Q (full storage).
// On return d[0..n) is diag(T) and e[0..n-1) its sub-diagonal.  d serves as
// the Householder work vector during the reduction, and the Householder
// scalars beta_k are kept in the (unused) upper triangle at A(k, k+1) until
// the backward accumulation consumes them.  N > 0 fixes n at compile time.
template <int N, class D>
P2_HD void tridiagonalize_dw(int n_rt, DwMat<D> A, DwVec<D> d, DwVec<D> e) {
    const int n = N > 0 ? N : n_rt;
    const D one = num_f<D>(1.f), zero = num_f<D>(0.f);
    DwVec<D> t = d;
#pragma unroll 1
    for (int k = 0; k + 2 < n; ++k) {
        // Householder reflector P = I - b v v^T with P x = beta e_1 for
        // x = A[k+1:n, k], in the normalisation that squares no small
        // quantity: beta = -sign(x0) ||x||, b = (beta - x0) / beta in [1, 2],
        // v = [1, x(2:) / (x0 - beta)] with |v_i| <= 1.  A column whose part
        // below x0 has squared norm under the type's tiny2 (entries below ~2^-48
        // of the scaled matrix's unit norm) is left as it is, a perturbation
        // of the order of the rounding, so every square stays in range.
        acc_t<D> sg = acc0<D>();
        for (int i = k + 2; i < n; ++i) acc_sqr(sg, A(i, k));
        const D sigma = acc_val(sg);
        const D x0 = A(k + 1, k);
        if (!(sigma.h >= NumT<D>::tiny2())) {
            A(k, k + 1) = zero;     // b_k
            e[k] = x0;
            continue;
        }
        acc_t<D> m2 = acc_from(sigma);
        acc_sqr(m2, x0);
        const D mu = dw_sqrt(acc_val(m2));
        const D beta = (x0.h >= 0.f) ? dw_neg(mu) : mu;
        const D b = dw_div(dw_sub(beta, x0), beta);
        const D inv_v0 = dw_recip(dw_sub(x0, beta));
        for (int i = k + 2; i < n; ++i) A(i, k) = dw_mul(A(i, k), inv_v0);
        A(k, k + 1) = b;
        e[k] = beta;
        // p = b A22 v (A22 symmetric, lower triangle stored), K = b/2 p^T v;
        // rows in pairs (two independent sums interleaved), pv in row order
        acc_t<D> pv = acc0<D>();
        int i2 = k + 1;
        for (; i2 + 1 < n; i2 += 2) {
            const int i = i2;
            acc_t<D> s0 = acc_from(A(i, k + 1));         // v_{k+1} = 1
            acc_t<D> s1 = acc_from(A(i + 1, k + 1));
            for (int j = k + 2; j < n; ++j) {
                const D vj = A(j, k);
                acc_fma(s0, (j <= i) ? A(i, j) : A(j, i), vj);
                acc_fma(s1, (j <= i + 1) ? A(i + 1, j) : A(j, i + 1), vj);
            }
            const D si0 = dw_mul(acc_val(s0), b);
            const D si1 = dw_mul(acc_val(s1), b);
            t[i] = si0;
            t[i + 1] = si1;
            if (i == k + 1)
                acc_add(pv, si0);
            else
                acc_fma(pv, si0, A(i, k));
            acc_fma(pv, si1, A(i + 1, k));
        }
        if (i2 < n) {
            const int i = i2;
            acc_t<D> s = acc_from(A(i, k + 1));
            for (int j = k + 2; j < n; ++j) acc_fma(s, (j <= i) ? A(i, j) : A(j, i), A(j, k));
            const D si = dw_mul(acc_val(s), b);
            t[i] = si;
            if (i == k + 1)
                acc_add(pv, si);
            else
                acc_fma(pv, si, A(i, k));
        }
        const D nK = dw_neg(dw_mul(dw_scale(b, 0.5f), acc_val(pv)));
        t[k + 1] = dw_add(t[k + 1], nK);                 // w = p - K v
        for (int i = k + 2; i < n; ++i) t[i] = dw_fma(nK, A(i, k), t[i]);
        for (int i = k + 1; i < n; ++i) {                // A22 -= v w^T + w v^T
            const D nvi = dw_neg((i == k + 1) ? one : A(i, k));
            const D nwi = dw_neg(t[i]);
            {                                            // j = k + 1: v_{k+1} = 1
                acc_t<D> a = acc_from(A(i, k + 1));
                acc_fma(a, nvi, t[k + 1]);
                acc_add(a, nwi);
                A(i, k + 1) = acc_val(a);
            }
            int j = k + 2;
            for (; j + 1 <= i; j += 2) {                 // entries in pairs
                acc_t<D> a0 = acc_from(A(i, j));
                acc_t<D> a1 = acc_from(A(i, j + 1));
                acc_fma(a0, nvi, t[j]);
                acc_fma(a1, nvi, t[j + 1]);
                acc_fma(a0, nwi, A(j, k));
                acc_fma(a1, nwi, A(j + 1, k));
                A(i, j) = acc_val(a0);
                A(i, j + 1) = acc_val(a1);
            }
            if (j <= i) {
                acc_t<D> a = acc_from(A(i, j));
                acc_fma(a, nvi, t[j]);
                acc_fma(a, nwi, A(j, k));
                A(i, j) = acc_val(a);
            }
        }
    }
    if (n >= 2) e[n - 2] = A(n - 1, n - 2);
    for (int i = 0; i < n; ++i) d[i] = A(i, i);

    // Backward accumulation Q = P_0 P_1 ... P_{n-3}, in place.
    if (n == 1) {
        A(0, 0) = one;
        return;
    }
    A(n - 1, n - 1) = one;
    A(n - 2, n - 2) = one;
    A(n - 1, n - 2) = zero;
    A(n - 2, n - 1) = zero;
#pragma unroll 1
    for (int k = n - 3; k >= 0; --k) {
        const D b = A(k, k + 1);
        A(k + 1, k + 1) = one;
        for (int j = k + 2; j < n; ++j) {
            A(k + 1, j) = zero;
            A(j, k + 1) = zero;
        }
        if (b.h == 0.f) continue;
        // column k+1 is e_{k+1}: its update is 1 - b and -b v_i
        const D nb = dw_neg(b);
        A(k + 1, k + 1) = dw_add(one, nb);
        for (int i = k + 2; i < n; ++i) A(i, k + 1) = dw_mul(nb, A(i, k));
        int c = k + 2;
        for (; c + 1 < n; c += 2) {                      // columns in pairs
            acc_t<D> s0 = acc0<D>(), s1 = acc0<D>();     // A(k+1, c) = 0 here
            for (int i = k + 2; i < n; ++i) {
                const D vi = A(i, k);
                acc_fma(s0, vi, A(i, c));
                acc_fma(s1, vi, A(i, c + 1));
            }
            const D ns0 = dw_mul(acc_val(s0), nb);
            const D ns1 = dw_mul(acc_val(s1), nb);
            A(k + 1, c) = ns0;
            A(k + 1, c + 1) = ns1;
            for (int i = k + 2; i < n; ++i) {
                const D vi = A(i, k);
                A(i, c) = dw_fma(ns0, vi, A(i, c));
                A(i, c + 1) = dw_fma(ns1, vi, A(i, c + 1));
            }
        }
        if (c < n) {
            acc_t<D> s = acc0<D>();
            for (int i = k + 2; i < n; ++i) acc_fma(s, A(i, k), A(i, c));
            const D ns = dw_mul(acc_val(s), nb);
            A(k + 1, c) = ns;
            for (int i = k + 2; i < n; ++i) A(i, c) = dw_fma(ns, A(i, k), A(i, c));
        }
    }
    A(0, 0) = one;
    for (int j = 1; j < n; ++j) {
        A(0, j) = zero;
        A(j, 0) = zero;
    }
}

// Implicit symmetric QR with Wilkinson shift on the tridiagonal (d, e);
// rotations are accumulated into the columns of Z (n x n, n <= 64).  Returns
// the number of QR steps taken, or -1 if max_steps was exceeded (d then holds
// the current, partly converged, diagonal).  *rotations (if given) is
// incremented by the number of Givens rotations applied.
//
// One flat loop, one Givens rotation per trip, so that the lanes of a warp
// run the same instructions whatever their sweep boundaries:
//  * the deflation tests of all n - 1 sub-diagonal positions are taken at
//    once into a bit mask, and the bottom q of the active block and its top p
//    follow from leading-zero counts (no serial scan);
//  * the Wilkinson shift of that block is formed on every trip and used by
//    the lanes that start a sweep;
//  * the trip that forms rotation k applies rotation k - 1 to Z (the pending
//    rotation, carried over sweep boundaries and flushed at the end): its
//    columns are loaded at the top of the trip and everything is stored at
//    the bottom, so the serial scalar recurrence and the vector work are free
//    to overlap.
// Each rotation is formed from one reciprocal square root: c = x / r,
// s = -z / r, r = t / sqrt(t) with t = x^2 + z^2, after scaling (x, z) by a
// power of two so that t cannot underflow (FP32's exponent range is far
// narrower than FP64's, and the converging sub-diagonal and the bulge can
// both become tiny).
template <int N, class D>
P2_HD int tridiagonal_qr_dw(int n_rt, DwMat<D> Z, DwVec<D> d, DwVec<D> e, int max_steps,
                            int *rotations = nullptr) {
    constexpr int NA = N > 0 ? N : 64;                   // register-array bound
    const int n = N > 0 ? N : n_rt;
    const D one = num_f<D>(1.f), zero = num_f<D>(0.f);
    if (n < 2) return 0;
    float an = 0.f;
    for (int i = 0; i < n; ++i) {
        float r = fabsf(d[i].h);
        if (i + 1 < n) r += fabsf(e[i].h);
        if (i > 0) r += fabsf(e[i - 1].h);
        an = fmaxf(an, r);
    }
    const int tiny_ex = f_expo(an) - NumT<D>::deflate_bits;
    int steps = 0, rot = 0, status = 0;
    int q = n - 1, p = 0, kr = 0;
    bool sweeping = false;
    D x = zero, z = zero, dk = zero, ek = zero;
    int kp = 0;
    D cp = one, sp = zero;
    // bit i: e[i] negligible against d[i], d[i + 1].  Taken for every position
    // once; afterwards a trip re-tests only the positions whose d or e it
    // wrote (the others keep their inputs, hence their bits).
    unsigned long long nm = 0;
#pragma unroll
    for (int i = 0; i + 1 < NA; ++i)
        if (i + 1 < n && dw_negligible(e[i], d[i], d[i + 1], tiny_ex)) nm |= 1ull << i;
    auto retest = [&](int i) {
        if (i >= 0 && i + 1 < n) {
            const unsigned long long b = 1ull << i;
            nm = dw_negligible(e[i], d[i], d[i + 1], tiny_ex) ? (nm | b) : (nm & ~b);
        }
    };
#pragma unroll 1
    while (true) {
        D za[NA], zb[NA];                               // pending rotation's columns
#pragma unroll
        for (int i = 0; i < NA; ++i)
            if (i < n) {
                za[i] = Z(i, kp);
                zb[i] = Z(i, kp + 1);
            }
        // ---- the block a new sweep would take, and its shift ----------------
        const unsigned long long nn = ~nm & ((1ull << q) - 1);
        const int qn = nn ? 64 - p2_clz64(nn) : 0;        // top non-negligible position + 1
        const unsigned long long nb = qn > 1 ? nm & ((1ull << (qn - 1)) - 1) : 0ull;
        const int pn = nb ? 64 - p2_clz64(nb) : 0;        // top of the unreduced block
        const int qs = qn > 0 ? qn : 1;
        const D eq = e[qs - 1];
        const D dd = dw_scale(dw_sub(d[qs - 1], d[qs]), 0.5f);
        acc_t<D> hh = acc0<D>();
        acc_sqr(hh, dd);
        acc_sqr(hh, eq);
        const D h = dw_sqrt(acc_val(hh));
        const D den = (dd.h >= 0.f) ? dw_add(dd, h) : dw_sub(dd, h);
        const D den_s = den.h != 0.f ? den : one;        // (qn = 0 only: value unused)
        const D mu = dw_sub(d[qs], dw_div(dw_sqr(eq), den_s));
        const D dpn = d[pn], epn = e[pn];
        bool clear_top = false;
        if (!sweeping) {
            if (qn == 0) break;
            if (++steps > max_steps) {
                status = -1;
                break;
            }
            q = qn;
            p = pn;
            rot += q - p;
            dk = dpn;
            ek = epn;
            x = dw_sub(dpn, mu);
            z = epn;
            kr = p;
            sweeping = true;
            clear_top = p > 0;
        }
        // ---- rotation kr -----------------------------------------------------
        const D bb = d[kr + 1];
        const D en = (kr + 1 < q) ? e[kr + 1] : zero;
        const int exx = f_expo(x.h), exz = f_expo(z.h);
        const int ex = exx > exz ? exx : exz;
        const bool nz = ex > 0;
        const float xsc = f_pow2(127 - ex);
        const D xs = dw_scale(x, xsc), zs = dw_scale(z, xsc);
        acc_t<D> ta = acc0<D>();
        acc_sqr(ta, xs);
        acc_sqr(ta, zs);
        const D tt = acc_val(ta);
        const D ir = dw_rsqrt(nz ? tt : one);
        const D c = nz ? dw_mul(xs, ir) : one;
        const D s = nz ? dw_neg(dw_mul(zs, ir)) : zero;
        const D r = nz ? dw_scale(dw_mul(tt, ir), f_pow2(ex - 127)) : zero;
        const D cc = dw_sqr(c), ss = dw_sqr(s), cs = dw_mul(c, s);
        const D cs2g = dw_scale(dw_mul(cs, ek), 2.f);
        acc_t<D> a0 = acc_from(dw_neg(cs2g));
        acc_fma(a0, cc, dk);
        acc_fma(a0, ss, bb);
        const D dkn = acc_val(a0);
        acc_t<D> a1 = acc_from(cs2g);
        acc_fma(a1, ss, dk);
        acc_fma(a1, cc, bb);
        const D dk1 = acc_val(a1);
        acc_t<D> a2 = acc0<D>();
        acc_fma(a2, cs, dw_sub(dk, bb));
        acc_fma(a2, dw_sub(cc, ss), ek);
        const D ekn = acc_val(a2);
        // ---- pending rotation on columns kp, kp + 1, then all stores ----------
        {
            const D nsp = dw_neg(sp);
#pragma unroll
            for (int i = 0; i < NA; ++i)
                if (i < n) {
                    const D a = dw_dot2(cp, za[i], nsp, zb[i]);
                    const D b = dw_dot2(sp, za[i], cp, zb[i]);
                    Z(i, kp) = a;
                    Z(i, kp + 1) = b;
                }
        }
        if (clear_top) e[p - 1] = zero;
        if (kr > p) e[kr - 1] = r;
        d[kr] = dkn;
        kp = kr;
        cp = c;
        sp = s;
        const int kw = kr;                                // the positions this trip wrote
        if (++kr < q) {
            z = dw_neg(dw_mul(s, en));
            ek = dw_mul(c, en);
            x = ekn;
            dk = dk1;
        } else {
            d[q] = dk1;
            e[q - 1] = ekn;
            sweeping = false;
            retest(q - 1);
            retest(q);
        }
        retest(kw - 1);
        retest(kw);
        if (clear_top) retest(p - 1);
    }
    {   // flush the last rotation
        const D nsp = dw_neg(sp);
        for (int i = 0; i < n; ++i) {
            const D za = Z(i, kp), zb = Z(i, kp + 1);
            Z(i, kp) = dw_dot2(cp, za, nsp, zb);
            Z(i, kp + 1) = dw_dot2(sp, za, cp, zb);
        }
    }
    if (rotations) *rotations += rot;
    return status < 0 ? -1 : steps;
}

}  // namespace p2
