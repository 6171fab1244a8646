// Procrustes kernel for larger R: eight lanes per subject (see below).
// Included by p2_polar_grp.cu; needs MatView and p2_rsqrt (p2_eig.cuh), the
// flop helpers (p2_polar.cuh), SmallState and FLAG_EIG_NOCONV.
#pragma once

namespace p2 {

// ---------------------------------------------------------------------------
// Larger R (up to 64): a group of PG = 8 lanes per subject, four subjects per
// warp.  A lane-per-subject kernel would need R^2 doubles of shared memory per
// lane (12.8 KB at R = 40), so only ~17 subjects would fit on an SM and the
// FP64 pipe would issue mostly empty warps.  Here the R x R working matrix of
// a subject lives once in shared memory and its eight lanes split the vector
// work by rows (or columns); the scalar parts of the Householder and QR steps
// run redundantly on the eight lanes of a group, so a warp instruction still
// serves four subjects.  Same mathematics, tolerances and output as above.
//
// Per subject: A (R x LD, LD = R | 1 to spread banks), d, e, t, w (R each).
// RB = R rounded up to a multiple of PG (register arrays); rows i are owned
// by lane i % PG.
constexpr int PG = 8;

inline __host__ __device__ int grp_ld(int R) { return R | 1; }
inline __host__ __device__ size_t grp_doubles(int R) {
    return (size_t)R * grp_ld(R) + 4 * (size_t)R;
}

template <int RB>
__global__ void __launch_bounds__(256, 1) k_polar_grp(const double *__restrict__ G,
                                                      const float *__restrict__ W, SmallState *st,
                                                      float *T, int64_t K, int R, double rtol2,
                                                      int spb) {
    constexpr int RPL = RB / PG;                     // rows per lane
    extern __shared__ __align__(16) double sm[];
    const int lane = threadIdx.x & 31;
    const int gl = lane & (PG - 1);
    const unsigned gmask = 0xffu << (lane & ~(PG - 1));
    const int slot = (threadIdx.x >> 3);
    const int64_t k = (int64_t)blockIdx.x * spb + slot;
    const double *__restrict__ H = st->H64;
    unsigned long long flops = 0;
    if (slot < spb && k < K) {
        const int LD = grp_ld(R);
        double *base = sm + (size_t)slot * grp_doubles(R);
        MatView A{base, 1, LD};                      // A(i, j) = base[i * LD + j]
        double *d = base + (size_t)R * LD;
        double *e = d + R;
        double *t = e + R;
        double *wv = t + R;
        const double *Gk = G + (size_t)k * (R * (R + 1) / 2);
        for (int i = gl; i < R; i += PG) wv[i] = (double)W[(size_t)k * R + i];
        __syncwarp(gmask);

        // ---- M = H B H^T with B = S G S ------------------------------------
        // U = B H^T, row by row in place (row i of B is held in registers).
#pragma unroll 1
        for (int ii = 0; ii < RPL; ++ii) {
            const int i = gl + PG * ii;
            if (i >= R) break;
            double b[RB];
            const double wi = wv[i];
#pragma unroll
            for (int j = 0; j < RB; ++j) {
                if (j < R) {
                    const int p = (j <= i) ? (i * (i + 1) / 2 + j) : (j * (j + 1) / 2 + i);
                    b[j] = Gk[p] * (wi * wv[j]);
                }
            }
#pragma unroll 1
            for (int c = 0; c < R; ++c) {
                double s = 0.0;
#pragma unroll
                for (int j = 0; j < RB; ++j)
                    if (j < R) s = fma(b[j], __ldg(&H[c * R + j]), s);
                A(i, c) = s;
            }
        }
        __syncwarp(gmask);
        // M = H U, column by column in place (lower triangle).
#pragma unroll 1
        for (int c = 0; c < R; ++c) {
            double u[RB];
#pragma unroll
            for (int i = 0; i < RB; ++i)
                if (i < R) u[i] = A(i, c);
            __syncwarp(gmask);
#pragma unroll 1
            for (int ii = 0; ii < RPL; ++ii) {
                const int r = gl + PG * ii;
                if (r >= R) break;
                if (r < c) continue;
                double s = 0.0;
#pragma unroll
                for (int i = 0; i < RB; ++i)
                    if (i < R) s = fma(__ldg(&H[r * R + i]), u[i], s);
                A(r, c) = s;
            }
            __syncwarp(gmask);
        }

        // ---- Householder tridiagonalisation (lower triangle) --------------
#pragma unroll 1
        for (int kk = 0; kk + 2 < R; ++kk) {
            double sig = 0.0;
            for (int i = gl; i < R; i += PG)
                if (i >= kk + 2) sig = fma(A(i, kk), A(i, kk), sig);
            sig += __shfl_xor_sync(gmask, sig, 4);
            sig += __shfl_xor_sync(gmask, sig, 2);
            sig += __shfl_xor_sync(gmask, sig, 1);
            const double x0 = A(kk + 1, kk);
            if (sig == 0.0) {
                __syncwarp(gmask);
                if (gl == 0) {
                    A(kk, kk + 1) = 0.0;
                    e[kk] = x0;
                }
                __syncwarp(gmask);
                continue;
            }
            const double mu = sqrt(fma(x0, x0, sig));
            const double v0 = (x0 <= 0.0) ? (x0 - mu) : (-sig / (x0 + mu));
            const double v02 = v0 * v0;
            const double bh = 2.0 * v02 / (sig + v02);
            const double inv_v0 = 1.0 / v0;
            __syncwarp(gmask);
            for (int i = gl; i < R; i += PG)
                if (i >= kk + 2) A(i, kk) *= inv_v0;
            if (gl == 0) {
                A(kk, kk + 1) = bh;
                e[kk] = mu;
            }
            __syncwarp(gmask);
            // p = bh * A22 v on my rows, pv = p . v
            double pv = 0.0;
            for (int i = gl; i < R; i += PG) {
                if (i < kk + 1) continue;
                double s = A(i, kk + 1);
                for (int j = kk + 2; j < R; ++j) {
                    const double aij = (j <= i) ? A(i, j) : A(j, i);
                    s = fma(aij, A(j, kk), s);
                }
                s *= bh;
                t[i] = s;
                pv = fma(s, (i == kk + 1) ? 1.0 : A(i, kk), pv);
            }
            pv += __shfl_xor_sync(gmask, pv, 4);
            pv += __shfl_xor_sync(gmask, pv, 2);
            pv += __shfl_xor_sync(gmask, pv, 1);
            const double Kc = 0.5 * bh * pv;
            for (int i = gl; i < R; i += PG)
                if (i >= kk + 1) t[i] = fma(-Kc, (i == kk + 1) ? 1.0 : A(i, kk), t[i]);
            __syncwarp(gmask);
            for (int i = gl; i < R; i += PG) {
                if (i < kk + 1) continue;
                const double vi = (i == kk + 1) ? 1.0 : A(i, kk);
                const double wi = t[i];
                A(i, kk + 1) = fma(-vi, t[kk + 1], A(i, kk + 1) - wi);
                for (int j = kk + 2; j <= i; ++j)
                    A(i, j) = fma(-vi, t[j], fma(-wi, A(j, kk), A(i, j)));
            }
            __syncwarp(gmask);
        }
        if (gl == 0 && R >= 2) e[R - 2] = A(R - 1, R - 2);
        for (int i = gl; i < R; i += PG) d[i] = A(i, i);
        __syncwarp(gmask);
        // backward accumulation of Q = P_0 ... P_{R-3}, columns split over lanes
        if (R == 1) {
            if (gl == 0) A(0, 0) = 1.0;
        } else {
            if (gl == 0) {
                A(R - 1, R - 1) = 1.0;
                A(R - 2, R - 2) = 1.0;
                A(R - 1, R - 2) = 0.0;
                A(R - 2, R - 1) = 0.0;
            }
            __syncwarp(gmask);
#pragma unroll 1
            for (int kk = R - 3; kk >= 0; --kk) {
                const double bh = A(kk, kk + 1);
                __syncwarp(gmask);
                for (int j = gl; j < R; j += PG) {
                    if (j == kk + 1) {
                        A(kk + 1, kk + 1) = 1.0;
                        for (int i = kk + 2; i < R; ++i) A(i, kk + 1) = 0.0;
                    } else if (j > kk + 1) {
                        A(kk + 1, j) = 0.0;
                    }
                }
                __syncwarp(gmask);
                if (bh != 0.0) {
                    for (int c = gl; c < R; c += PG) {
                        if (c < kk + 1) continue;
                        double s = A(kk + 1, c);
                        for (int i = kk + 2; i < R; ++i) s = fma(A(i, kk), A(i, c), s);
                        s *= bh;
                        A(kk + 1, c) -= s;
                        for (int i = kk + 2; i < R; ++i) A(i, c) = fma(-s, A(i, kk), A(i, c));
                    }
                }
                __syncwarp(gmask);
            }
            for (int j = gl; j < R; j += PG) {
                if (j == 0) {
                    A(0, 0) = 1.0;
                } else {
                    A(0, j) = 0.0;
                    A(j, 0) = 0.0;
                }
            }
        }
        __syncwarp(gmask);

        // ---- implicit QR with Wilkinson shift; rotations on my rows of Z ----
        // One flat loop, one Givens rotation per trip, so that the four
        // groups of a warp execute the rotation body together whatever their
        // sweep boundaries.  The scalar recurrence runs on all eight lanes
        // (identical values); d[k+1] and e[k+1] of a sweep are read before
        // anything writes them and d[k], e[k] are carried in registers.
        // Deflation tests compare binary exponents in integer arithmetic
        // (p2_negligible).
        const double eps = 2.220446049250313e-16;
        double an = 0.0;
        for (int i = gl; i < R; i += PG) {
            double r = fabs(d[i]);
            if (i + 1 < R) r += fabs(e[i]);
            if (i > 0) r += fabs(e[i - 1]);
            an = fmax(an, r);
        }
        an = fmax(an, __shfl_xor_sync(gmask, an, 4));
        an = fmax(an, __shfl_xor_sync(gmask, an, 2));
        an = fmax(an, __shfl_xor_sync(gmask, an, 1));
        const int tiny_ex = p2_expo(eps * an);
        int steps = 0, rot = 0;
        const int max_steps = 30 * R;
        int q = R - 1, p = 0, kr = 0;
        bool sweeping = false, failed = false;
        double x = 0.0, z = 0.0, dk = 0.0, ek = 0.0;
        // Software pipelining: a trip computes the Givens scalars of rotation
        // kr and applies rotation kr - 1 (kp, cp, sp) to the lanes' rows of Z;
        // the two are independent, so the serial scalar chain overlaps FP64
        // work.  A sweep starts with the identity pending and flushes its last
        // rotation when it ends.
        int kp = 0;
        double cp = 1.0, sp = 0.0;
#pragma unroll 1
        while (true) {
            if (!sweeping) {
                while (q > 0 && p2_negligible(e[q - 1], d[q - 1], d[q], tiny_ex)) --q;
                if (q == 0) break;
                p = q - 1;
                while (p > 0 && !p2_negligible(e[p - 1], d[p - 1], d[p], tiny_ex)) --p;
                if (++steps > max_steps) {
                    failed = true;
                    break;
                }
                rot += q - p;
                const double eq = e[q - 1];
                const double dd = 0.5 * (d[q - 1] - d[q]);
                const double h = sqrt(fma(dd, dd, eq * eq));
                const double mu = d[q] - eq * eq / (dd + (dd >= 0.0 ? h : -h));
                dk = d[p];
                ek = e[p];
                x = dk - mu;
                z = ek;
                kr = p;
                kp = p;
                cp = 1.0;
                sp = 0.0;
                sweeping = true;
                __syncwarp(gmask);
                if (gl == 0 && p > 0) e[p - 1] = 0.0;
            }
            const double bb = d[kr + 1];
            const double en = (kr + 1 < q) ? e[kr + 1] : 0.0;
            __syncwarp(gmask);
            double za[RPL], zb[RPL];
#pragma unroll
            for (int ii = 0; ii < RPL; ++ii) {
                const int i = gl + PG * ii;
                if (i < R) {
                    za[ii] = A(i, kp);
                    zb[ii] = A(i, kp + 1);
                }
            }
            const double tt = fma(x, x, z * z);
            const bool nz = tt > 0.0;
            const double ir = p2_rsqrt(nz ? tt : 1.0);
            const double c = nz ? x * ir : 1.0;
            const double s = nz ? -z * ir : 0.0;
            const double r = nz ? tt * ir : 0.0;
            if (kr > p) e[kr - 1] = r;
            const double cc = c * c, ss = s * s, cs = c * s;
            const double cs2g = 2.0 * cs * ek;
            d[kr] = fma(cc, dk, fma(ss, bb, -cs2g));
            const double dk1 = fma(ss, dk, fma(cc, bb, cs2g));
            const double ekn = fma(cs, dk - bb, (cc - ss) * ek);
#pragma unroll
            for (int ii = 0; ii < RPL; ++ii) {
                const int i = gl + PG * ii;
                if (i < R) {
                    A(i, kp) = fma(cp, za[ii], -sp * zb[ii]);
                    A(i, kp + 1) = fma(sp, za[ii], cp * zb[ii]);
                }
            }
            kp = kr;
            cp = c;
            sp = s;
            if (++kr < q) {
                z = -s * en;
                ek = c * en;
                x = ekn;
                dk = dk1;
            } else {
                d[q] = dk1;
                e[q - 1] = ekn;
                for (int i = gl; i < R; i += PG) {      // flush the sweep's last rotation
                    const double zk = A(i, kp), zk1 = A(i, kp + 1);
                    A(i, kp) = fma(cp, zk, -sp * zk1);
                    A(i, kp + 1) = fma(sp, zk, cp * zk1);
                }
                sweeping = false;
                __syncwarp(gmask);
            }
        }
        if (failed && gl == 0) atomicOr(&st->flags, FLAG_EIG_NOCONV);
        __syncwarp(gmask);

        // ---- cut, Z scaled by d^-1/4 (columns split over lanes) -------------
        double lmax = 0.0;
        for (int i = gl; i < R; i += PG) lmax = fmax(lmax, d[i]);
        lmax = fmax(lmax, __shfl_xor_sync(gmask, lmax, 4));
        lmax = fmax(lmax, __shfl_xor_sync(gmask, lmax, 2));
        lmax = fmax(lmax, __shfl_xor_sync(gmask, lmax, 1));
        const double cut = rtol2 * lmax;
        for (int i = gl; i < R; i += PG) {
            const double di = d[i];
            const double sf = (lmax > 0.0 && di > cut) ? sqrt(p2_rsqrt(di)) : 0.0;
            for (int r = 0; r < R; ++r) A(r, i) *= sf;
        }
        __syncwarp(gmask);
        // ---- T = Z' (Z'^T H S), one column of T at a time -------------------
        const size_t tb = (size_t)k * R * R;
#pragma unroll 1
        for (int c = 0; c < R; ++c) {
            const double wc = wv[c];
            for (int i = gl; i < R; i += PG) {       // t = Z'^T h_c w_c on my columns
                double s = 0.0;
                for (int r = 0; r < R; ++r) s = fma(A(r, i), __ldg(&H[r * R + c]), s);
                t[i] = s * wc;
            }
            __syncwarp(gmask);
            double tv[RB];
#pragma unroll
            for (int i = 0; i < RB; ++i)
                if (i < R) tv[i] = t[i];
            __syncwarp(gmask);
#pragma unroll 1
            for (int ii = 0; ii < RPL; ++ii) {
                const int r = gl + PG * ii;
                if (r >= R) break;
                double s = 0.0;
#pragma unroll
                for (int i = 0; i < RB; ++i)
                    if (i < R) s = fma(A(r, i), tv[i], s);
                T[tb + r * R + c] = (float)s;
            }
        }
        if (gl == 0) flops = polar_fixed_flops(R) + qr_flops(R, steps, rot);
    }
    add_flops(st, flops);
}

}  // namespace p2
