// Procrustes kernel for larger R: eight or sixteen lanes per subject,
// double-word arithmetic (p2_dw.cuh) or, for the opt-in FP64 arm, FP64
// (p2_num.cuh).  Included by p2_polar_grp.cu; needs the flop
// helpers (p2_polar.cuh), SmallState and FLAG_EIG_NOCONV.
#pragma once

#include <type_traits>

#include "p2_num.cuh"

namespace p2 {

// ---------------------------------------------------------------------------
// Larger R (up to 64): a group of PG = 8 lanes per subject, four subjects per
// warp.  A lane-per-subject kernel would need R^2 double-words of shared
// memory per lane (12.8 KB at R = 40), so only ~17 subjects would fit on an
// SM.  Here the R x R working matrix of a subject lives once in shared memory
// and its eight lanes split the vector work by rows (or columns); the scalar
// parts of the Householder and QR steps run redundantly on the eight lanes of
// a group, so a warp instruction still serves four subjects.  Same
// mathematics, scalings, tolerances and output as the lane-per-subject kernel.
//
// Shared memory: H' (R x R floats) for the block, then per subject A (R x LD,
// LD = R | 1 to spread banks), d, e, t (R each) and w' (R floats in R
// double-word slots).  RB = R rounded up to a multiple of PG (register
// arrays); rows i are owned by lane i % PG.
constexpr int PG_DEFAULT = 8;

inline __host__ __device__ int grp_ld(int R) { return R | 1; }
// double-words per subject
inline __host__ __device__ size_t grp_dws(int R) { return (size_t)R * grp_ld(R) + 4 * (size_t)R; }
// double-words for the block's H'
inline __host__ __device__ size_t grp_hdws(int R) { return ((size_t)R * R + 1) / 2; }

static __device__ __forceinline__ dw shfl_xor_dw(unsigned mask, dw v, int o) {
    return dw{__shfl_xor_sync(mask, v.h, o), __shfl_xor_sync(mask, v.l, o)};
}
static __device__ __forceinline__ f64n shfl_xor_dw(unsigned mask, f64n v, int o) {
    return f64n{__shfl_xor_sync(mask, v.h, o)};
}
// sum over the PG lanes of a group (same result on every lane: the
// butterfly adds the same two operands in the same order on both partners)
template <int PG, class D>
static __device__ __forceinline__ D group_sum(unsigned mask, D v) {
#pragma unroll
    for (int o = PG / 2; o > 0; o >>= 1) v = dw_add(v, shfl_xor_dw(mask, v, o));
    return v;
}
template <int PG>
static __device__ __forceinline__ int group_max(unsigned mask, int v) {
#pragma unroll
    for (int o = PG / 2; o > 0; o >>= 1) v = max(v, __shfl_xor_sync(mask, v, o));
    return v;
}
template <int PG>
static __device__ __forceinline__ float group_maxf(unsigned mask, float v) {
#pragma unroll
    for (int o = PG / 2; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(mask, v, o));
    return v;
}
template <int PG>
static __device__ __forceinline__ unsigned long long group_or(unsigned mask, unsigned long long v) {
#pragma unroll
    for (int o = PG / 2; o > 0; o >>= 1) v |= __shfl_xor_sync(mask, v, o);
    return v;
}

// Scratch of the split Procrustes step: kernel MODE 1 (of k_polar_grp for
// R > 12, of the lane kernel k_polar_reg in p2_polar.cu for R <= 12) reduces
// each subject of a chunk to tridiagonal form and stores Q_h, d, e,
// w' and the output exponent (meta, GRP_ZERO for a zero subject);
// k_qr_record runs the QR iteration on (d, e) alone, one lane per subject,
// and records every Givens rotation (cap per subject; nrec = -1 when they
// do not fit or the iteration failed); MODE 2 applies the recorded rotations
// to Q_h and forms T_k.  kdev (nullable): the number of subjects is *kdev
// (the fused kernel's pass over the subjects the record could not hold).
template <class D> struct RotRec {
    D c, s;
};
constexpr int GRP_ZERO = -1000000;
template <class D> struct GrpSplit {
    D *qh = nullptr;
    D *de = nullptr;
    D *dout = nullptr;
    float *wv = nullptr;
    int *meta = nullptr;
    RotRec<D> *rec = nullptr;
    uint8_t *rkr = nullptr;
    int32_t *nrec = nullptr;
    int64_t cap = 0;                // records per subject slot
    int64_t lim = 0;                // records a subject may use (<= cap)
    // record n of slot i at rec[i * rsub + n * rstep] (rsub = 0: cap, the
    // grouped kernel's layout; the lane kernel interleaves the records of a
    // chunk's slots: rsub = 1, rstep = chunk)
    int64_t rsub = 0, rstep = 1;
    // lane kernel: Q_h entry (r, c) of slot i at qh[(r R + c) chunk + i]
    int64_t chunk = 0;
    const int32_t *kdev = nullptr;
    // nullable: every subject's M' (packed lower, indexed by subject), formed
    // on the tensor cores; the kernels then load it instead of forming it
    const dw *mpre = nullptr;
};
static __device__ __forceinline__ dw shfl_dw(unsigned mask, dw v, int src) {
    return dw{__shfl_sync(mask, v.h, src), __shfl_sync(mask, v.l, src)};
}
static __device__ __forceinline__ f64n shfl_dw(unsigned mask, f64n v, int src) {
    return f64n{__shfl_sync(mask, v.h, src)};
}

template <int RB, int PG, int RT = 0, class D = dw, int MODE = 0>
__global__ void __launch_bounds__(256, 1) k_polar_grp(const dw *__restrict__ G,
                                                      const float *__restrict__ W, SmallState *st,
                                                      float *T, int64_t K, int R_rt, float rtol2,
                                                      int spb, const int32_t *__restrict__ order,
                                                      int32_t *qrcnt, GrpSplit<D> sc) {
    const int R = RT > 0 ? RT : R_rt;   // RT > 0: the rank fixed at compile time
    constexpr int RPL = RB / PG;                     // rows per lane
    extern __shared__ __align__(16) unsigned char smg_raw[];
    D *smg = reinterpret_cast<D *>(smg_raw);
    __shared__ int s_eh;
    const int lane = threadIdx.x & 31;
    const int gl = lane & (PG - 1);
    const unsigned gmask = (unsigned)((1ull << PG) - 1) << (lane & ~(PG - 1));
    const int slot = threadIdx.x / PG;
    const int64_t kslot = (int64_t)blockIdx.x * spb + slot;
    const D one = num_f<D>(1.f), zero = num_f<D>(0.f);
    float *Hs = reinterpret_cast<float *>(smg);
    if (threadIdx.x == 0) s_eh = 0;
    __syncthreads();
    {
        int eh = 0;
        for (int i = threadIdx.x; i < R * R; i += blockDim.x) {
            const float h = (float)st->H64[i];      // exact: H is FP32
            Hs[i] = h;
            eh = max(eh, f_expo(h));
        }
        atomicMax(&s_eh, eh);
    }
    __syncthreads();
    {
        const float hsc = f_pow2(127 - s_eh);        // H' = H 2^sh, max |H'| in [1, 2)
        for (int i = threadIdx.x; i < R * R; i += blockDim.x) Hs[i] = f_mul(Hs[i], hsc);
    }
    __syncthreads();
    unsigned long long flops = 0;
    // the number of subjects may come from the device (the fallback list)
    const int64_t Klim = sc.kdev ? (int64_t)min((int64_t)*sc.kdev, K) : K;
    if (slot < spb && kslot < Klim) {
        const int64_t k = order ? (int64_t)order[kslot] : kslot;
        const int LD = grp_ld(R);
        D *base = smg + grp_hdws(R) + (size_t)slot * grp_dws(R);
        auto A = [base, LD](int i, int j) -> D & { return base[i * LD + j]; };
        D *d = base + (size_t)R * LD;
        D *e = d + R;
        D *t = e + R;
        float *wv = reinterpret_cast<float *>(t + R);
        const dw *Gk = G + (size_t)k * (R * (R + 1) / 2);
        const size_t tb = (size_t)k * R * R;

        int so = 0;
        bool live = true;                               // a subject with a Q-step to finish
        if constexpr (MODE != 2) {
            // ---- scalings: S' = S 2^sw, G' = G 2^sg ------------------------------
            int ew = 0, eg = 0;
            for (int i = gl; i < R; i += PG) {
                const float w = W[(size_t)k * R + i];
                wv[i] = w;
                ew = max(ew, f_expo(w));
                eg = max(eg, f_expo(Gk[i * (i + 1) / 2 + i].h));
            }
            ew = group_max<PG>(gmask, ew);
            eg = group_max<PG>(gmask, eg);
            const int sg = 127 - eg;
            const float gsc = f_pow2(sg);
            {
                const float wsc = f_pow2(127 - ew);
                for (int i = gl; i < R; i += PG) wv[i] = f_mul(wv[i], wsc);
            }
            __syncwarp(gmask);

            int em = 0;
            if (std::is_same<D, dw>::value && sc.mpre) {
                // M' formed on the tensor cores (same scalings, double-word accuracy)
                const dw *Mk = sc.mpre + (size_t)k * (R * (R + 1) / 2);
                for (int i = gl; i < R; i += PG) {
                    for (int j = 0; j <= i; ++j) A(i, j) = from_dw<D>(Mk[i * (i + 1) / 2 + j]);
                    em = max(em, f_expo(A(i, i).h));
                }
                __syncwarp(gmask);
            } else {
                // ---- M' = H' B H'^T with B = S' G' S' -------------------------------
                // U = B H'^T, row by row in place (row i of B is held in registers).
                #pragma unroll 1
                for (int ii = 0; ii < RPL; ++ii) {
                    const int i = gl + PG * ii;
                    if (i >= R) break;
                    D b[RB];
                    const float wi = wv[i];
                #pragma unroll
                    for (int j = 0; j < RB; ++j) {
                        if (j < R) {
                            const int p = (j <= i) ? (i * (i + 1) / 2 + j) : (j * (j + 1) / 2 + i);
                            b[j] = dw_mul(dw_scale(from_dw<D>(Gk[p]), gsc), num_prod<D>(wi, wv[j]));
                        }
                    }
                    int c = 0;
                #pragma unroll 1
                    for (; c + 1 < R; c += 2) {             // columns in pairs
                        acc_t<D> s0 = acc0<D>(), s1 = acc0<D>();
                #pragma unroll
                        for (int j = 0; j < RB; ++j)
                            if (j < R) {
                                acc_fmaf(s0, b[j], Hs[c * R + j]);
                                acc_fmaf(s1, b[j], Hs[(c + 1) * R + j]);
                            }
                        A(i, c) = acc_val(s0);
                        A(i, c + 1) = acc_val(s1);
                    }
                    if (c < R) {
                        acc_t<D> s = acc0<D>();
                #pragma unroll
                        for (int j = 0; j < RB; ++j)
                            if (j < R) acc_fmaf(s, b[j], Hs[c * R + j]);
                        A(i, c) = acc_val(s);
                    }
                }
                __syncwarp(gmask);
                // M' = H' U, column by column in place (lower triangle).
                #pragma unroll 1
                for (int c = 0; c < R; ++c) {
                    D u[RB];
                #pragma unroll
                    for (int i = 0; i < RB; ++i)
                        if (i < R) u[i] = A(i, c);
                    __syncwarp(gmask);
                    int r2 = gl;                            // the lane's rows in pairs
                    while (r2 < c) r2 += PG;
                    for (; r2 + PG < R; r2 += 2 * PG) {
                        const int r = r2, r1 = r2 + PG;
                        acc_t<D> s0 = acc0<D>(), s1 = acc0<D>();
                #pragma unroll
                        for (int i = 0; i < RB; ++i)
                            if (i < R) {
                                acc_fmaf(s0, u[i], Hs[r * R + i]);
                                acc_fmaf(s1, u[i], Hs[r1 * R + i]);
                            }
                        const D m0 = acc_val(s0), m1 = acc_val(s1);
                        A(r, c) = m0;
                        A(r1, c) = m1;
                        if (r == c) em = max(em, f_expo(m0.h));
                    }
                    if (r2 < R) {
                        const int r = r2;
                        acc_t<D> s = acc0<D>();
                #pragma unroll
                        for (int i = 0; i < RB; ++i)
                            if (i < R) acc_fmaf(s, u[i], Hs[r * R + i]);
                        const D m = acc_val(s);
                        A(r, c) = m;
                        if (r == c) em = max(em, f_expo(m.h));
                    }
                    __syncwarp(gmask);
                }
            }
            em = group_max<PG>(gmask, em);
            if (eg == 0 || ew == 0 || em == 0) {
                // G, W or M is zero (or below the normal range): A_k = 0, Q_k = 0
                for (int i = gl; i < R * R; i += PG) T[tb + i] = 0.f;
                if (qrcnt && gl == 0) qrcnt[k] = 0;
                if constexpr (MODE == 1) {
                    if (gl == 0) sc.meta[kslot] = GRP_ZERO;
                }
                live = false;
            } else {
                // M'' = M' 2^sm, max diag in [0.5, 2), sm + sg even
                int sm = 127 - em;
                if ((sm + sg) & 1) --sm;
                {
                    const float msc = f_pow2(sm);
                    for (int i = gl; i < R; i += PG)
                        for (int j = 0; j <= i; ++j) A(i, j) = dw_scale(A(i, j), msc);
                }
                __syncwarp(gmask);

                // ---- Householder tridiagonalisation (lower triangle) ----------
    #pragma unroll 1
                for (int kk = 0; kk + 2 < R; ++kk) {
                    acc_t<D> sa = acc0<D>();
                    for (int i = gl; i < R; i += PG)
                        if (i >= kk + 2) acc_sqr(sa, A(i, kk));
                    const D sig = group_sum<PG>(gmask, acc_val(sa));
                    const D x0 = A(kk + 1, kk);
                    if (!(sig.h >= NumT<D>::tiny2())) {          // reflector as in p2_eig_dw.cuh
                        __syncwarp(gmask);
                        if (gl == 0) {
                            A(kk, kk + 1) = zero;
                            e[kk] = x0;
                        }
                        __syncwarp(gmask);
                        continue;
                    }
                    acc_t<D> m2 = acc_from(sig);
                    acc_sqr(m2, x0);
                    const D mu = dw_sqrt(acc_val(m2));
                    const D beta = (x0.h >= 0.f) ? dw_neg(mu) : mu;
                    const D bh = dw_div(dw_sub(beta, x0), beta);
                    const D inv_v0 = dw_recip(dw_sub(x0, beta));
                    __syncwarp(gmask);
                    for (int i = gl; i < R; i += PG)
                        if (i >= kk + 2) A(i, kk) = dw_mul(A(i, kk), inv_v0);
                    if (gl == 0) {
                        A(kk, kk + 1) = bh;
                        e[kk] = beta;
                    }
                    __syncwarp(gmask);
                    // p = bh A22 v on my rows, pv = p . v
                    // (the lane's rows in pairs, two independent sums
                    // interleaved; pa in row order)
                    acc_t<D> pa = acc0<D>();
                    int i2 = gl;
                    while (i2 < kk + 1) i2 += PG;
                    for (; i2 + PG < R; i2 += 2 * PG) {
                        const int i = i2, i1 = i2 + PG;
                        acc_t<D> s0 = acc_from(A(i, kk + 1));
                        acc_t<D> s1 = acc_from(A(i1, kk + 1));
                        for (int j = kk + 2; j < R; ++j) {
                            const D vj = A(j, kk);
                            acc_fma(s0, (j <= i) ? A(i, j) : A(j, i), vj);
                            acc_fma(s1, (j <= i1) ? A(i1, j) : A(j, i1), vj);
                        }
                        const D si0 = dw_mul(acc_val(s0), bh);
                        const D si1 = dw_mul(acc_val(s1), bh);
                        t[i] = si0;
                        t[i1] = si1;
                        if (i == kk + 1)
                            acc_add(pa, si0);
                        else
                            acc_fma(pa, si0, A(i, kk));
                        acc_fma(pa, si1, A(i1, kk));
                    }
                    if (i2 < R) {
                        const int i = i2;
                        acc_t<D> s = acc_from(A(i, kk + 1));
                        for (int j = kk + 2; j < R; ++j)
                            acc_fma(s, (j <= i) ? A(i, j) : A(j, i), A(j, kk));
                        const D si = dw_mul(acc_val(s), bh);
                        t[i] = si;
                        if (i == kk + 1)
                            acc_add(pa, si);
                        else
                            acc_fma(pa, si, A(i, kk));
                    }
                    const D pv = group_sum<PG>(gmask, acc_val(pa));
                    const D nK = dw_neg(dw_mul(dw_scale(bh, 0.5f), pv));
                    for (int i = gl; i < R; i += PG) {
                        if (i == kk + 1)
                            t[i] = dw_add(t[i], nK);
                        else if (i > kk + 1)
                            t[i] = dw_fma(nK, A(i, kk), t[i]);
                    }
                    __syncwarp(gmask);
                    for (int i = gl; i < R; i += PG) {
                        if (i < kk + 1) continue;
                        const D nvi = dw_neg((i == kk + 1) ? one : A(i, kk));
                        const D nwi = dw_neg(t[i]);
                        {                                    // j = kk + 1: v_{kk+1} = 1
                            acc_t<D> a = acc_from(A(i, kk + 1));
                            acc_fma(a, nvi, t[kk + 1]);
                            acc_add(a, nwi);
                            A(i, kk + 1) = acc_val(a);
                        }
                        int j = kk + 2;
                        for (; j + 1 <= i; j += 2) {         // entries in pairs
                            acc_t<D> a0 = acc_from(A(i, j));
                            acc_t<D> a1 = acc_from(A(i, j + 1));
                            acc_fma(a0, nvi, t[j]);
                            acc_fma(a1, nvi, t[j + 1]);
                            acc_fma(a0, nwi, A(j, kk));
                            acc_fma(a1, nwi, A(j + 1, kk));
                            A(i, j) = acc_val(a0);
                            A(i, j + 1) = acc_val(a1);
                        }
                        if (j <= i) {
                            acc_t<D> a = acc_from(A(i, j));
                            acc_fma(a, nvi, t[j]);
                            acc_fma(a, nwi, A(j, kk));
                            A(i, j) = acc_val(a);
                        }
                    }
                    __syncwarp(gmask);
                }
                if (gl == 0 && R >= 2) e[R - 2] = A(R - 1, R - 2);
                for (int i = gl; i < R; i += PG) d[i] = A(i, i);
                __syncwarp(gmask);
                // backward accumulation of Q = P_0 ... P_{R-3}, columns split over lanes
                if (R == 1) {
                    if (gl == 0) A(0, 0) = one;
                } else {
                    if (gl == 0) {
                        A(R - 1, R - 1) = one;
                        A(R - 2, R - 2) = one;
                        A(R - 1, R - 2) = zero;
                        A(R - 2, R - 1) = zero;
                    }
                    __syncwarp(gmask);
    #pragma unroll 1
                    for (int kk = R - 3; kk >= 0; --kk) {
                        const D bh = A(kk, kk + 1);
                        __syncwarp(gmask);
                        const D nb = dw_neg(bh);
                        const bool act = bh.h != 0.f;
                        for (int j = gl; j < R; j += PG) {
                            if (j == kk + 1) {                    // column e_{k+1} -> (1 - b, -b v)
                                A(kk + 1, kk + 1) = act ? dw_add(one, nb) : one;
                                for (int i = kk + 2; i < R; ++i) A(i, kk + 1) = act ? dw_mul(nb, A(i, kk)) : zero;
                            } else if (j > kk + 1) {
                                A(kk + 1, j) = zero;
                            }
                        }
                        __syncwarp(gmask);
                        if (act) {
                            int c2 = gl;                        // the lane's columns in pairs
                            while (c2 < kk + 2) c2 += PG;
                            for (; c2 + PG < R; c2 += 2 * PG) {
                                const int c = c2, c1 = c2 + PG;
                                acc_t<D> s0 = acc0<D>(), s1 = acc0<D>();   // A(kk+1, c) = 0 here
                                for (int i = kk + 2; i < R; ++i) {
                                    const D vi = A(i, kk);
                                    acc_fma(s0, vi, A(i, c));
                                    acc_fma(s1, vi, A(i, c1));
                                }
                                const D ns0 = dw_mul(acc_val(s0), nb);
                                const D ns1 = dw_mul(acc_val(s1), nb);
                                A(kk + 1, c) = ns0;
                                A(kk + 1, c1) = ns1;
                                for (int i = kk + 2; i < R; ++i) {
                                    const D vi = A(i, kk);
                                    A(i, c) = dw_fma(ns0, vi, A(i, c));
                                    A(i, c1) = dw_fma(ns1, vi, A(i, c1));
                                }
                            }
                            if (c2 < R) {
                                const int c = c2;
                                acc_t<D> s = acc0<D>();
                                for (int i = kk + 2; i < R; ++i) acc_fma(s, A(i, kk), A(i, c));
                                const D ns = dw_mul(acc_val(s), nb);
                                A(kk + 1, c) = ns;
                                for (int i = kk + 2; i < R; ++i) A(i, c) = dw_fma(ns, A(i, kk), A(i, c));
                            }
                        }
                        __syncwarp(gmask);
                    }
                    for (int j = gl; j < R; j += PG) {
                        if (j == 0) {
                            A(0, 0) = one;
                        } else {
                            A(0, j) = zero;
                            A(j, 0) = zero;
                        }
                    }
                }
                __syncwarp(gmask);

                so = (sm + sg) / 2;
                if constexpr (MODE == 1) {
                    // hand Q_h, the tridiagonal and w' to the QR and finishing
                    // kernels (row-major Q_h; d, e; w' as floats)
                    D *qh = sc.qh + (size_t)kslot * R * R;
                    for (int i = gl; i < R; i += PG)
                        for (int j = 0; j < R; ++j) qh[(size_t)i * R + j] = A(i, j);
                    D *de = sc.de + (size_t)kslot * 2 * R;
                    for (int i = gl; i < R; i += PG) {
                        de[i] = d[i];
                        de[R + i] = (i + 1 < R) ? e[i] : zero;
                        sc.wv[(size_t)kslot * R + i] = wv[i];
                    }
                    if (gl == 0) sc.meta[kslot] = so;
                    live = false;
                }
            }
        } else {
            // the subject's Q_h, w' and eigenvalues from the other kernels;
            // subjects that were zero or whose rotations did not fit the record
            // (finished by the fused kernel instead) are skipped
            const int meta = sc.meta[kslot];
            const int32_t nrec = sc.nrec[kslot];
            live = meta != GRP_ZERO && nrec >= 0;
            if (live) {
                so = meta;
                const D *qh = sc.qh + (size_t)kslot * R * R;
                for (int i = gl; i < R; i += PG)
                    for (int j = 0; j < R; ++j) A(i, j) = qh[(size_t)i * R + j];
                for (int i = gl; i < R; i += PG) {
                    d[i] = sc.dout[(size_t)kslot * R + i];
                    wv[i] = sc.wv[(size_t)kslot * R + i];
                }
                __syncwarp(gmask);
                // the rotations in the order the QR formed them, each on the
                // lanes' rows of columns (kr, kr + 1), with the arithmetic of the
                // fused kernel (which first applies an identity rotation to
                // columns 0 and 1: so does this one, for bitwise equal results)
                const RotRec<D> *rec = sc.rec + (size_t)kslot * sc.cap;
                const uint8_t *rkr = sc.rkr + (size_t)kslot * sc.cap;
                D cp = one, sp = zero;
                int kp = 0;
                if (R > 1) {
                    const D nsp = dw_neg(sp);
#pragma unroll
                    for (int ii = 0; ii < RPL; ++ii) {
                        const int i = gl + PG * ii;
                        if (i < R) {
                            const D za = A(i, kp), zb = A(i, kp + 1);
                            A(i, kp) = dw_dot2(cp, za, nsp, zb);
                            A(i, kp + 1) = dw_dot2(sp, za, cp, zb);
                        }
                    }
                }
#pragma unroll 1
                for (int32_t n0 = 0; n0 < nrec; n0 += PG) {
                    // PG records loaded by the group's lanes, then broadcast
                    RotRec<D> mine{zero, zero};
                    int mkr = 0;
                    if (n0 + gl < nrec) {
                        mine = rec[n0 + gl];
                        mkr = rkr[n0 + gl];
                    }
                    const int nb = (nrec - n0) < PG ? (nrec - n0) : PG;
                    for (int j = 0; j < nb; ++j) {
                        const int src = (lane & ~(PG - 1)) + j;
                        const D c = shfl_dw(gmask, mine.c, src);
                        const D s = shfl_dw(gmask, mine.s, src);
                        kp = __shfl_sync(gmask, mkr, src);
                        const D ns = dw_neg(s);
#pragma unroll
                        for (int ii = 0; ii < RPL; ++ii) {
                            const int i = gl + PG * ii;
                            if (i < R) {
                                const D za = A(i, kp), zb = A(i, kp + 1);
                                A(i, kp) = dw_dot2(c, za, ns, zb);
                                A(i, kp + 1) = dw_dot2(s, za, c, zb);
                            }
                        }
                    }
                }
                __syncwarp(gmask);
            }
        }
        if constexpr (MODE == 0) {
            if (live) {
                // ---- implicit QR with Wilkinson shift; rotations on my rows of Z --
                // One flat loop, one Givens rotation per trip, so that the four
                // groups of a warp execute the rotation body together whatever
                // their sweep boundaries.  The scalar recurrence runs on all eight
                // lanes (identical values); d[k+1] and e[k+1] of a sweep are read
                // before anything writes them and d[k], e[k] are carried in
                // registers.  A trip forms rotation kr and applies rotation kr - 1
                // (kp, cp, sp) to the lanes' rows of Z; the pending rotation
                // carries over sweep boundaries and is flushed at the end.
                float an = 0.f;
                for (int i = gl; i < R; i += PG) {
                    float r = fabsf(d[i].h);
                    if (i + 1 < R) r += fabsf(e[i].h);
                    if (i > 0) r += fabsf(e[i - 1].h);
                    an = fmaxf(an, r);
                }
                an = group_maxf<PG>(gmask, an);
                const int tiny_ex = f_expo(an) - NumT<D>::deflate_bits;
                int steps = 0, rot = 0;
                const int max_steps = 30 * R;
                int q = R - 1, p = 0, kr = 0;
                bool sweeping = false, failed = false;
                D x = zero, z = zero, dk = zero, ek = zero;
                int kp = 0;
                D cp = one, sp = zero;
    #pragma unroll 1
                while (true) {
                    if (!sweeping) {
                        // deflation tests of all positions at once, split over
                        // the eight lanes and OR-ed together; the active block
                        // follows from leading-zero counts
                        unsigned long long nm = 0;
                        for (int i = gl; i + 1 < R; i += PG)
                            if (dw_negligible(e[i], d[i], d[i + 1], tiny_ex)) nm |= 1ull << i;
                        nm = group_or<PG>(gmask, nm);
                        const unsigned long long nn = ~nm & ((1ull << q) - 1);
                        q = nn ? 64 - p2_clz64(nn) : 0;
                        if (q == 0) break;
                        const unsigned long long nb = q > 1 ? nm & ((1ull << (q - 1)) - 1) : 0ull;
                        p = nb ? 64 - p2_clz64(nb) : 0;
                        if (++steps > max_steps) {
                            failed = true;
                            break;
                        }
                        rot += q - p;
                        const D eq = e[q - 1];
                        const D dd = dw_scale(dw_sub(d[q - 1], d[q]), 0.5f);
                        acc_t<D> hh = acc0<D>();
                        acc_sqr(hh, dd);
                        acc_sqr(hh, eq);
                        const D h = dw_sqrt(acc_val(hh));
                        const D den = (dd.h >= 0.f) ? dw_add(dd, h) : dw_sub(dd, h);
                        const D mu = dw_sub(d[q], dw_div(dw_sqr(eq), den));
                        dk = d[p];
                        ek = e[p];
                        x = dw_sub(dk, mu);
                        z = ek;
                        kr = p;
                        sweeping = true;
                        __syncwarp(gmask);
                        if (gl == 0 && p > 0) e[p - 1] = zero;
                    }
                    const D bb = d[kr + 1];
                    const D en = (kr + 1 < q) ? e[kr + 1] : zero;
                    __syncwarp(gmask);
                    D za[RPL], zb[RPL];
    #pragma unroll
                    for (int ii = 0; ii < RPL; ++ii) {
                        const int i = gl + PG * ii;
                        if (i < R) {
                            za[ii] = A(i, kp);
                            zb[ii] = A(i, kp + 1);
                        }
                    }
                    const int ex = max(f_expo(x.h), f_expo(z.h));   // scaled as in p2_eig_dw.cuh
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
                    const D rr = nz ? dw_scale(dw_mul(tt, ir), f_pow2(ex - 127)) : zero;
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
                    {
                        const D nsp = dw_neg(sp);
    #pragma unroll
                        for (int ii = 0; ii < RPL; ++ii) {
                            const int i = gl + PG * ii;
                            if (i < R) {
                                A(i, kp) = dw_dot2(cp, za[ii], nsp, zb[ii]);
                                A(i, kp + 1) = dw_dot2(sp, za[ii], cp, zb[ii]);
                            }
                        }
                    }
                    if (gl == 0) {
                        if (kr > p) e[kr - 1] = rr;
                        d[kr] = dkn;
                    }
                    kp = kr;
                    cp = c;
                    sp = s;
                    if (++kr < q) {
                        z = dw_neg(dw_mul(s, en));
                        ek = dw_mul(c, en);
                        x = ekn;
                        dk = dk1;
                    } else {
                        if (gl == 0) {
                            d[q] = dk1;
                            e[q - 1] = ekn;
                        }
                        sweeping = false;
                        __syncwarp(gmask);
                    }
                }
                __syncwarp(gmask);
                if (R > 1) {                                 // flush the last rotation
                    const D nsp = dw_neg(sp);
                    for (int i = gl; i < R; i += PG) {
                        const D zk = A(i, kp), zk1 = A(i, kp + 1);
                        A(i, kp) = dw_dot2(cp, zk, nsp, zk1);
                        A(i, kp + 1) = dw_dot2(sp, zk, cp, zk1);
                    }
                }
                if (failed && gl == 0) atomicOr(&st->flags, FLAG_EIG_NOCONV);
                __syncwarp(gmask);

                if (gl == 0) {
                    flops = qr_flops(R, steps, rot);
                    if (qrcnt) qrcnt[k] = rot;
                }
            }
        }
        if constexpr (MODE != 1) {
            if (live) {
                // ---- cut, Z scaled by d^-1/4 (columns split over lanes) ---------
                float lmax = 0.f;
                for (int i = gl; i < R; i += PG) lmax = fmaxf(lmax, d[i].h);
                lmax = group_maxf<PG>(gmask, lmax);
                const float cut = rtol2 * lmax;
                for (int i = gl; i < R; i += PG) {
                    const D di = d[i];
                    const D sf = (lmax > 0.f && di.h > cut) ? dw_sqrt(dw_rsqrt(di)) : zero;
                    for (int r = 0; r < R; ++r) A(r, i) = dw_mul(A(r, i), sf);
                }
                __syncwarp(gmask);
                // ---- T = 2^so Z' (Z'^T H' S'), one column of T at a time ----------
                const float o1 = f_pow2(so / 2), o2 = f_pow2(so - so / 2);
    #pragma unroll 1
                for (int c = 0; c < R; ++c) {
                    for (int i = gl; i < R; i += PG) {       // t = Z'^T h'_c on my columns
                        acc_t<D> s = acc0<D>();
                        for (int r = 0; r < R; ++r) acc_fmaf(s, A(r, i), Hs[r * R + c]);
                        t[i] = acc_val(s);
                    }
                    __syncwarp(gmask);
                    D tv[RB];
    #pragma unroll
                    for (int i = 0; i < RB; ++i)
                        if (i < R) tv[i] = t[i];
                    __syncwarp(gmask);
                    const float wc = wv[c];
    #pragma unroll 1
                    for (int ii = 0; ii < RPL; ++ii) {
                        const int r = gl + PG * ii;
                        if (r >= R) break;
                        acc_t<D> s = acc0<D>();
    #pragma unroll
                        for (int i = 0; i < RB; ++i)
                            if (i < R) acc_fma(s, A(r, i), tv[i]);
                        const D v = dw_mulf(acc_val(s), wc);
                        T[tb + r * R + c] = store_f(v, o1, o2);
                    }
                }
                if (gl == 0) flops += polar_fixed_flops(R);
            }
        }
    }
    add_flops(st, flops);
}

// ---------------------------------------------------------------------------
// QR iteration of the split Procrustes step: one lane per subject on the
// tridiagonal (d, e) that MODE 1 stored, with the grouped kernel's scalar
// recurrence (deflation, Wilkinson shift, Givens rotations formed from one
// reciprocal square root after power-of-two scaling) but without the
// eigenvector matrix: every rotation is recorded (c, s, and its column kr)
// for MODE 2 to apply.  In the fused kernel each lane of a group runs this
// recurrence redundantly; here one lane serves a subject, so the recurrence
// costs 1/16 of the warp instructions it did there.
// ---------------------------------------------------------------------------
constexpr int QR_THREADS = 128;       // threads per block of k_qr_record (a constant
                                      // stride: the lanes' d, e provably distinct)
template <int RT, class D>
__global__ void __launch_bounds__(QR_THREADS) k_qr_record(GrpSplit<D> sc, int64_t K, int R_rt,
                                                   const int32_t *__restrict__ order,
                                                   int32_t *qrcnt, SmallState *st) {
    const int R = RT > 0 ? RT : R_rt;
    extern __shared__ __align__(16) unsigned char sqr_raw[];
    D *smq = reinterpret_cast<D *>(sqr_raw);
    const int t = threadIdx.x;
    constexpr int NT = QR_THREADS;
    const int64_t slot = (int64_t)blockIdx.x * NT + t;
    D *dv = smq + t;
    D *ev = smq + (size_t)R * NT + t;
    auto d = [dv](int i) -> D & { return dv[(size_t)i * NT]; };
    auto e = [ev](int i) -> D & { return ev[(size_t)i * NT]; };
    const D one = num_f<D>(1.f), zero = num_f<D>(0.f);
    unsigned long long flops = 0;
    if (slot < K && sc.meta[slot] != GRP_ZERO) {
        const int64_t k = order ? (int64_t)order[slot] : slot;
        const D *de = sc.de + (size_t)slot * 2 * R;
        for (int i = 0; i < R; ++i) {
            d(i) = de[i];
            e(i) = de[R + i];
        }
        const int64_t rs = sc.rsub ? sc.rsub : sc.cap;
        RotRec<D> *rec = sc.rec + (size_t)slot * rs;
        uint8_t *rkr = sc.rkr + (size_t)slot * rs;
        int64_t n = 0;
        bool full = false;
        float an = 0.f;
        for (int i = 0; i < R; ++i) {
            float r = fabsf(d(i).h);
            if (i + 1 < R) r += fabsf(e(i).h);
            if (i > 0) r += fabsf(e(i - 1).h);
            an = fmaxf(an, r);
        }
        const int tiny_ex = f_expo(an) - NumT<D>::deflate_bits;
        int steps = 0, rot = 0;
        const int max_steps = 30 * R;
        int q = R - 1, p = 0, kr = 0;
        bool sweeping = false, failed = false;
        D x = zero, z = zero, dk = zero, ek = zero;
#pragma unroll 1
        while (true) {
            if (!sweeping) {
                unsigned long long nm = 0;
                for (int i = 0; i + 1 < R; ++i)
                    if (dw_negligible(e(i), d(i), d(i + 1), tiny_ex)) nm |= 1ull << i;
                const unsigned long long nn = ~nm & ((1ull << q) - 1);
                q = nn ? 64 - p2_clz64(nn) : 0;
                if (q == 0) break;
                const unsigned long long nb = q > 1 ? nm & ((1ull << (q - 1)) - 1) : 0ull;
                p = nb ? 64 - p2_clz64(nb) : 0;
                if (++steps > max_steps) {
                    failed = true;
                    break;
                }
                rot += q - p;
                const D eq = e(q - 1);
                const D dd = dw_scale(dw_sub(d(q - 1), d(q)), 0.5f);
                acc_t<D> hh = acc0<D>();
                acc_sqr(hh, dd);
                acc_sqr(hh, eq);
                const D h = dw_sqrt(acc_val(hh));
                const D den = (dd.h >= 0.f) ? dw_add(dd, h) : dw_sub(dd, h);
                const D mu = dw_sub(d(q), dw_div(dw_sqr(eq), den));
                dk = d(p);
                ek = e(p);
                x = dw_sub(dk, mu);
                z = ek;
                kr = p;
                sweeping = true;
                if (p > 0) e(p - 1) = zero;
            }
            const D bb = d(kr + 1);
            const D en = (kr + 1 < q) ? e(kr + 1) : zero;
            const int ex = max(f_expo(x.h), f_expo(z.h));
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
            const D rr = nz ? dw_scale(dw_mul(tt, ir), f_pow2(ex - 127)) : zero;
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
            if (n >= sc.lim) {                          // the record is full
                full = true;
                break;
            }
            rec[n * sc.rstep] = RotRec<D>{c, s};
            rkr[n * sc.rstep] = (uint8_t)kr;
            ++n;
            if (kr > p) e(kr - 1) = rr;
            d(kr) = dkn;
            if (++kr < q) {
                z = dw_neg(dw_mul(s, en));
                ek = dw_mul(c, en);
                x = ekn;
                dk = dk1;
            } else {
                d(q) = dk1;
                e(q - 1) = ekn;
                sweeping = false;
            }
        }
        if (failed || full) {
            sc.nrec[slot] = -1;                         // the fused kernel redoes this subject
        } else {
            for (int i = 0; i < R; ++i) sc.dout[(size_t)slot * R + i] = d(i);
            sc.nrec[slot] = (int32_t)n;
            flops = qr_flops(R, steps, rot);
            if (qrcnt) qrcnt[k] = rot;
        }
    } else if (slot < K) {
        sc.nrec[slot] = 0;
    }
    add_flops(st, flops);
}

// Subjects of a chunk whose rotations did not fit their record (or whose QR
// iteration failed): appended to list (count: *cnt) for the fused kernel.
static __global__ void k_split_collect(const int32_t *__restrict__ nrec, int64_t K,
                                const int32_t *__restrict__ order, int32_t *list, int32_t *cnt) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < K;
         i += (int64_t)gridDim.x * blockDim.x)
        if (nrec[i] < 0) list[atomicAdd(cnt, 1)] = order ? order[i] : (int32_t)i;
}

}  // namespace p2
