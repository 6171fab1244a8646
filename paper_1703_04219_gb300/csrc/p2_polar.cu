// Procrustes step of the Q-step (Section 3.2, Algorithm 2's SVD loop), one
// GPU lane per subject, in double-word arithmetic (p2_dw.cuh).
//
// For subject k with Gram G_k = Z_k^T Z_k (Z_k = X_k V) and S_k = diag(W(k,:)):
//   M   = H S G S H^T                  (= A_k^T A_k, A_k = X_k V S_k H^T)
//   M   = Z diag(d) Z^T                (Householder tridiagonalisation + implicit QR)
//   f_i = d_i^{-1/2} if d_i > rtol^2 max(d) else 0    (rank cut of the SVD)
//   C   = Z diag(f) Z^T                (pseudo-inverse square root of M)
//   T_k = C H S = Z' (Z'^T H S), Z' = Z diag(f)^{1/2}   (stored FP32; Q_k = X_k V T_k^T)
// Precision: T_k is stored in FP32, whose rounding already perturbs Q_k by
// ~2^-24 cond(A_k); the eigen-decomposition of M = A_k^T A_k in double-word
// arithmetic (~2^-46 normwise) perturbs it by ~2^-46 cond(A_k)^2, below the
// storage error for every cond(A_k) <= 1 / rank_rtol the rank cut admits.
// Range: G, W and H are scaled by powers of two (exactly) so that every
// intermediate stays inside the FP32 exponent range, and the exponents are
// folded back into T_k at the end.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <algorithm>
#include <type_traits>

#include "p2_internal.cuh"
#include "p2_eig_dw.cuh"
#include "p2_polar.cuh"
#include "p2_polar_grp.cuh"

namespace p2 {

template <int R>
static __device__ __forceinline__ int pk(int i, int j) {   // packed lower index
    return (j <= i) ? (i * (i + 1) / 2 + j) : (j * (j + 1) / 2 + i);
}

// Shared memory: H (scaled, FP32) for the block, then per lane the working
// matrix (R x R) and the tridiagonal (d, e), interleaved across the lanes:
// R^2 + 2R double-words per lane (MODE 2 below: R^2, plus w' for R > 10; its
// d in registers: 256 lanes at R = 10 instead of 224).  The block has as
// many lanes as a block's opt-in shared memory (227 KB) holds, at most 256,
// a multiple of 32: a compile-time constant, so that the interleaved
// addresses of different entries are provably distinct and the compiler may
// reorder their loads and stores.
constexpr int REG_SMEM_OPTIN = 232448;
template <int R>
__host__ __device__ constexpr size_t reg_hbytes() { return (size_t)((R * R + 1) / 2) * sizeof(dw); }
template <int R, int MODE>
__host__ __device__ constexpr size_t reg_lane_bytes() {
    return (size_t)(MODE == 2 ? R * R + (R > 10 ? R : 0) : R * R + 2 * R) * sizeof(dw);
}
template <int R, int MODE>
__host__ __device__ constexpr int reg_threads() {
    return (int)(((REG_SMEM_OPTIN - reg_hbytes<R>()) / reg_lane_bytes<R, MODE>() < 256
                      ? (REG_SMEM_OPTIN - reg_hbytes<R>()) / reg_lane_bytes<R, MODE>()
                      : 256) /
                 32 * 32);
}
//
// MODE 0 runs the whole step.  The split step runs it in three kernels over
// a chunk of subjects: MODE 1 forms M, reduces it to tridiagonal form and
// stores Q_h, d, e, w' and the output exponent; k_qr_record
// (p2_polar_grp.cuh) runs the QR iteration on (d, e) alone, one lane per
// subject at full occupancy, recording every rotation; MODE 2 applies the
// records to Q_h, then the cut and T_k.  Same arithmetic in the same order as
// MODE 0, hence the same results bit for bit.  Q_h and the records are
// interleaved over the chunk's slots (coalesced).  sc.kdev (nullable): the
// number of subjects is *sc.kdev (MODE 0 over the subjects whose rotations
// did not fit the record).
template <int R, class D, int MODE = 0>
__global__ void __launch_bounds__(reg_threads<R, MODE>(), 1) k_polar_reg(const dw *__restrict__ G,
                                                   const float *__restrict__ W, SmallState *st,
                                                   float *T, int64_t K, float rtol2,
                                                   const int32_t *__restrict__ order,
                                                   int32_t *qrcnt, GrpSplit<D> sc) {
    constexpr int P = R * (R + 1) / 2;
    constexpr int HW = (R * R + 1) / 2;                  // double-word slots holding H
    extern __shared__ __align__(16) unsigned char smr_raw[];
    D *smd = reinterpret_cast<D *>(smr_raw);
    constexpr int NT = reg_threads<R, MODE>();           // = blockDim.x
    static_assert(sizeof(D) == sizeof(dw), "one double-word slot per element");
    const int t = threadIdx.x;
    float *Hs = reinterpret_cast<float *>(smd);
    D *th = smd + HW;
    for (int i = t; i < R * R; i += NT) Hs[i] = (float)st->H64[i];   // exact: H is FP32
    __syncthreads();
    int eh = 0;
    for (int i = 0; i < R * R; ++i) eh = max(eh, f_expo(Hs[i]));
    const float hsc = f_pow2(127 - eh);                  // H' = H 2^sh, max |H'| in [1, 2)
    __syncthreads();
    for (int i = t; i < R * R; i += NT) Hs[i] = f_mul(Hs[i], hsc);
    __syncthreads();
    const int64_t slot = (int64_t)blockIdx.x * NT + t;
    const int64_t Klim = sc.kdev ? min((int64_t)*sc.kdev, K) : K;
    unsigned long long flops = 0;
    if (slot < Klim) {
        const int64_t k = order ? (int64_t)order[slot] : slot;
        const D zero = num_f<D>(0.f), one = num_f<D>(1.f);
        DwMat<D> A{th + t, NT, R};
        DwVec<D> d{th + (size_t)R * R * NT + t, NT};     // (not MODE 2)
        DwVec<D> e{th + (size_t)(MODE == 2 ? R * R : R * R + R) * NT + t, NT};
        D dr[MODE == 2 ? R : 1];                         // MODE 2: the eigenvalues
        const size_t tb = (size_t)k * R * R;
        int so = 0;
        bool live = true;                                // a subject with T_k to form
        float w[R];
        if constexpr (MODE != 2) {
            const dw *Gk = G + (size_t)k * P;
            int ew = 0, eg = 0;
#pragma unroll
            for (int i = 0; i < R; ++i) {
                w[i] = W[(size_t)k * R + i];
                ew = max(ew, f_expo(w[i]));
                eg = max(eg, f_expo(Gk[i * (i + 1) / 2 + i].h));   // |G_ij| <= max_i G_ii
            }
            // M' = H' S' G' S' H'^T with S' = S 2^sw, G' = G 2^sg (exact scalings)
            const int sg = 127 - eg;
            const float wsc = f_pow2(127 - ew), gsc = f_pow2(sg);
#pragma unroll
            for (int i = 0; i < R; ++i) w[i] = f_mul(w[i], wsc);
            // g = S' G' S' held in registers (packed lower); M' column by column
            // into the lower triangle of A
            int em = 0;
            {
                D g[P];
#pragma unroll
                for (int i = 0, p = 0; i < R; ++i)
#pragma unroll
                    for (int j = 0; j <= i; ++j, ++p)
                        g[p] = dw_mul(dw_scale(from_dw<D>(Gk[p]), gsc), num_prod<D>(w[i], w[j]));
#pragma unroll 1
                for (int c = 0; c < R; ++c) {
                    float hc[R];
#pragma unroll
                    for (int j = 0; j < R; ++j) hc[j] = Hs[c * R + j];
                    D tv[R];
#pragma unroll
                    for (int i = 0; i < R; ++i) {
                        acc_t<D> s = acc0<D>();
#pragma unroll
                        for (int j = 0; j < R; ++j) acc_fmaf(s, g[pk<R>(i, j)], hc[j]);
                        tv[i] = acc_val(s);
                    }
                    int r = c;
                    for (; r + 1 < R; r += 2) {             // entries in pairs
                        acc_t<D> s0 = acc0<D>(), s1 = acc0<D>();
#pragma unroll
                        for (int i = 0; i < R; ++i) {
                            acc_fmaf(s0, tv[i], Hs[r * R + i]);
                            acc_fmaf(s1, tv[i], Hs[(r + 1) * R + i]);
                        }
                        const D m0 = acc_val(s0), m1 = acc_val(s1);
                        A(r, c) = m0;
                        A(r + 1, c) = m1;
                        if (r == c) em = max(em, f_expo(m0.h));
                    }
                    if (r < R) {
                        acc_t<D> s = acc0<D>();
#pragma unroll
                        for (int i = 0; i < R; ++i) acc_fmaf(s, tv[i], Hs[r * R + i]);
                        const D m = acc_val(s);
                        A(r, c) = m;
                        if (r == c) em = max(em, f_expo(m.h));
                    }
                }
            }
            if (eg == 0 || ew == 0 || em == 0) {
                // G, W or M is zero (or below the normal range): A_k = 0, Q_k = 0
                for (int i = 0; i < R * R; ++i) T[tb + i] = 0.f;
                if (qrcnt) qrcnt[k] = 0;
                if constexpr (MODE == 1) sc.meta[slot] = GRP_ZERO;
                live = false;
            } else {
                // M'' = M' 2^sm with max diag in [0.5, 2); sm + sg even so that
                // M^{-1/2} H S = 2^{(sm + sg) / 2} M''^{-1/2} H' S'
                int sm = 127 - em;
                if ((sm + sg) & 1) --sm;
                const float msc = f_pow2(sm);
#pragma unroll 1
                for (int r = 0; r < R; ++r)
                    for (int c = 0; c <= r; ++c) A(r, c) = dw_scale(A(r, c), msc);
                tridiagonalize_dw<R>(R, A, d, e);
                so = (sm + sg) / 2;
                if constexpr (MODE == 1) {
                    // hand Q_h (interleaved over the chunk), the tridiagonal
                    // and w' to the QR recorder and MODE 2
#pragma unroll 1
                    for (int r = 0; r < R; ++r)
#pragma unroll
                        for (int c = 0; c < R; ++c)
                            sc.qh[(size_t)(r * R + c) * sc.chunk + slot] = A(r, c);
                    D *de = sc.de + (size_t)slot * 2 * R;
#pragma unroll
                    for (int i = 0; i < R; ++i) {
                        de[i] = d[i];
                        de[R + i] = (i + 1 < R) ? e[i] : zero;
                        sc.wv[(size_t)slot * R + i] = w[i];
                    }
                    sc.meta[slot] = so;
                    live = false;
                } else {
                    int rot = 0;
                    const int steps = tridiagonal_qr_dw<R>(R, A, d, e, 30 * R, &rot);
                    if (steps < 0) atomicOr(&st->flags, FLAG_EIG_NOCONV);
                    flops = qr_flops(R, steps, rot);
                    if (qrcnt) qrcnt[k] = rot;
                }
            }
        } else {
            // Q_h, w' and the eigenvalues from the other kernels; subjects that
            // were zero, or whose rotations did not fit the record (finished by
            // MODE 0 instead), are skipped
            const int meta = sc.meta[slot];
            const int32_t nrec = sc.nrec[slot];
            live = meta != GRP_ZERO && nrec >= 0;
            if (live) {
                so = meta;
#pragma unroll 1
                for (int r = 0; r < R; ++r)
#pragma unroll
                    for (int c = 0; c < R; ++c)
                        A(r, c) = sc.qh[(size_t)(r * R + c) * sc.chunk + slot];
#pragma unroll
                for (int i = 0; i < R; ++i) {
                    dr[i] = sc.dout[(size_t)slot * R + i];
                    w[i] = sc.wv[(size_t)slot * R + i];
                }
                if constexpr (R > 1) {
                    // The rotations in the order the QR formed them, after the
                    // identity rotation on columns 0 and 1 that MODE 0 applies
                    // first; the records are loaded PF rotations ahead (each
                    // lane reads its own subject's, interleaved: coalesced).
                    {
                        const D nz = dw_neg(zero);
#pragma unroll
                        for (int i = 0; i < R; ++i) {
                            const D za = A(i, 0), zb = A(i, 1);
                            A(i, 0) = dw_dot2(one, za, nz, zb);
                            A(i, 1) = dw_dot2(zero, za, one, zb);
                        }
                    }
                    constexpr int PF = 4;
                    const RotRec<D> *rp = sc.rec + slot;
                    const uint8_t *kq = sc.rkr + slot;
                    const int64_t rs = sc.rstep;
                    RotRec<D> rb[PF];
                    int kb[PF];
#pragma unroll
                    for (int j = 0; j < PF; ++j) {
                        rb[j] = RotRec<D>{zero, zero};
                        kb[j] = 0;
                        if (j < nrec) {
                            rb[j] = rp[j * rs];
                            kb[j] = kq[j * rs];
                        }
                    }
#pragma unroll 1
                    for (int32_t n0 = 0; n0 < nrec; n0 += PF) {
#pragma unroll
                        for (int j = 0; j < PF; ++j) {
                            if (n0 + j < nrec) {
                                const D c = rb[j].c, s = rb[j].s;
                                const int kp = kb[j];
                                if (n0 + PF + j < nrec) {
                                    rb[j] = rp[(int64_t)(n0 + PF + j) * rs];
                                    kb[j] = kq[(int64_t)(n0 + PF + j) * rs];
                                }
                                const D ns = dw_neg(s);
                                D za[R], zb[R];
#pragma unroll
                                for (int i = 0; i < R; ++i) {
                                    za[i] = A(i, kp);
                                    zb[i] = A(i, kp + 1);
                                }
#pragma unroll
                                for (int i = 0; i < R; ++i) {
                                    A(i, kp) = dw_dot2(c, za[i], ns, zb[i]);
                                    A(i, kp + 1) = dw_dot2(s, za[i], c, zb[i]);
                                }
                            }
                        }
                    }
                }
            }
        }
        if constexpr (MODE != 1) {
            if (live) {
                float lmax = 0.f;
#pragma unroll
                for (int i = 0; i < R; ++i) {
                    if constexpr (MODE == 2)
                        lmax = fmaxf(lmax, dr[i].h);
                    else
                        lmax = fmaxf(lmax, d[i].h);
                }
                const float cut = rtol2 * lmax;
                auto cut_column = [&](int i, D di) {
                    const D sf = (lmax > 0.f && di.h > cut) ? dw_sqrt(dw_rsqrt(di)) : zero;  // d^-1/4
#pragma unroll
                    for (int r = 0; r < R; ++r) A(r, i) = dw_mul(A(r, i), sf);
                };
                if constexpr (MODE == 2) {
#pragma unroll
                    for (int i = 0; i < R; ++i) cut_column(i, dr[i]);
                } else {
#pragma unroll 1
                    for (int i = 0; i < R; ++i) cut_column(i, d[i]);
                }
                const float o1 = f_pow2(so / 2), o2 = f_pow2(so - so / 2);
                if constexpr (R <= 10) {
                    // C = Z' Z'^T (packed lower, in registers) by rank-one updates,
                    // one column of Z' at a time, then T = C H' S'
                    acc_t<D> C[P];
#pragma unroll
                    for (int p = 0; p < P; ++p) C[p] = acc0<D>();
#pragma unroll 1
                    for (int i = 0; i < R; ++i) {
                        D a[R];
#pragma unroll
                        for (int r = 0; r < R; ++r) a[r] = A(r, i);
#pragma unroll
                        for (int r = 0, p = 0; r < R; ++r)
#pragma unroll
                            for (int c = 0; c <= r; ++c, ++p) acc_fma(C[p], a[r], a[c]);
                    }
                    D Cv[P];
#pragma unroll
                    for (int p = 0; p < P; ++p) Cv[p] = acc_val(C[p]);
#pragma unroll 1
                    for (int c = 0; c < R; ++c) {
                        float hc[R];
#pragma unroll
                        for (int u = 0; u < R; ++u) hc[u] = Hs[u * R + c];
                        float wc = 0.f;
#pragma unroll
                        for (int u = 0; u < R; ++u) wc = (u == c) ? w[u] : wc;
#pragma unroll
                        for (int r = 0; r < R; ++r) {             // T(r, c) = (C h'_c)_r w'_c
                            acc_t<D> t = acc0<D>();
#pragma unroll
                            for (int u = 0; u < R; ++u) acc_fmaf(t, Cv[pk<R>(r, u)], hc[u]);
                            const D v = dw_mulf(acc_val(t), wc);
                            T[tb + r * R + c] = store_f(v, o1, o2);
                        }
                    }
                } else {
#pragma unroll
                    for (int i = 0; i < R; ++i) e[i] = num_f<D>(w[i]);    // w' where the T loop can index it
#pragma unroll 1
                    for (int c = 0; c < R; ++c) {
                        D y[R];                                 // y = Z'^T h'_c
                        {
                            acc_t<D> s[R];
#pragma unroll
                            for (int i = 0; i < R; ++i) s[i] = acc0<D>();
#pragma unroll 1
                            for (int r = 0; r < R; ++r) {
                                const float hr = Hs[r * R + c];
#pragma unroll
                                for (int i = 0; i < R; ++i) acc_fmaf(s[i], A(r, i), hr);
                            }
#pragma unroll
                            for (int i = 0; i < R; ++i) y[i] = acc_val(s[i]);
                        }
#pragma unroll 1
                        for (int r = 0; r < R; ++r) {             // T(r, c) = (Z' y)_r w'_c
                            acc_t<D> s = acc0<D>();
#pragma unroll
                            for (int i = 0; i < R; ++i) acc_fma(s, A(r, i), y[i]);
                            const D v = dw_mulf(acc_val(s), e[c].h);
                            T[tb + r * R + c] = store_f(v, o1, o2);
                        }
                    }
                }
                flops += polar_fixed_flops(R);
            }
        }
    }
    add_flops(st, flops);
}

// ---- Q-step order -------------------------------------------------------------
// Lanes (or lane groups) of a warp run their QR iterations in lock step until
// the slowest has converged, so subjects are processed in decreasing order of
// the rotation count of their previous Q-step (which changes little between
// ALS iterations): a counting sort into 256 bins of min(count, 255), chunked
// so that no global atomics are needed.  The order within a bin is arbitrary;
// every subject's result is independent of the slot that computes it.
__global__ void __launch_bounds__(256) k_order_count(const int32_t *__restrict__ cnt, int64_t K,
                                                      int32_t *rank, int32_t *binoff) {
    __shared__ int h[P2_ORDER_BINS];
    for (int i = threadIdx.x; i < P2_ORDER_BINS; i += blockDim.x) h[i] = 0;
    __syncthreads();
    const int64_t a = (int64_t)blockIdx.x * P2_ORDER_CHUNK;
    const int64_t b = (a + P2_ORDER_CHUNK < K) ? (a + P2_ORDER_CHUNK) : K;
    for (int64_t k = a + threadIdx.x; k < b; k += blockDim.x) {
        const int v = min(max((int)cnt[k], 0), P2_ORDER_BINS - 1);
        rank[k] = atomicAdd(&h[v], 1);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < P2_ORDER_BINS; i += blockDim.x)
        binoff[(size_t)blockIdx.x * P2_ORDER_BINS + i] = h[i];
}

// one block of P2_ORDER_BINS threads: per-chunk bin counts -> slot offsets,
// bins in decreasing order of the count
__global__ void __launch_bounds__(P2_ORDER_BINS) k_order_scan(int32_t *binoff, int nchunk) {
    __shared__ int tot[P2_ORDER_BINS];
    const int b = threadIdx.x;
    int run = 0;
    for (int j = 0; j < nchunk; ++j) {
        const int v = binoff[(size_t)j * P2_ORDER_BINS + b];
        binoff[(size_t)j * P2_ORDER_BINS + b] = run;
        run += v;
    }
    tot[b] = run;
    __syncthreads();
    int off = 0;
    for (int b2 = P2_ORDER_BINS - 1; b2 > b; --b2) off += tot[b2];
    for (int j = 0; j < nchunk; ++j) binoff[(size_t)j * P2_ORDER_BINS + b] += off;
}

__global__ void __launch_bounds__(256) k_order_place(const int32_t *__restrict__ cnt,
                                                      const int32_t *__restrict__ rank,
                                                      const int32_t *__restrict__ binoff,
                                                      int64_t K, int32_t *order) {
    const int64_t a = (int64_t)blockIdx.x * P2_ORDER_CHUNK;
    const int64_t b = (a + P2_ORDER_CHUNK < K) ? (a + P2_ORDER_CHUNK) : K;
    const int32_t *off = binoff + (size_t)blockIdx.x * P2_ORDER_BINS;
    for (int64_t k = a + threadIdx.x; k < b; k += blockDim.x) {
        const int v = min(max((int)cnt[k], 0), P2_ORDER_BINS - 1);
        order[off[v] + rank[k]] = (int32_t)k;
    }
}

template <int R, class D, int MODE = 0>
static int launch_reg(const p2_ctx *c, const dw *G, const float *W, SmallState *st, float *T,
                      int64_t K, cudaStream_t s, float rtol2, const int32_t *order,
                      int32_t *qrcnt, GrpSplit<D> sc = GrpSplit<D>{}) {
    constexpr int nt = reg_threads<R, MODE>();
    const size_t smem = reg_hbytes<R>() + (size_t)nt * reg_lane_bytes<R, MODE>();
    if (nt < 32 || smem > (size_t)c->geo.smem_optin) return -1;
    const int nblk = (int)((K + nt - 1) / nt);
    k_polar_reg<R, D, MODE><<<nblk, nt, smem, s>>>(G, W, st, T, K, rtol2, order, qrcnt, sc);
    return 0;
}

// Pointers into the context's scratch for one chunk of the lane kernel's
// split step (the regions of the grouped kernel's split step; the records
// and Q_h interleaved over the chunk's slots).
static GrpSplit<dw> reg_split_scratch(const p2_ctx *c) {
    const int64_t CH = c->split_chunk, R = c->R, cap = c->split_cap;
    unsigned char *b = c->d_split;
    auto take = [&b](size_t bytes) {
        unsigned char *p = b;
        b += (bytes + 255) & ~(size_t)255;
        return p;
    };
    GrpSplit<dw> sc;
    sc.qh = reinterpret_cast<dw *>(take(sizeof(dw) * CH * R * R));
    sc.de = reinterpret_cast<dw *>(take(sizeof(dw) * CH * 2 * R));
    sc.dout = reinterpret_cast<dw *>(take(sizeof(dw) * CH * R));
    sc.wv = reinterpret_cast<float *>(take(sizeof(float) * CH * R));
    sc.meta = reinterpret_cast<int *>(take(sizeof(int) * CH));
    sc.nrec = reinterpret_cast<int32_t *>(take(sizeof(int32_t) * CH));
    sc.rec = reinterpret_cast<RotRec<dw> *>(take(sizeof(RotRec<dw>) * CH * cap));
    sc.rkr = reinterpret_cast<uint8_t *>(take((size_t)CH * cap));
    sc.cap = cap;
    const int64_t want = c->tune.split_record_cap;
    sc.lim = (want > 0 && want < cap) ? want : cap;
    sc.rsub = 1;
    sc.rstep = CH;
    sc.chunk = CH;
    return sc;
}

// The split step of the lane kernel over chunks of subjects: MODE 1,
// k_qr_record, MODE 2, then MODE 0 for the subjects whose rotations did not
// fit (k_split_collect lists them).
template <int R>
static int launch_reg_split(const p2_ctx *c, const dw *G, const float *W, SmallState *st,
                            float *T, int64_t K, cudaStream_t s, float rtol2,
                            const int32_t *order, int32_t *qrcnt) {
    GrpSplit<dw> sc = reg_split_scratch(c);
    const int64_t CH = c->split_chunk;
    const int nt = QR_THREADS;
    const size_t smb = (size_t)2 * R * nt * sizeof(dw);
    for (int64_t c0 = 0; c0 < K; c0 += CH) {
        const int64_t n = (K - c0) < CH ? (K - c0) : CH;
        const int32_t *ord = order + c0;
        if (launch_reg<R, dw, 1>(c, G, W, st, T, n, s, rtol2, ord, qrcnt, sc) != 0) return -1;
        k_qr_record<R, dw><<<(unsigned)((n + nt - 1) / nt), nt, smb, s>>>(sc, n, R, ord, qrcnt, st);
        if (launch_reg<R, dw, 2>(c, G, W, st, T, n, s, rtol2, ord, qrcnt, sc) != 0) return -1;
        cudaMemsetAsync(c->d_split_cnt, 0, sizeof(int32_t), s);
        k_split_collect<<<(unsigned)((n + 255) / 256 < 1024 ? (n + 255) / 256 : 1024), 256, 0, s>>>(
            sc.nrec, n, ord, c->d_split_list, c->d_split_cnt);
        GrpSplit<dw> fb{};
        fb.kdev = c->d_split_cnt;
        if (launch_reg<R, dw, 0>(c, G, W, st, T, n, s, rtol2, c->d_split_list, qrcnt, fb) != 0)
            return -1;
    }
    return 0;
}

// the lane kernel's split step: double-word arithmetic, R >= 2, the scratch
// allocated, the subjects in a Q-step order and the tuning selecting it
static bool use_reg_split(const p2_ctx *c, int64_t K, const int32_t *order) {
    return c->R >= 2 && c->R <= 12 && !c->opt.fp64_procrustes && c->d_split && order && K > 0 &&
           c->tune.procrustes_split;
}

template <class D>
static cudaError_t allow_reg(int cap) {
    cudaError_t e = cudaSuccess;
#define P2_ALLOW(r) \
    if (e == cudaSuccess) \
        e = cudaFuncSetAttribute(k_polar_reg<r, D, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, cap); \
    if constexpr (std::is_same<D, dw>::value) { \
        if (e == cudaSuccess) \
            e = cudaFuncSetAttribute(k_polar_reg<r, D, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, cap); \
        if (e == cudaSuccess) \
            e = cudaFuncSetAttribute(k_polar_reg<r, D, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, cap); \
    }
    P2_ALLOW(1);
    P2_ALLOW(2);
    P2_ALLOW(3);
    P2_ALLOW(4);
    P2_ALLOW(5);
    P2_ALLOW(6);
    P2_ALLOW(7);
    P2_ALLOW(8);
    P2_ALLOW(9);
    P2_ALLOW(10);
    P2_ALLOW(11);
    P2_ALLOW(12);
#undef P2_ALLOW
    return e;
}

bool tc_m_wanted(const p2_ctx *c) {
    if (c->opt.fp64_procrustes || !form_m_tc_supported(c->R)) return false;
    return c->opt.tensor_core_m > 0;
}

int polar_configure(p2_ctx *c) {
    const int cap = c->geo.smem_optin;
    cudaError_t e = c->opt.fp64_procrustes ? allow_reg<f64n>(cap) : allow_reg<dw>(cap);
    if (e == cudaSuccess) e = polar_grp_configure(cap, c->opt.fp64_procrustes != 0);
    if (e == cudaSuccess && tc_m_wanted(c)) e = form_m_tc_configure(c->R);
    if (e != cudaSuccess) {
        set_error("configuring the Procrustes kernels: %s", cudaGetErrorString(e));
        return P2_ECUDA;
    }
    return P2_OK;
}

// Enqueue the Procrustes kernel for K subjects (Gram G, weights W, state st
// holding H64) writing T; returns a cudaError_t.
cudaError_t launch_polar_on(const p2_ctx *c, const dw *G, const float *W, SmallState *st,
                            float *T, int64_t K, cudaStream_t s, const int32_t *order,
                            int32_t *qrcnt, const dw *mpre) {
    const int R = c->R;
    const double rtol2 = c->opt.rank_rtol * c->opt.rank_rtol;
    if (K <= 0) return cudaSuccess;
    if (R > 12) return launch_polar_grp(c, G, W, st, T, K, s, rtol2, order, qrcnt, mpre);
    const float rt2 = (float)rtol2;
    const bool f64 = c->opt.fp64_procrustes != 0;
    int rc = -1;
    const bool split = use_reg_split(c, K, order);
    switch (R) {
#define P2_CASE(r) \
        case r: rc = f64 ? launch_reg<r, f64n>(c, G, W, st, T, K, s, rt2, order, qrcnt) \
                   : split ? launch_reg_split<r>(c, G, W, st, T, K, s, rt2, order, qrcnt) \
                           : launch_reg<r, dw>(c, G, W, st, T, K, s, rt2, order, qrcnt); break;
        P2_CASE(1) P2_CASE(2) P2_CASE(3) P2_CASE(4) P2_CASE(5) P2_CASE(6)
        P2_CASE(7) P2_CASE(8) P2_CASE(9) P2_CASE(10) P2_CASE(11) P2_CASE(12)
#undef P2_CASE
        default: break;
    }
    if (rc != 0) return cudaErrorInvalidConfiguration;   // shared memory below 32 lanes' need
    return cudaGetLastError();
}

cudaError_t launch_order_desc(const int32_t *key, int64_t K, int32_t *rank, int32_t *binoff,
                              int32_t *order, cudaStream_t s) {
    if (K <= 0) return cudaSuccess;
    const int nchunk = (int)((K + P2_ORDER_CHUNK - 1) / P2_ORDER_CHUNK);
    k_order_count<<<nchunk, 256, 0, s>>>(key, K, rank, binoff);
    k_order_scan<<<1, P2_ORDER_BINS, 0, s>>>(binoff, nchunk);
    k_order_place<<<nchunk, 256, 0, s>>>(key, rank, binoff, K, order);
    return cudaGetLastError();
}

// key of a subject's bin: its non-zero count in steps of four, clamped
__global__ void k_subject_key(const int64_t *__restrict__ subj_nnz, int64_t K, int32_t *key) {
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < K;
         k += (int64_t)gridDim.x * blockDim.x) {
        const int64_t n = subj_nnz[k + 1] - subj_nnz[k];
        key[k] = (int32_t)((n >> 2) < P2_ORDER_BINS - 1 ? (n >> 2) : P2_ORDER_BINS - 1);
    }
}

cudaError_t launch_subject_bins(p2_ctx *c) {
    const int64_t K = c->X.K;
    if (K <= 0) return cudaSuccess;
    // the rotation counts are not in use yet (zero until the first Q-step):
    // their buffer holds the keys, and is cleared again afterwards
    k_subject_key<<<(int)std::min<int64_t>((K + 255) / 256, 4096), 256, 0, c->stream>>>(
        c->X.subj_nnz, K, c->d_qrcnt);
    cudaError_t e = launch_order_desc(c->d_qrcnt, K, c->d_rank, c->d_binoff, c->d_sorder,
                                      c->stream);
    if (e == cudaSuccess)
        e = cudaMemsetAsync(c->d_qrcnt, 0, sizeof(int32_t) * (size_t)K, c->stream);
    return e;
}

// The Q-step of the iteration: order the subjects by their last rotation
// counts, form every subject's M' on the tensor cores where selected, then
// the Procrustes kernel(s) (polar_launches kernels in all).
cudaError_t launch_polar(p2_ctx *c) {
    const int64_t K = c->X.K;
    if (K <= 0) return cudaSuccess;
    cudaError_t e = launch_order_desc(c->d_qrcnt, K, c->d_rank, c->d_binoff, c->d_order,
                                      c->stream);
    if (e != cudaSuccess) return e;
    if (c->d_Mtc) {
        e = launch_form_m_tc(c, c->d_G, c->d_W, c->d_s, c->d_Mtc, K, c->stream);
        if (e != cudaSuccess) return e;
    }
    return launch_polar_on(c, c->d_G, c->d_W, c->d_s, c->d_T, K, c->stream, c->d_order,
                           c->d_qrcnt, c->d_Mtc);
}

int polar_launches(const p2_ctx *c) {
    const int64_t K = c->X.K;
    if (K <= 0) return 0;
    int n = 3 + (c->d_Mtc ? 1 : 0);                      // ordering (+ M' on the tensor cores)
    if (c->R >= 2 && !c->opt.fp64_procrustes && c->d_split && c->tune.procrustes_split) {
        const int64_t chunks = (K + c->split_chunk - 1) / c->split_chunk;
        n += (int)(5 * chunks);                          // MODE 1, QR record, MODE 2, collect, fallback
    } else {
        n += 1;
    }
    return n;
}

}  // namespace p2
