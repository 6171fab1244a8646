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

#include "p2_internal.cuh"
#include "p2_eig_dw.cuh"
#include "p2_polar.cuh"

namespace p2 {

template <int R>
static __device__ __forceinline__ int pk(int i, int j) {   // packed lower index
    return (j <= i) ? (i * (i + 1) / 2 + j) : (j * (j + 1) / 2 + i);
}

// Shared memory: H (scaled, FP32) for the block, then per lane the working
// matrix (R x R) and the tridiagonal (d, e), interleaved across the lanes:
// R^2 + 2R double-words per lane.
template <int R, class D>
__global__ void __launch_bounds__(256, 1) k_polar_reg(const dw *__restrict__ G,
                                                   const float *__restrict__ W, SmallState *st,
                                                   float *T, int64_t K, float rtol2,
                                                   const int32_t *__restrict__ order,
                                                   int32_t *qrcnt) {
    constexpr int P = R * (R + 1) / 2;
    constexpr int HW = (R * R + 1) / 2;                  // double-word slots holding H
    extern __shared__ __align__(16) unsigned char smr_raw[];
    D *smd = reinterpret_cast<D *>(smr_raw);
    const int NT = blockDim.x;
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
    unsigned long long flops = 0;
    if (slot < K) {
        const int64_t k = order ? (int64_t)order[slot] : slot;
        const D zero = num_f<D>(0.f);
        DwMat<D> A{th + t, NT, R};
        DwVec<D> d{th + (size_t)R * R * NT + t, NT};
        DwVec<D> e{th + (size_t)(R * R + R) * NT + t, NT};
        const size_t tb = (size_t)k * R * R;
        const dw *Gk = G + (size_t)k * P;
        float w[R];
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
                for (int r = c; r < R; ++r) {
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
            int rot = 0;
            const int steps = tridiagonal_qr_dw<R>(R, A, d, e, 30 * R, &rot);
            if (steps < 0) atomicOr(&st->flags, FLAG_EIG_NOCONV);
            float lmax = 0.f;
#pragma unroll
            for (int i = 0; i < R; ++i) lmax = fmaxf(lmax, d[i].h);
            const float cut = rtol2 * lmax;
#pragma unroll 1
            for (int i = 0; i < R; ++i) {
                const D di = d[i];
                const D sf = (lmax > 0.f && di.h > cut) ? dw_sqrt(dw_rsqrt(di)) : zero;  // d^-1/4
#pragma unroll
                for (int r = 0; r < R; ++r) A(r, i) = dw_mul(A(r, i), sf);
            }
            const int so = (sm + sg) / 2;
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
            flops = polar_fixed_flops(R) + qr_flops(R, steps, rot);
            if (qrcnt) qrcnt[k] = rot;
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

template <int R, class D>
static int launch_reg(const p2_ctx *c, const dw *G, const float *W, SmallState *st, float *T,
                      int64_t K, cudaStream_t s, float rtol2, const int32_t *order,
                      int32_t *qrcnt) {
    const int cap = c->geo.smem_optin;
    const size_t hbytes = (size_t)((R * R + 1) / 2) * sizeof(dw);
    const size_t per = (size_t)(R * R + 2 * R) * sizeof(dw);
    int nt = (int)((cap - hbytes) / per);
    if (nt > 256) nt = 256;
    nt = (nt / 32) * 32;
    if (nt < 32) return -1;
    const size_t smem = hbytes + (size_t)nt * per;
    const int nblk = (int)((K + nt - 1) / nt);
    k_polar_reg<R, D><<<nblk, nt, smem, s>>>(G, W, st, T, K, rtol2, order, qrcnt);
    return 0;
}

template <class D>
static cudaError_t allow_reg(int cap) {
    cudaError_t e = cudaSuccess;
#define P2_ALLOW(r) \
    if (e == cudaSuccess) \
        e = cudaFuncSetAttribute(k_polar_reg<r, D>, cudaFuncAttributeMaxDynamicSharedMemorySize, cap)
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
    switch (R) {
#define P2_CASE(r) \
        case r: rc = f64 ? launch_reg<r, f64n>(c, G, W, st, T, K, s, rt2, order, qrcnt) \
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
    if (c->R > 12 && !c->opt.fp64_procrustes && c->d_split && c->tune.procrustes_split) {
        const int64_t chunks = (K + c->split_chunk - 1) / c->split_chunk;
        n += (int)(5 * chunks);                          // MODE 1, QR record, MODE 2, collect, fallback
    } else {
        n += 1;
    }
    return n;
}

}  // namespace p2
