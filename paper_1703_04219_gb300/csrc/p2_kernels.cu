// Kernels of one PARAFAC2-ALS iteration in SPARTan's formulation.
//
// Notation (Perros et al., KDD 2017, Sections 3-4): X_k is I_k x J sparse,
// H is R x R, V is J x R, W is K x R and S_k = diag(W(k,:)).
//
// The schedule works on per-subject R x R state instead of materialising
// Q_k or Y_k (identities that follow from the paper's definitions):
//   Z_k = X_k V                       (never stored; recomputed per pass)
//   A_k = Z_k S_k H^T                 (Procrustes input: H S_k V^T X_k^T = A_k^T)
//   G_k = Z_k^T Z_k                   (accumulated in FP64)
//   C_k = (A_k^T A_k)^{+1/2}, Q_k = A_k C_k   (polar factor, FP64)
//   T_k = C_k H S_k, so Q_k = Z_k T_k^T and Y_k = Q_k^T X_k = T_k Z_k^T X_k
//   mode 1 (Eq. mttkrp1_3):  Y_k V = T_k G_k
//   mode 2 (Eq. mttkrp2_3):  Y_k^T H S_k = X_k^T (Z_k F_k), F_k = T_k^T H S_k
//   mode 3 (Eq. mttkrp3_row_wise): Y_k V' = T_k Z_k^T Z'_k, Z'_k = X_k V'
// so an iteration streams X twice: pass beta (mode 2) and pass alpha (mode
// 3, the W row, and the next Q-step's Gram), with the R x R work in between.
//
// Determinism: every reduction over subjects uses fixed per-block partials
// summed in block order; the only atomics are 64-bit integer adds of
// fixed-point mode-2 terms, which are associative.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "p2_internal.cuh"
#include "p2_eig.cuh"

namespace p2 {

#define FULLMASK 0xffffffffu

static __device__ __forceinline__ int warp_excl_scan(int v, int lane) {
    int x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(FULLMASK, x, o);
        if (lane >= o) x += y;
    }
    return x - v;
}

struct XView {
    const int64_t *__restrict__ subj_row;
    const int64_t *__restrict__ subj_nnz;
    const uint16_t *__restrict__ row_len;
    const uint16_t *__restrict__ col;
    const float *__restrict__ val;
    int64_t K;
};

static XView xview(const p2_ctx *c) {
    return XView{c->X.subj_row, c->X.subj_nnz, c->X.row_len, c->X.col, c->X.val, c->X.K};
}

// z rows of up to 32 consecutive rows: z1[i][:] = X(row i, :) V1 and, when
// TWO, z2[i][:] = X(row i, :) V2.  LPR lanes share a row (lane sub-index
// covers components sub and sub + LPR), RPP rows per pass.  FP32 FMA in
// column order within a row.
template <bool TWO>
static __device__ __forceinline__ void gather_rows(const XView &X, int nr, int64_t base, int len,
                                                   int off, const float *__restrict__ V1,
                                                   const float *__restrict__ V2, float *z1,
                                                   float *z2, int R, int LPR, int RPP, int lane) {
    const int g = lane / LPR;
    const int sub = lane - g * LPR;
    for (int i0 = 0; i0 < nr; i0 += RPP) {
        const int i = i0 + g;
        const int src = (i < 32) ? i : 31;
        const int ro = __shfl_sync(FULLMASK, off, src);
        const int rl = __shfl_sync(FULLMASK, len, src);
        const bool valid = (g < RPP) && (i < nr);
        float a1[2] = {0.f, 0.f}, a2[2] = {0.f, 0.f};
        if (valid) {
            for (int e = 0; e < rl; ++e) {
                const int64_t idx = base + ro + e;
                const int j = X.col[idx];
                const float x = X.val[idx];
                const float *v1 = V1 + (size_t)j * R;
                const float *v2 = TWO ? (V2 + (size_t)j * R) : nullptr;
#pragma unroll
                for (int t = 0; t < 2; ++t) {
                    const int c = sub + t * LPR;
                    if (c < R) {
                        a1[t] = fmaf(x, __ldg(v1 + c), a1[t]);
                        if (TWO) a2[t] = fmaf(x, __ldg(v2 + c), a2[t]);
                    }
                }
            }
#pragma unroll
            for (int t = 0; t < 2; ++t) {
                const int c = sub + t * LPR;
                if (c < R) {
                    z1[i * R + c] = a1[t];
                    if (TWO) z2[i * R + c] = a2[t];
                }
            }
        }
    }
}

// ---------------------------------------------------------------------------
// Pass alpha: for each subject, Gram of Z'_k = X_k V (FP64, packed lower)
// and, with MODE3, the mode-3 MTTKRP row M3(k,:) = coldot(H, T_k Z_k^T Z'_k)
// with Z_k = X_k Vprev, followed by W(k,:) = M3(k,:) (V^TV * H^TH)^+.
// ---------------------------------------------------------------------------
template <bool MODE3>
__global__ void __launch_bounds__(512) k_alpha(XView X, const float *__restrict__ Vprev,
                                               const float *__restrict__ V,
                                               const float *__restrict__ H,
                                               const float *__restrict__ T,
                                               const SmallState *__restrict__ st, double *G,
                                               float *W, float *M3, int R) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int P = R * (R + 1) / 2;
    const int LPR = R < 32 ? R : 32;
    const int RPP = 32 / LPR;
    // CTA-shared: G3inv (R*R doubles), H (R*R floats), packed index table
    double *G3s = reinterpret_cast<double *>(smem_raw);
    float *Hs = reinterpret_cast<float *>(G3s + R * R);
    uint8_t *pr = reinterpret_cast<uint8_t *>(Hs + R * R);
    uint8_t *pc = pr + P;
    size_t cta_bytes = ((size_t)R * R * 8 + (size_t)R * R * 4 + 2 * (size_t)P + 15) & ~(size_t)15;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const size_t warp_bytes = (size_t)P * 8 + ((size_t)64 * R + 2 * (size_t)R * R) * 4;
    unsigned char *wb = smem_raw + cta_bytes + warp * warp_bytes;
    double *Gacc = reinterpret_cast<double *>(wb);
    float *zo = reinterpret_cast<float *>(Gacc + P);   // 32 R  (zo and zn contiguous: 64 R scratch)
    float *zn = zo + 32 * R;                            // 32 R
    float *Tk = zn + 32 * R;                            // R R
    float *Cacc = Tk + R * R;                           // R R

    for (int i = threadIdx.x; i < R * R; i += blockDim.x) {
        G3s[i] = st->G3inv[i];
        Hs[i] = H[i];
    }
    for (int p = threadIdx.x; p < P; p += blockDim.x) {
        int r = (int)((sqrt(8.0 * p + 1.0) - 1.0) * 0.5);
        while ((r + 1) * (r + 2) / 2 <= p) ++r;
        while (r * (r + 1) / 2 > p) --r;
        pr[p] = (uint8_t)r;
        pc[p] = (uint8_t)(p - r * (r + 1) / 2);
    }
    __syncthreads();

    const int64_t nwarps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t k = (int64_t)blockIdx.x * (blockDim.x >> 5) + warp; k < X.K; k += nwarps) {
        const int64_t r0 = X.subj_row[k], r1 = X.subj_row[k + 1];
        int64_t base = X.subj_nnz[k];
        for (int p = lane; p < P; p += 32) Gacc[p] = 0.0;
        if (MODE3)
            for (int e = lane; e < R * R; e += 32) Cacc[e] = 0.f;
        for (int64_t cr = r0; cr < r1; cr += 32) {
            const int nr = (int)((r1 - cr) < 32 ? (r1 - cr) : 32);
            const int len = (lane < nr) ? (int)X.row_len[cr + lane] : 0;
            const int off = warp_excl_scan(len, lane);
            const int tot = __shfl_sync(FULLMASK, off + len, 31);
            if (MODE3)
                gather_rows<true>(X, nr, base, len, off, Vprev, V, zo, zn, R, LPR, RPP, lane);
            else
                gather_rows<false>(X, nr, base, len, off, V, nullptr, zn, nullptr, R, LPR, RPP,
                                   lane);
            __syncwarp();
            if (MODE3) {
                for (int e = lane; e < R * R; e += 32) {
                    const int r = e / R, s = e - r * R;
                    float acc = 0.f;
                    for (int i = 0; i < nr; ++i) acc = fmaf(zo[i * R + r], zn[i * R + s], acc);
                    Cacc[e] += acc;
                }
            }
            for (int p = lane; p < P; p += 32) {
                const int r = pr[p], s = pc[p];
                double acc = 0.0;
                for (int i = 0; i < nr; ++i)
                    acc = fma((double)zn[i * R + r], (double)zn[i * R + s], acc);
                Gacc[p] += acc;
            }
            __syncwarp();
            base += tot;
        }
        double *Gk = G + (size_t)k * P;
        for (int p = lane; p < P; p += 32) Gk[p] = Gacc[p];
        if (MODE3) {
            const float *Tg = T + (size_t)k * R * R;
            for (int e = lane; e < R * R; e += 32) Tk[e] = Tg[e];
            __syncwarp();
            float *scr = zo;   // 64 R >= R R floats of scratch
            for (int e = lane; e < R * R; e += 32) {
                const int r = e / R, s = e - r * R;
                float b = 0.f;
                for (int u = 0; u < R; ++u) b = fmaf(Tk[r * R + u], Cacc[u * R + s], b);
                scr[e] = Hs[e] * b;
            }
            __syncwarp();
            for (int s = lane; s < R; s += 32) {
                float m = 0.f;
                for (int r = 0; r < R; ++r) m += scr[r * R + s];
                M3[(size_t)k * R + s] = m;
                Tk[s] = m;
            }
            __syncwarp();
            for (int s = lane; s < R; s += 32) {
                double w = 0.0;
                for (int u = 0; u < R; ++u) w = fma((double)Tk[u], G3s[u * R + s], w);
                W[(size_t)k * R + s] = (float)w;
            }
            __syncwarp();
        }
    }
}

// ---------------------------------------------------------------------------
// Pass beta: mode-2 MTTKRP M2 = sum_k X_k^T (Z_k F_k), F_k = T_k^T H S_k.
// Terms are rounded to 64-bit fixed point with a per-component power-of-two
// scale and added with integer atomics (order independent).  Columns below
// Hc (the most frequent after relabelling) accumulate in shared memory first.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(512) k_beta(XView X, const float *__restrict__ V,
                                              const float *__restrict__ H,
                                              const float *__restrict__ T,
                                              const float *__restrict__ W,
                                              SmallState *st, unsigned long long *m2acc,
                                              int R, int Hc) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int LPR = R < 32 ? R : 32;
    const int RPP = 32 / LPR;
    unsigned long long *hot = reinterpret_cast<unsigned long long *>(smem_raw);
    float *Hs = reinterpret_cast<float *>(hot + (size_t)Hc * R);
    float *scale = Hs + R * R;
    size_t cta_bytes = ((size_t)Hc * R * 8 + (size_t)R * R * 4 + (size_t)R * 4 + 15) & ~(size_t)15;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const size_t warp_bytes = ((size_t)64 * R + 2 * (size_t)R * R + R) * 4;
    float *zo = reinterpret_cast<float *>(smem_raw + cta_bytes + warp * warp_bytes);
    float *pp = zo + 32 * R;
    float *Tk = pp + 32 * R;
    float *Fk = Tk + R * R;
    float *wk = Fk + R * R;

    for (int i = threadIdx.x; i < Hc * R; i += blockDim.x) hot[i] = 0ull;
    for (int i = threadIdx.x; i < R * R; i += blockDim.x) Hs[i] = H[i];
    for (int i = threadIdx.x; i < R; i += blockDim.x) scale[i] = st->m2scale[i];
    __syncthreads();
    const float lim = 4.0e18f;   // < 2^62
    bool ovf = false;

    const int64_t nwarps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t k = (int64_t)blockIdx.x * (blockDim.x >> 5) + warp; k < X.K; k += nwarps) {
        const int64_t r0 = X.subj_row[k], r1 = X.subj_row[k + 1];
        if (r1 == r0) continue;
        int64_t base = X.subj_nnz[k];
        const float *Tg = T + (size_t)k * R * R;
        for (int e = lane; e < R * R; e += 32) Tk[e] = Tg[e];
        for (int s = lane; s < R; s += 32) wk[s] = W[(size_t)k * R + s];
        __syncwarp();
        for (int e = lane; e < R * R; e += 32) {
            const int u = e / R, s = e - u * R;
            float f = 0.f;
            for (int r = 0; r < R; ++r) f = fmaf(Tk[r * R + u], Hs[r * R + s], f);
            Fk[e] = f * wk[s];
        }
        __syncwarp();
        for (int64_t cr = r0; cr < r1; cr += 32) {
            const int nr = (int)((r1 - cr) < 32 ? (r1 - cr) : 32);
            const int len = (lane < nr) ? (int)X.row_len[cr + lane] : 0;
            const int off = warp_excl_scan(len, lane);
            const int tot = __shfl_sync(FULLMASK, off + len, 31);
            gather_rows<false>(X, nr, base, len, off, V, nullptr, zo, nullptr, R, LPR, RPP, lane);
            __syncwarp();
            for (int e = lane; e < nr * R; e += 32) {
                const int i = e / R, s = e - i * R;
                float p = 0.f;
                for (int u = 0; u < R; ++u) p = fmaf(zo[i * R + u], Fk[u * R + s], p);
                pp[e] = p;
            }
            __syncwarp();
            const int g = lane / LPR, sub = lane - g * LPR;
            for (int i0 = 0; i0 < nr; i0 += RPP) {
                const int i = i0 + g;
                const int src = (i < 32) ? i : 31;
                const int ro = __shfl_sync(FULLMASK, off, src);
                const int rl = __shfl_sync(FULLMASK, len, src);
                if ((g < RPP) && (i < nr)) {
                    for (int e = 0; e < rl; ++e) {
                        const int64_t idx = base + ro + e;
                        const int j = X.col[idx];
                        const float x = X.val[idx];
#pragma unroll
                        for (int t = 0; t < 2; ++t) {
                            const int c = sub + t * LPR;
                            if (c < R) {
                                float v = x * pp[i * R + c] * scale[c];
                                if (!(fabsf(v) < lim)) {
                                    ovf = true;
                                    v = (v != v) ? 0.f : copysignf(lim, v);
                                }
                                const long long q = __float2ll_rn(v);
                                if (q != 0) {
                                    if (j < Hc)
                                        atomicAdd(&hot[(size_t)j * R + c], (unsigned long long)q);
                                    else
                                        atomicAdd(&m2acc[(size_t)j * R + c], (unsigned long long)q);
                                }
                            }
                        }
                    }
                }
            }
            __syncwarp();
            base += tot;
        }
    }
    if (ovf) atomicOr(&st->flags, FLAG_FIXED_OVF);
    __syncthreads();
    for (int i = threadIdx.x; i < Hc * R; i += blockDim.x)
        if (hot[i] != 0ull) atomicAdd(&m2acc[i], hot[i]);
}

// M2 = fixed-point sums scaled back to FP64; accumulators reset for next use.
__global__ void k_m2_finalize(unsigned long long *m2acc, double *M2, const SmallState *st,
                              int64_t n, int R) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int s = (int)(e % R);
        const long long q = (long long)m2acc[e];
        M2[e] = (double)q * st->m2inv[s];
        m2acc[e] = 0ull;
    }
}

// ---------------------------------------------------------------------------
// Procrustes step, one GPU lane per subject, FP64.
// M = H S G S H^T (= A_k^T A_k), M = Z diag(d) Z^T, f_i = d_i^{-1/2} for
// d_i > rtol2 * max(d) else 0, T_k = Z diag(f) Z^T H S  (stored FP32).
// Per-thread matrices live in interleaved shared memory.
// ---------------------------------------------------------------------------
// FP64 flops of the Procrustes kernel for one subject (fused multiply-add =
// 2; sqrt and division = 1), counted from the operations it performs: the
// fixed part below plus 11 per QR step and 29 + 6R per Givens rotation.
static __host__ __device__ unsigned long long polar_fixed_flops(int R) {
    unsigned long long f = 0;
    const unsigned long long r = (unsigned long long)R, P = r * (r + 1) / 2;
    f += 2 * P;                                     // S G S
    f += 2 * r * r * r + r * r * (r + 1);           // M = H (S G S) H^T, lower triangle
    for (unsigned long long m = 2; m + 1 <= r; ++m) {
        f += 4 * m * m + 10 * m + 10;               // Householder step on an m-vector
        f += m * (4 * m - 2);                       // backward accumulation of that step
    }
    f += 3 * r;                                     // QR scale estimate
    f += 3 * r + 1;                                 // eigenvalue cut and d^-1/2
    f += 4 * r * r * r + 2 * r * r;                 // T = Z diag(f) Z^T H S
    return f;
}

__global__ void __launch_bounds__(128) k_polar(const double *__restrict__ G,
                                               const float *__restrict__ W,
                                               SmallState *st, float *T,
                                               int64_t K, int R, double rtol2) {
    extern __shared__ __align__(16) double sm[];
    const int NT = blockDim.x;
    const int t = threadIdx.x;
    const int P = R * (R + 1) / 2;
    double *Hs = sm;                       // R*R, H64
    double *th = sm + R * R;
    for (int i = t; i < R * R; i += NT) Hs[i] = st->H64[i];
    __syncthreads();
    const int64_t k = (int64_t)blockIdx.x * NT + t;
    unsigned long long flops = 0;
    if (k < K) {
        MatView A{th + t, NT, R};
        double *gp = th + (size_t)R * R * NT + t;          // packed scaled Gram, stride NT
        VecView d{gp + (size_t)P * NT, NT};
        VecView e{gp + (size_t)(P + R) * NT, NT};
        VecView bt{gp + (size_t)(P + 2 * R) * NT, NT};
        VecView tv{gp + (size_t)(P + 3 * R) * NT, NT};
        VecView w{gp + (size_t)(P + 4 * R) * NT, NT};

        const float *Wk = W + (size_t)k * R;
        for (int i = 0; i < R; ++i) w[i] = (double)Wk[i];
        const double *Gk = G + (size_t)k * P;
        for (int i = 0, p = 0; i < R; ++i)
            for (int j = 0; j <= i; ++j, ++p) gp[(size_t)p * NT] = Gk[p] * w[i] * w[j];
        // M = H Gs H^T, lower triangle, column by column
        for (int c = 0; c < R; ++c) {
            for (int i = 0; i < R; ++i) {
                double s = 0.0;
                for (int j = 0; j < R; ++j) {
                    const int p = (j <= i) ? (i * (i + 1) / 2 + j) : (j * (j + 1) / 2 + i);
                    s = fma(gp[(size_t)p * NT], Hs[c * R + j], s);
                }
                tv[i] = s;
            }
            for (int r = c; r < R; ++r) {
                double s = 0.0;
                for (int i = 0; i < R; ++i) s = fma(Hs[r * R + i], tv[i], s);
                A(r, c) = s;
            }
        }
        tridiagonalize(R, A, d, e, bt, tv);
        int rot = 0;
        const int steps = tridiagonal_qr(R, A, d, e, 30 * R, &rot);
        if (steps < 0) atomicOr(&st->flags, FLAG_EIG_NOCONV);
        double lmax = 0.0;
        for (int i = 0; i < R; ++i) lmax = fmax(lmax, d[i]);
        const double cut = rtol2 * lmax;
        for (int i = 0; i < R; ++i) d[i] = (lmax > 0.0 && d[i] > cut) ? 1.0 / sqrt(d[i]) : 0.0;
        float *Tk = T + (size_t)k * R * R;
        for (int c = 0; c < R; ++c) {
            const double wc = w[c];
            for (int i = 0; i < R; ++i) {
                double s = 0.0;
                for (int u = 0; u < R; ++u) s = fma(A(u, i), Hs[u * R + c], s);
                tv[i] = s * d[i] * wc;
            }
            for (int r = 0; r < R; ++r) {
                double s = 0.0;
                for (int i = 0; i < R; ++i) s = fma(A(r, i), tv[i], s);
                Tk[r * R + c] = (float)s;
            }
        }
        flops = polar_fixed_flops(R) + 11ull * (unsigned long long)(steps > 0 ? steps : 0) +
                (29ull + 6ull * R) * (unsigned long long)rot;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) flops += __shfl_down_sync(FULLMASK, flops, o);
    if ((t & 31) == 0 && flops) atomicAdd(&st->polar_flops, flops);
}

// ---------------------------------------------------------------------------
// Mode 1: partials of M1 = sum_k (T_k G_k) * 1 W(k,:), one block per fixed
// contiguous subject range; FP32 products, FP64 accumulation.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_mode1(const float *__restrict__ T,
                                               const double *__restrict__ G,
                                               const float *__restrict__ W, double *part,
                                               int64_t K, int R) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int P = R * (R + 1) / 2;
    float *Ts = reinterpret_cast<float *>(smem_raw);
    float *Gs = Ts + R * R;   // full R x R in FP32
    float *ws = Gs + R * R;
    const int64_t per = (K + gridDim.x - 1) / gridDim.x;
    const int64_t k0 = (int64_t)blockIdx.x * per;
    const int64_t k1 = (k0 + per < K) ? (k0 + per) : K;
    double acc[16];
#pragma unroll
    for (int q = 0; q < 16; ++q) acc[q] = 0.0;
    for (int64_t k = k0; k < k1; ++k) {
        const float *Tg = T + (size_t)k * R * R;
        const double *Gg = G + (size_t)k * P;
        for (int e = threadIdx.x; e < R * R; e += blockDim.x) Ts[e] = Tg[e];
        for (int p = threadIdx.x; p < P; p += blockDim.x) {
            int r = (int)((sqrt(8.0 * p + 1.0) - 1.0) * 0.5);
            while ((r + 1) * (r + 2) / 2 <= p) ++r;
            while (r * (r + 1) / 2 > p) --r;
            const int s = p - r * (r + 1) / 2;
            const float g = (float)Gg[p];
            Gs[r * R + s] = g;
            Gs[s * R + r] = g;
        }
        for (int s = threadIdx.x; s < R; s += blockDim.x) ws[s] = W[(size_t)k * R + s];
        __syncthreads();
#pragma unroll
        for (int q = 0; q < 16; ++q) {
            const int e = threadIdx.x + q * blockDim.x;
            if (e < R * R) {
                const int r = e / R, c = e - r * R;
                float s = 0.f;
                for (int u = 0; u < R; ++u) s = fmaf(Ts[r * R + u], Gs[u * R + c], s);
                acc[q] += (double)(s * ws[c]);
            }
        }
        __syncthreads();
    }
#pragma unroll
    for (int q = 0; q < 16; ++q) {
        const int e = threadIdx.x + q * blockDim.x;
        if (e < R * R) part[(size_t)blockIdx.x * R * R + e] = acc[q];
    }
}

// ---------------------------------------------------------------------------
// Partials of W^TW, <W, M3> and max |W(:, s)| over fixed subject ranges.
// part layout per block: [R*R WtW][R wmax][1 wm3]
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_gram_w(const float *__restrict__ W,
                                                const float *__restrict__ M3, double *part,
                                                int64_t K, int R, int with_m3) {
    const int64_t per = (K + gridDim.x - 1) / gridDim.x;
    const int64_t k0 = (int64_t)blockIdx.x * per;
    const int64_t k1 = (k0 + per < K) ? (k0 + per) : K;
    const size_t stride = (size_t)R * R + R + 1;
    double *out = part + (size_t)blockIdx.x * stride;
    double acc[16];
#pragma unroll
    for (int q = 0; q < 16; ++q) acc[q] = 0.0;
    double wm3 = 0.0;
    float wmx = 0.f;
    for (int64_t k = k0; k < k1; ++k) {
        const float *wk = W + (size_t)k * R;
#pragma unroll
        for (int q = 0; q < 16; ++q) {
            const int e = threadIdx.x + q * blockDim.x;
            if (e < R * R) {
                const int r = e / R, s = e - r * R;
                acc[q] = fma((double)wk[r], (double)wk[s], acc[q]);
            }
        }
        if (threadIdx.x < R) {
            const float v = wk[threadIdx.x];
            wmx = fmaxf(wmx, fabsf(v));
            if (with_m3) wm3 = fma((double)v, (double)M3[(size_t)k * R + threadIdx.x], wm3);
        }
    }
#pragma unroll
    for (int q = 0; q < 16; ++q) {
        const int e = threadIdx.x + q * blockDim.x;
        if (e < R * R) out[e] = acc[q];
    }
    __shared__ double sw[P2_RMAX];
    if (threadIdx.x < R) {
        out[R * R + threadIdx.x] = (double)wmx;
        sw[threadIdx.x] = wm3;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int i = 0; i < R; ++i) s += sw[i];
        out[R * R + R] = s;
    }
}

// Partials of V^T V (V stored FP32, products exact in FP64) over row ranges.
__global__ void __launch_bounds__(256) k_gram_v(const float *__restrict__ V, double *part,
                                                int64_t J, int R) {
    const int64_t per = (J + gridDim.x - 1) / gridDim.x;
    const int64_t j0 = (int64_t)blockIdx.x * per;
    const int64_t j1 = (j0 + per < J) ? (j0 + per) : J;
    double acc[16];
#pragma unroll
    for (int q = 0; q < 16; ++q) acc[q] = 0.0;
    for (int64_t j = j0; j < j1; ++j) {
        const float *vj = V + (size_t)j * R;
#pragma unroll
        for (int q = 0; q < 16; ++q) {
            const int e = threadIdx.x + q * blockDim.x;
            if (e < R * R) {
                const int r = e / R, s = e - r * R;
                acc[q] = fma((double)vj[r], (double)vj[s], acc[q]);
            }
        }
    }
#pragma unroll
    for (int q = 0; q < 16; ++q) {
        const int e = threadIdx.x + q * blockDim.x;
        if (e < R * R) part[(size_t)blockIdx.x * R * R + e] = acc[q];
    }
}

// ---------------------------------------------------------------------------
// Small FP64 linear algebra on one CTA.
// ---------------------------------------------------------------------------

// Symmetric eigen-decomposition of A (n x n, shared memory, row stride n) by
// parallel cyclic Jacobi (round-robin pairing, n/2 disjoint rotations per
// round, element-parallel updates).  On return diag(A) holds the eigenvalues
// and U the eigenvectors (columns).
static __device__ void cta_jacobi(double *A, double *U, int n, int *flags) {
    __shared__ double cs_c[P2_RMAX / 2], cs_s[P2_RMAX / 2];
    __shared__ int cs_p[P2_RMAX / 2], cs_q[P2_RMAX / 2];
    __shared__ int rotated;
    const int tid = threadIdx.x, nt = blockDim.x;
    const double eps = 2.220446049250313e-16;
    for (int e = tid; e < n * n; e += nt) U[e] = (e / n == e % n) ? 1.0 : 0.0;
    const int m = n + (n & 1);
    const int half = m / 2;
    __syncthreads();
    if (n <= 1) return;
    int sweep;
    for (sweep = 0; sweep < 60; ++sweep) {
        if (tid == 0) rotated = 0;
        __syncthreads();
        for (int round = 0; round < m - 1; ++round) {
            if (tid < half) {
                auto pos = [&](int ps) { return ps == 0 ? 0 : ((ps - 1 + round) % (m - 1)) + 1; };
                int p = pos(tid), q = pos(m - 1 - tid);
                if (p > q) { int tmp = p; p = q; q = tmp; }
                double c = 1.0, s = 0.0;
                if (q < n) {
                    const double apq = A[p * n + q];
                    const double app = A[p * n + p], aqq = A[q * n + q];
                    if (fabs(apq) > eps * sqrt(fabs(app * aqq)) && fabs(apq) > 1e-300) {
                        const double tau = (aqq - app) / (2.0 * apq);
                        const double tt = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
                        c = 1.0 / sqrt(1.0 + tt * tt);
                        s = tt * c;
                        rotated = 1;
                    }
                }
                cs_c[tid] = c;
                cs_s[tid] = s;
                cs_p[tid] = p;
                cs_q[tid] = (q < n) ? q : -1;
            }
            __syncthreads();
            // columns of A and U
            for (int e = tid; e < n * half; e += nt) {
                const int i = e / half, kk = e - i * half;
                const int q = cs_q[kk];
                if (q < 0 || cs_s[kk] == 0.0) continue;
                const int p = cs_p[kk];
                const double c = cs_c[kk], s = cs_s[kk];
                double x = A[i * n + p], y = A[i * n + q];
                A[i * n + p] = c * x - s * y;
                A[i * n + q] = s * x + c * y;
                x = U[i * n + p];
                y = U[i * n + q];
                U[i * n + p] = c * x - s * y;
                U[i * n + q] = s * x + c * y;
            }
            __syncthreads();
            for (int e = tid; e < n * half; e += nt) {
                const int j = e / half, kk = e - j * half;
                const int q = cs_q[kk];
                if (q < 0 || cs_s[kk] == 0.0) continue;
                const int p = cs_p[kk];
                const double c = cs_c[kk], s = cs_s[kk];
                const double x = A[p * n + j], y = A[q * n + j];
                A[p * n + j] = c * x - s * y;
                A[q * n + j] = s * x + c * y;
            }
            __syncthreads();
        }
        const int any = rotated;
        __syncthreads();
        if (!any) break;
    }
    if (sweep == 60 && tid == 0) atomicOr(flags, FLAG_EIG_NOCONV);
    __syncthreads();
}

// out = A^+ for the symmetric PSD n x n matrix in A (destroyed); U is n x n
// scratch.  Eigenvalues <= n * 2^-52 * lambda_max are dropped.
static __device__ void cta_pinv(double *A, double *U, double *out, int n, int *flags) {
    __shared__ double f[P2_RMAX];
    cta_jacobi(A, U, n, flags);
    if (threadIdx.x == 0) {
        double lmax = 0.0;
        for (int i = 0; i < n; ++i) lmax = fmax(lmax, A[i * n + i]);
        const double cut = (double)n * 2.220446049250313e-16 * lmax;
        for (int i = 0; i < n; ++i) {
            const double l = A[i * n + i];
            f[i] = (lmax > 0.0 && l > cut) ? 1.0 / l : 0.0;
        }
    }
    __syncthreads();
    for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
        const int i = e / n, j = e - i * n;
        double s = 0.0;
        for (int l = 0; l < n; ++l) s = fma(U[i * n + l] * f[l], U[j * n + l], s);
        out[e] = s;
    }
    __syncthreads();
}

// H solve: M1 = sum of partials; H = normalize(M1 (W^TW * V^TV)^+); H64, HtH.
__global__ void __launch_bounds__(256) k_solve_h(const double *__restrict__ part, int nparts,
                                                 SmallState *st, float *H, int R) {
    extern __shared__ __align__(16) double sd[];
    double *A = sd, *U = A + R * R, *Pi = U + R * R, *Hn = Pi + R * R;
    __shared__ double nrm[P2_RMAX];
    for (int e = threadIdx.x; e < R * R; e += blockDim.x) {
        double s = 0.0;
        for (int b = 0; b < nparts; ++b) s += part[(size_t)b * R * R + e];
        st->M1[e] = s;
        A[e] = st->WtW[e] * st->VtV[e];
    }
    __syncthreads();
    cta_pinv(A, U, Pi, R, &st->flags);
    for (int e = threadIdx.x; e < R * R; e += blockDim.x) {
        const int i = e / R, j = e - i * R;
        double s = 0.0;
        for (int l = 0; l < R; ++l) s = fma(st->M1[i * R + l], Pi[l * R + j], s);
        Hn[e] = s;
    }
    __syncthreads();
    for (int j = threadIdx.x; j < R; j += blockDim.x) {
        double s = 0.0;
        for (int i = 0; i < R; ++i) s = fma(Hn[i * R + j], Hn[i * R + j], s);
        nrm[j] = sqrt(s);
    }
    __syncthreads();
    for (int e = threadIdx.x; e < R * R; e += blockDim.x) {
        const int j = e % R;
        const float h = nrm[j] > 0.0 ? (float)(Hn[e] / nrm[j]) : 0.f;
        H[e] = h;
        st->H64[e] = (double)h;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < R * R; e += blockDim.x) {
        const int i = e / R, j = e - i * R;
        double s = 0.0;
        for (int l = 0; l < R; ++l) s = fma(st->H64[l * R + i], st->H64[l * R + j], s);
        st->HtH[e] = s;
    }
}

// HtH (and H64) for a freshly set H.
__global__ void k_init_h(const float *__restrict__ H, SmallState *st, int R) {
    for (int e = threadIdx.x; e < R * R; e += blockDim.x) st->H64[e] = (double)H[e];
    __syncthreads();
    for (int e = threadIdx.x; e < R * R; e += blockDim.x) {
        const int i = e / R, j = e - i * R;
        double s = 0.0;
        for (int l = 0; l < R; ++l) s = fma(st->H64[l * R + i], st->H64[l * R + j], s);
        st->HtH[e] = s;
    }
}

// V solve, part a: (W^TW * H^TH)^+.
__global__ void __launch_bounds__(256) k_solve_v_pinv(SmallState *st, int R) {
    extern __shared__ __align__(16) double sd[];
    double *A = sd, *U = A + R * R;
    for (int e = threadIdx.x; e < R * R; e += blockDim.x) A[e] = st->WtW[e] * st->HtH[e];
    __syncthreads();
    cta_pinv(A, U, st->P2inv, R, &st->flags);
}

// V solve, part b: Vun = M2 P2inv; partial column sums of squares per block.
__global__ void __launch_bounds__(256) k_solve_v_rows(const double *__restrict__ M2,
                                                      const SmallState *__restrict__ st,
                                                      double *Vun, double *part, int64_t J,
                                                      int R) {
    extern __shared__ __align__(16) double sd[];
    double *Pi = sd;            // R*R
    double *red = Pi + R * R;   // blockDim
    for (int e = threadIdx.x; e < R * R; e += blockDim.x) Pi[e] = st->P2inv[e];
    __syncthreads();
    const int64_t per = (J + gridDim.x - 1) / gridDim.x;
    const int64_t j0 = (int64_t)blockIdx.x * per;
    const int64_t j1 = (j0 + per < J) ? (j0 + per) : J;
    const int rows_per = blockDim.x / R;
    const int rr = threadIdx.x / R, s = threadIdx.x - rr * R;
    double cs = 0.0;
    if (rr < rows_per) {
        for (int64_t j = j0 + rr; j < j1; j += rows_per) {
            double v = 0.0;
            for (int u = 0; u < R; ++u) v = fma(M2[(size_t)j * R + u], Pi[u * R + s], v);
            Vun[(size_t)j * R + s] = v;
            cs = fma(v, v, cs);
        }
    }
    red[threadIdx.x] = (rr < rows_per) ? cs : 0.0;
    __syncthreads();
    if (threadIdx.x < R) {
        double t = 0.0;
        for (int q = threadIdx.x; q < rows_per * R; q += R) t += red[q];
        part[(size_t)blockIdx.x * R + threadIdx.x] = t;
    }
}

// V solve, part c: column norms from the partials.
__global__ void k_solve_v_norm(const double *__restrict__ part, int nparts, SmallState *st,
                               int R) {
    for (int s = threadIdx.x; s < R; s += blockDim.x) {
        double t = 0.0;
        for (int b = 0; b < nparts; ++b) t += part[(size_t)b * R + s];
        st->colnorm[s] = sqrt(t);
    }
}

// V solve, part d: Vprev <- V; V <- Vun / colnorm (FP32).
__global__ void k_solve_v_store(const double *__restrict__ Vun, const SmallState *st, float *V,
                                float *Vprev, int64_t n, int R) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int s = (int)(e % R);
        const double nr = st->colnorm[s];
        Vprev[e] = V[e];
        V[e] = nr > 0.0 ? (float)(Vun[e] / nr) : 0.f;
    }
}

// Sum V^TV partials; G3inv = (V^TV * H^TH)^+.
__global__ void __launch_bounds__(256) k_fin_v(const double *__restrict__ part, int nparts,
                                               SmallState *st, int R, int with_g3) {
    extern __shared__ __align__(16) double sd[];
    double *A = sd, *U = A + R * R;
    for (int e = threadIdx.x; e < R * R; e += blockDim.x) {
        double s = 0.0;
        for (int b = 0; b < nparts; ++b) s += part[(size_t)b * R * R + e];
        st->VtV[e] = s;
        A[e] = s * st->HtH[e];
    }
    __syncthreads();
    if (with_g3) cta_pinv(A, U, st->G3inv, R, &st->flags);
}

// Sum the W partials; loss / fit; fixed-point scales for the next mode-2 pass.
__global__ void k_fin_w(const double *__restrict__ part, int nparts, SmallState *st, int R,
                        int with_fit) {
    const size_t stride = (size_t)R * R + R + 1;
    __shared__ double red[256];
    double lsum = 0.0;
    for (int e = threadIdx.x; e < R * R; e += blockDim.x) {
        double s = 0.0;
        for (int b = 0; b < nparts; ++b) s += part[(size_t)b * stride + e];
        st->WtW[e] = s;
        lsum += s * st->HtH[e] * st->VtV[e];
    }
    red[threadIdx.x] = lsum;
    for (int s = threadIdx.x; s < R; s += blockDim.x) {
        double mx = 0.0;
        for (int b = 0; b < nparts; ++b) mx = fmax(mx, part[(size_t)b * stride + R * R + s]);
        st->wmax[s] = mx;
        // |term| <= xbound * wmax: choose 2^E with xbound * wmax * 2^E < 2^61
        const double bound = st->xbound * mx;
        int E = 0;
        if (bound > 0.0) {
            int ex;
            frexp(bound, &ex);          // bound < 2^ex
            E = 61 - ex;
            if (E > 120) E = 120;
            if (E < -120) E = -120;
        }
        st->m2scale[s] = ldexpf(1.0f, E);
        st->m2inv[s] = ldexp(1.0, -E);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int i = 0; i < (int)blockDim.x; ++i) t += red[i];
        if (with_fit) {
            double wm3 = 0.0;
            for (int b = 0; b < nparts; ++b) wm3 += part[(size_t)b * stride + R * R + R];
            st->wm3 = wm3;
            const double loss = st->normx2 - 2.0 * wm3 + t;
            st->loss = loss;
            st->fit = 1.0 - sqrt(fmax(loss, 0.0)) / sqrt(st->normx2);
            if (!isfinite(loss)) atomicOr(&st->flags, FLAG_NONFINITE);
            st->iter += 1;
        }
    }
}

// ---------------------------------------------------------------------------
// host-side enqueue
// ---------------------------------------------------------------------------
static size_t alpha_cta_bytes(int R) {
    const int P = R * (R + 1) / 2;
    return ((size_t)R * R * 8 + (size_t)R * R * 4 + 2 * (size_t)P + 15) & ~(size_t)15;
}
static size_t alpha_warp_bytes(int R) {
    const int P = R * (R + 1) / 2;
    return (size_t)P * 8 + ((size_t)64 * R + 2 * (size_t)R * R) * 4;
}
static size_t beta_warp_bytes(int R) { return ((size_t)64 * R + 2 * (size_t)R * R + R) * 4; }

struct Launch {
    int alpha_warps, beta_warps, beta_hc, polar_nt;
    size_t alpha_smem, beta_smem, polar_smem;
};

static Launch plan(const p2_ctx *c) {
    Launch L{};
    const int R = c->R;
    const size_t cap = (size_t)c->geo.smem_optin;
    int aw = 16;
    while (aw > 1 && alpha_cta_bytes(R) + aw * alpha_warp_bytes(R) > cap) --aw;
    L.alpha_warps = aw;
    L.alpha_smem = alpha_cta_bytes(R) + aw * alpha_warp_bytes(R);
    int bw = R <= 16 ? 8 : 4;
    L.beta_warps = bw;
    size_t fixed = (size_t)R * R * 4 + (size_t)R * 4 + 16 + bw * beta_warp_bytes(R);
    int hc = (int)((cap - fixed) / (8 * (size_t)R));
    if (hc > c->X.J) hc = c->X.J;
    if (hc < 0) hc = 0;
    L.beta_hc = hc;
    L.beta_smem = (((size_t)hc * R * 8 + (size_t)R * R * 4 + (size_t)R * 4 + 15) & ~(size_t)15) +
                  bw * beta_warp_bytes(R);
    const int P = R * (R + 1) / 2;
    const size_t per_thread = ((size_t)R * R + P + 5 * (size_t)R) * 8;
    const size_t avail = cap - (size_t)R * R * 8;
    int nt = (int)(avail / per_thread);
    if (nt > 128) nt = 128;
    if (nt >= 32) nt = (nt / 32) * 32;
    if (nt < 1) nt = 1;
    L.polar_nt = nt;
    L.polar_smem = (size_t)R * R * 8 + (size_t)nt * per_thread;
    return L;
}

template <class F>
static int allow_dynamic_smem(F *fn, int cap, const char *name) {
    cudaFuncAttributes fa;
    cudaError_t e = cudaFuncGetAttributes(&fa, fn);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 cap - (int)fa.sharedSizeBytes);
    if (e != cudaSuccess) {
        set_error("configuring %s: %s", name, cudaGetErrorString(e));
        return P2_ECUDA;
    }
    return P2_OK;
}

int configure_kernels(p2_ctx *c) {
    const int cap = c->geo.smem_optin;
    int rc = P2_OK;
    if (rc == P2_OK) rc = allow_dynamic_smem(k_alpha<true>, cap, "k_alpha<true>");
    if (rc == P2_OK) rc = allow_dynamic_smem(k_alpha<false>, cap, "k_alpha<false>");
    if (rc == P2_OK) rc = allow_dynamic_smem(k_beta, cap, "k_beta");
    if (rc == P2_OK) rc = allow_dynamic_smem(k_polar, cap, "k_polar");
    if (rc == P2_OK) rc = allow_dynamic_smem(k_solve_h, cap, "k_solve_h");
    if (rc == P2_OK) rc = allow_dynamic_smem(k_solve_v_pinv, cap, "k_solve_v_pinv");
    if (rc == P2_OK) rc = allow_dynamic_smem(k_fin_v, cap, "k_fin_v");
    return rc;
}

static int check_launch(const char *what) {
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        set_error("launch of %s failed: %s", what, cudaGetErrorString(e));
        return P2_ECUDA;
    }
    return P2_OK;
}

#define P2_LAUNCH_CHECK(name)                         \
    do {                                              \
        int _rc = check_launch(name);                 \
        if (_rc != P2_OK) return _rc;                 \
        c->enqueued += 1;                             \
    } while (0)

// Phase boundary event; recorded as an event-record node when the stream is
// being captured into the iteration graph.
static void mark(p2_ctx *c, int i) {
    if (c->opt.timing) cudaEventRecordWithFlags(c->ev[i], c->stream, cudaEventRecordExternal);
}

static int enqueue_qstep(p2_ctx *c, const Launch &L) {
    const int R = c->R;
    cudaStream_t s = c->stream;
    const int nb = c->geo.red_blocks;
    double rtol2 = c->opt.rank_rtol * c->opt.rank_rtol;
    const int64_t K = c->X.K;
    if (K > 0) {
        const int nblk = (int)((K + L.polar_nt - 1) / L.polar_nt);
        k_polar<<<nblk, L.polar_nt, L.polar_smem, s>>>(c->d_G, c->d_W, c->d_s, c->d_T, K, R,
                                                       rtol2);
        P2_LAUNCH_CHECK("k_polar");
    }
    mark(c, 6);
    const size_t m1_smem = ((size_t)2 * R * R + R) * 4;
    k_mode1<<<nb, 256, m1_smem, s>>>(c->d_T, c->d_G, c->d_W, c->d_part, K, R);
    P2_LAUNCH_CHECK("k_mode1");
    return P2_OK;
}

int enqueue_factor_stats(p2_ctx *c) {
    const int R = c->R;
    cudaStream_t s = c->stream;
    const int nb = c->geo.red_blocks;
    k_init_h<<<1, 256, 0, s>>>(c->d_H, c->d_s, R);
    P2_LAUNCH_CHECK("k_init_h");
    k_gram_v<<<nb, 256, 0, s>>>(c->d_V, c->d_part2, c->X.J, R);
    P2_LAUNCH_CHECK("k_gram_v");
    k_fin_v<<<1, 256, (size_t)2 * R * R * 8, s>>>(c->d_part2, nb, c->d_s, R, 0);
    P2_LAUNCH_CHECK("k_fin_v");
    k_gram_w<<<nb, 256, 0, s>>>(c->d_W, c->d_M3, c->d_part2, c->X.K, R, 0);
    P2_LAUNCH_CHECK("k_gram_w");
    k_fin_w<<<1, 256, 0, s>>>(c->d_part2, nb, c->d_s, R, 0);
    P2_LAUNCH_CHECK("k_fin_w");
    return P2_OK;
}

int enqueue_prologue(p2_ctx *c) {
    const Launch L = plan(c);
    const int R = c->R;
    cudaStream_t s = c->stream;
    const int nsm = c->geo.nsm;
    XView X = xview(c);
    k_alpha<false><<<nsm, L.alpha_warps * 32, L.alpha_smem, s>>>(
        X, nullptr, c->d_V, c->d_H, c->d_T, c->d_s, c->d_G, c->d_W, c->d_M3, R);
    P2_LAUNCH_CHECK("k_alpha<false>");
    return enqueue_qstep(c, L);
}

int enqueue_iteration(p2_ctx *c) {
    const Launch L = plan(c);
    const int R = c->R;
    cudaStream_t s = c->stream;
    const int nsm = c->geo.nsm;
    const int nb = c->geo.red_blocks;
    const int64_t J = c->X.J, K = c->X.K;
    XView X = xview(c);
    const size_t sm_pinv = (size_t)4 * R * R * 8;
    // H step (Algorithm 1 line 3 with U = H; mode-1 MTTKRP from the previous pass)
    mark(c, 0);
    k_solve_h<<<1, 256, sm_pinv, s>>>(c->d_part, nb, c->d_s, c->d_H, R);
    P2_LAUNCH_CHECK("k_solve_h");
    // pass beta: mode-2 MTTKRP
    mark(c, 1);
    k_beta<<<nsm, L.beta_warps * 32, L.beta_smem, s>>>(X, c->d_V, c->d_H, c->d_T, c->d_W, c->d_s,
                                                       c->d_m2acc, R, L.beta_hc);
    P2_LAUNCH_CHECK("k_beta");
    const int64_t nJR = J * R;
    const int fb = (int)((nJR + 255) / 256 < 4 * nsm ? (nJR + 255) / 256 : 4 * nsm);
    k_m2_finalize<<<fb, 256, 0, s>>>(c->d_m2acc, c->d_M2, c->d_s, nJR, R);
    P2_LAUNCH_CHECK("k_m2_finalize");
    // V step (Algorithm 1 line 5)
    mark(c, 2);
    k_solve_v_pinv<<<1, 256, sm_pinv, s>>>(c->d_s, R);
    P2_LAUNCH_CHECK("k_solve_v_pinv");
    k_solve_v_rows<<<nb, 256, ((size_t)R * R + 256) * 8, s>>>(c->d_M2, c->d_s, c->d_Vun,
                                                               c->d_part2, J, R);
    P2_LAUNCH_CHECK("k_solve_v_rows");
    k_solve_v_norm<<<1, 64, 0, s>>>(c->d_part2, nb, c->d_s, R);
    P2_LAUNCH_CHECK("k_solve_v_norm");
    k_solve_v_store<<<fb, 256, 0, s>>>(c->d_Vun, c->d_s, c->d_V, c->d_Vprev, nJR, R);
    P2_LAUNCH_CHECK("k_solve_v_store");
    k_gram_v<<<nb, 256, 0, s>>>(c->d_V, c->d_part2, J, R);
    P2_LAUNCH_CHECK("k_gram_v");
    k_fin_v<<<1, 256, sm_pinv, s>>>(c->d_part2, nb, c->d_s, R, 1);
    P2_LAUNCH_CHECK("k_fin_v");
    // pass alpha: mode-3 MTTKRP + W step (Algorithm 1 line 7) + Gram for the next Q-step
    mark(c, 3);
    k_alpha<true><<<nsm, L.alpha_warps * 32, L.alpha_smem, s>>>(
        X, c->d_Vprev, c->d_V, c->d_H, c->d_T, c->d_s, c->d_G, c->d_W, c->d_M3, R);
    P2_LAUNCH_CHECK("k_alpha<true>");
    mark(c, 4);
    k_gram_w<<<nb, 256, 0, s>>>(c->d_W, c->d_M3, c->d_part2, K, R, 1);
    P2_LAUNCH_CHECK("k_gram_w");
    k_fin_w<<<1, 256, 0, s>>>(c->d_part2, nb, c->d_s, R, 1);
    P2_LAUNCH_CHECK("k_fin_w");
    // next Q-step (Algorithm 2's SVD loop) and its mode-1 MTTKRP
    mark(c, 5);
    int rc = enqueue_qstep(c, L);
    mark(c, 7);
    return rc;
}

}  // namespace p2
