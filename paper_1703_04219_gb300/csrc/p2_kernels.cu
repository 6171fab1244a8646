// Kernels of one PARAFAC2-ALS iteration in SPARTan's formulation.
//
// Notation (Perros et al., KDD 2017, Sections 3-4): X_k is I_k x J sparse,
// H is R x R, V is J x R, W is K x R and S_k = diag(W(k,:)).
//
// The schedule works on per-subject R x R state instead of materialising
// Q_k or Y_k (identities that follow from the paper's definitions):
//   Z_k = X_k V                       (never stored; recomputed per pass)
//   A_k = Z_k S_k H^T                 (Procrustes input: H S_k V^T X_k^T = A_k^T)
//   G_k = Z_k^T Z_k                   (error-free FP32 pairs: FP64-accurate)
//   C_k = (A_k^T A_k)^{+1/2}, Q_k = A_k C_k   (polar factor, FP64)
//   T_k = C_k H S_k, so Q_k = Z_k T_k^T and Y_k = Q_k^T X_k = T_k Z_k^T X_k
//   mode 1 (Eq. mttkrp1_3):  Y_k V = T_k G_k
//   mode 2 (Eq. mttkrp2_3):  Y_k^T H S_k = X_k^T (Z_k F_k), F_k = T_k^T H S_k
//   mode 3 (Eq. mttkrp3_row_wise): Y_k V' = T_k Z_k^T Z'_k, Z'_k = X_k V'
// so an iteration streams X twice: pass beta (mode 2) and pass alpha (mode
// 3, the W row, and the next Q-step's Gram), with the R x R work in between.
//
// Determinism: every reduction over subjects or non-zeros uses fixed
// per-block partials summed in a fixed order; there are no floating-point
// atomics (integer atomics only count columns at load time, raise error
// flags and count flops).
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <algorithm>
#include <utility>

#include "p2_internal.cuh"

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

static XView xview(const p2_ctx *c) {
    // subject bins pay above R = 16, where a subject's work is large enough
    // for the tail of the persistent grid to matter (R = 40: alpha pass -3%);
    // at R = 10 the natural order's sequential walk over X is worth more
    // (+1.5%); the tuning can override the rule
    const bool bins = c->tune.subject_bins < 0 ? c->R > 16 : c->tune.subject_bins != 0;
    return XView{c->X.subj_row, c->X.subj_nnz, c->X.row_len, c->X.col, c->X.val, c->X.K,
                 bins ? c->d_sorder : nullptr};
}

// The error-free transformations below hold only if every rounding happens
// exactly as written: a product that the compiler contracted with the
// following sum into one FMA (nvcc's default --fmad=true allows it) would
// leave TwoSum's error term wrong.  So every operation goes through the
// __f*_rn intrinsics of p2_dw.cuh (f_add, f_sub, f_mul, f_fma), which are
// never contracted or reassociated.
// a + b = s + e exactly (Knuth's TwoSum)
static __device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
    s = f_add(a, b);
    const float bv = f_sub(s, a);
    e = f_add(f_sub(a, f_sub(s, bv)), f_sub(b, bv));
}
// (hi, lo) += x: an unevaluated float pair, error-free up to the rounding of lo
static __device__ __forceinline__ void pair_add(float &hi, float &lo, float x) {
    float t, e;
    two_sum(hi, x, t, e);
    hi = t;
    lo = f_add(lo, e);
}
// (hi, lo) += a * b, the product split exactly with an FMA (Dekker's TwoProduct)
static __device__ __forceinline__ void pair_fma(float &hi, float &lo, float a, float b) {
    const float p = f_mul(a, b);
    const float pe = f_fma(a, b, -p);
    float t, e;
    two_sum(hi, p, t, e);
    hi = t;
    lo = f_add(lo, f_add(e, pe));
}

// z rows of up to 32 consecutive rows: z1[i][:] = X(row i, :) V1 and, when
// TWO, z2[i][:] = X(row i, :) V2.  One lane per row, so a chunk costs one
// round of dependent loads; the row's components are accumulated in
// registers in blocks of CB (FP32 FMA in column order within the row) and
// stored with the odd row stride RS (no shared-memory bank conflicts).  With
// TWO the row is walked once per operand so that only CB accumulators are
// live (register pressure decides the occupancy of the passes).
// a[0 .. CB) += x * V(j, cb .. cb + CB) from a 16-byte aligned, zero-padded
// row segment v, with 16-byte loads; lim = R - cb valid components.
template <int CB>
static __device__ __forceinline__ void axpy_row(float *a, float x, const float *__restrict__ v,
                                                int lim) {
    const float4 *v4 = reinterpret_cast<const float4 *>(v);
#pragma unroll
    for (int q = 0; q < CB / 4; ++q) {
        if (4 * q < lim) {
            const float4 t = __ldg(v4 + q);
            a[4 * q] = fmaf(x, t.x, a[4 * q]);
            a[4 * q + 1] = fmaf(x, t.y, a[4 * q + 1]);
            a[4 * q + 2] = fmaf(x, t.z, a[4 * q + 2]);
            a[4 * q + 3] = fmaf(x, t.w, a[4 * q + 3]);
        }
    }
}
template <int CB>
static __device__ __forceinline__ void axpy_row(float *a, float x, const bf16_t *__restrict__ v,
                                                int lim) {
    const uint4 *v8 = reinterpret_cast<const uint4 *>(v);
#pragma unroll
    for (int q = 0; q < CB / 8; ++q) {
        if (8 * q < lim) {
            const uint4 t = __ldg(v8 + q);
            const unsigned w[4] = {t.x, t.y, t.z, t.w};
#pragma unroll
            for (int h = 0; h < 4; ++h) {       // two bfloat16 per word, low half first
                a[8 * q + 2 * h] = fmaf(x, __int_as_float((int)(w[h] << 16)), a[8 * q + 2 * h]);
                a[8 * q + 2 * h + 1] =
                    fmaf(x, __int_as_float((int)(w[h] & 0xffff0000u)), a[8 * q + 2 * h + 1]);
            }
        }
    }
}

template <int CB, bool TWO, class S>
static __device__ __forceinline__ void gather_rows(const XView &X, int nr, int64_t base, int len,
                                                   int off, const S *__restrict__ V1,
                                                   const S *__restrict__ V2, float *z1,
                                                   float *z2, int R, int RS, int lane) {
    if (lane >= nr) return;
    const int64_t b0 = base + off;
    const int VS = v_stride<S>(R);
    if (TWO && CB >= 32 && R <= CB) {
        // the whole row in one block: one walk over the row's non-zeros feeds
        // both operands (one round of dependent column loads instead of two);
        // for CB >= 32 only, where the kernel may hold both accumulator rows
        // (one block per SM; at CB = 16 the registers of three blocks per SM
        // do not hold them)
        float a1[CB], a2[CB];
#pragma unroll
        for (int c = 0; c < CB; ++c) {
            a1[c] = 0.f;
            a2[c] = 0.f;
        }
        for (int e = 0; e < len; ++e) {
            const int j = X.col[b0 + e];
            const float x = X.val[b0 + e];
            axpy_row<CB>(a1, x, V1 + (size_t)j * VS, R);
            axpy_row<CB>(a2, x, V2 + (size_t)j * VS, R);
        }
#pragma unroll
        for (int c = 0; c < CB; ++c)
            if (c < R) {
                z1[lane * RS + c] = a1[c];
                z2[lane * RS + c] = a2[c];
            }
        return;
    }
#pragma unroll 1
    for (int which = 0; which < (TWO ? 2 : 1); ++which) {
        const S *__restrict__ Vw = which ? V2 : V1;
        float *zw = which ? z2 : z1;
        for (int cb = 0; cb < R; cb += CB) {
            float a[CB];
#pragma unroll
            for (int c = 0; c < CB; ++c) a[c] = 0.f;
            for (int e = 0; e < len; ++e) {
                const int j = X.col[b0 + e];
                const float x = X.val[b0 + e];
                axpy_row<CB>(a, x, Vw + (size_t)j * VS + cb, R - cb);
            }
#pragma unroll
            for (int c = 0; c < CB; ++c)
                if (cb + c < R) zw[lane * RS + cb + c] = a[c];
        }
    }
}

static __host__ __device__ __forceinline__ int row_stride(int R) { return R | 1; }

// Rows of small R x R operands read as 16-byte broadcasts are padded to a
// multiple of four floats.
static __host__ __device__ __forceinline__ int f_stride(int R) { return (R + 3) & ~3; }

// Per-warp shared memory of the alpha pass: C_k or B_k (R x f_stride),
// 64 z rows, T_k (R x R), the Gram pairs (2 P) and, for R <= 16 (mode 3 one
// lane per row), the lanes' mode-3 partial rows (32 x row_stride); a
// multiple of 16 bytes.
static __host__ __device__ __forceinline__ size_t alpha_warp_bytes_dev(int R) {
    const size_t P = (size_t)R * (R + 1) / 2;
    const size_t zrows = R <= 16 ? 96 : 64;
    const size_t b = ((size_t)R * f_stride(R) + zrows * row_stride(R) + (size_t)R * R) * 4 +
                     8 * P;
    return (b + 15) & ~(size_t)15;
}

// Row and column of entry e of an n-column row-major array, for e advancing by
// 32 (one warp's stride) without an integer division per step.
struct RowCol {
    int r, c;
    __device__ __forceinline__ RowCol(int e, int n) : r(e / n), c(e - (e / n) * n) {}
    __device__ __forceinline__ void next(int n) {
        c += 32;
        while (c >= n) {
            c -= n;
            ++r;
        }
    }
};

// ---------------------------------------------------------------------------
// Pass alpha: for each subject, Gram of Z'_k = X_k V (packed lower; every
// product z_r z_s is split exactly into p + e with an FMA (Dekker's
// TwoProduct) and summed into an unevaluated float pair with Knuth's TwoSum,
// so the Gram carries ~2^-48 relative error without using the FP64 pipe)
// and, with MODE3, the mode-3 MTTKRP row M3(k,:) = coldot(H, T_k Z_k^T Z'_k)
// with Z_k = X_k Vprev, followed by W(k,:) = M3(k,:) (V^TV * H^TH)^+.
// For R <= 16 the mode-3 row is taken row by row: with B_k = T_k^T H,
// M3(k,:) = sum_i z'_i o (B_k^T z_i), one lane per row, B_k read as 16-byte
// broadcasts; for larger R through C_k = Z_k^T Z'_k and coldot(H, T_k C_k).
// ---------------------------------------------------------------------------
template <int CB, bool MODE3, class S, int RT = 0>
__global__ void __launch_bounds__(256, CB >= 32 ? 1 : 3) k_alpha(XView X, const S *__restrict__ Vprev,
                                               const S *__restrict__ V,
                                               const float *__restrict__ H,
                                               const float *__restrict__ T,
                                               const SmallState *__restrict__ st, dw *G,
                                               float *Gf, float *W, float *M3, int R_rt) {
    // RT > 0: the rank fixed at compile time (loop bounds, strides and
    // shared-memory offsets become constants); RT = 0: the rank R_rt
    const int R = RT > 0 ? RT : R_rt;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int P = R * (R + 1) / 2;
    const int RS = row_stride(R);
    // CTA-shared: G3inv (R*R doubles), H (R*R floats), packed index table
    // G3inv = (V^TV * H^TH)^+ (FP64) as an unevaluated float pair hi + lo
    float *G3h = reinterpret_cast<float *>(smem_raw);
    float *G3l = G3h + R * R;
    float *Hs = G3l + R * R;
    uint8_t *pr = reinterpret_cast<uint8_t *>(Hs + R * R);
    uint8_t *pc = pr + P;
    size_t cta_bytes = ((size_t)R * R * 8 + (size_t)R * R * 4 + 2 * (size_t)P + 15) & ~(size_t)15;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int FS = f_stride(R);
    unsigned char *wb = smem_raw + cta_bytes + warp * alpha_warp_bytes_dev(R);
    float *Cacc = reinterpret_cast<float *>(wb);        // R FS: C_k (R R) or B_k rows (16-byte aligned)
    float *Bt = Cacc;
    float *zo = Cacc + R * FS;                          // 32 RS (zo and zn contiguous: 64 RS scratch)
    float *zn = zo + 32 * RS;                           // 32 RS
    float *Tk = zn + 32 * RS;                           // R R
    float *Ghi = Tk + R * R;                            // P
    float *Glo = Ghi + P;                               // P
    float *M3p = Glo + P;                               // 32 RS: each lane's mode-3 partial row
    constexpr bool ROWWISE = CB <= 16;                  // mode 3 one lane per row

    for (int i = threadIdx.x; i < R * R; i += blockDim.x) {
        const double g = st->G3inv[i];
        const float gh = (float)g;
        G3h[i] = gh;
        G3l[i] = (float)(g - (double)gh);
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
    for (int64_t ki = (int64_t)blockIdx.x * (blockDim.x >> 5) + warp; ki < X.K; ki += nwarps) {
        const int64_t k = X.order ? (int64_t)X.order[ki] : ki;
        const int64_t r0 = X.subj_row[k], r1 = X.subj_row[k + 1];
        int64_t base = X.subj_nnz[k];
        for (int p = lane; p < P; p += 32) {
            Ghi[p] = 0.f;
            Glo[p] = 0.f;
        }
        if (MODE3 && ROWWISE) {
            // B_k = T_k^T H into Bt (row u = column u of B_k^T ... rows padded to FS)
            const float *Tg = T + (size_t)k * R * R;
            for (int e = lane; e < R * R; e += 32) Tk[e] = Tg[e];
            __syncwarp();
            RowCol ur(lane, R);
            for (int e = lane; e < R * R; e += 32, ur.next(R)) {
                float b = 0.f;
                for (int s2 = 0; s2 < R; ++s2) b = fmaf(Tk[s2 * R + ur.r], Hs[s2 * R + ur.c], b);
                Bt[ur.r * FS + ur.c] = b;
            }
            for (int e = lane; e < R * (FS - R); e += 32) {
                const int u = e / (FS - R);
                Bt[u * FS + R + (e - u * (FS - R))] = 0.f;
            }
            for (int c = 0; c < R; ++c) M3p[lane * RS + c] = 0.f;
            __syncwarp();
        } else if (MODE3) {
            for (int e = lane; e < R * R; e += 32) Cacc[e] = 0.f;
        }
        for (int64_t cr = r0; cr < r1; cr += 32) {
            const int nr = (int)((r1 - cr) < 32 ? (r1 - cr) : 32);
            const int len = (lane < nr) ? (int)X.row_len[cr + lane] : 0;
            const int off = warp_excl_scan(len, lane);
            const int tot = __shfl_sync(FULLMASK, off + len, 31);
            if (MODE3)
                gather_rows<CB, true, S>(X, nr, base, len, off, Vprev, V, zo, zn, R, RS, lane);
            else
                gather_rows<CB, false, S>(X, nr, base, len, off, V, nullptr, zn, nullptr, R, RS,
                                          lane);
            __syncwarp();
            if (MODE3 && ROWWISE) {
                if (lane < nr) {                        // u = B_k^T z_i, m3 += z'_i o u
                    const float *zi = zo + lane * RS;
                    const float *zpi = zn + lane * RS;
                    float acc[ROWWISE ? CB : 1];
#pragma unroll
                    for (int c = 0; c < (ROWWISE ? CB : 1); ++c) acc[c] = 0.f;
                    for (int u = 0; u < R; ++u) {
                        const float zu = zi[u];
                        const float4 *b4 = reinterpret_cast<const float4 *>(Bt + u * FS);
#pragma unroll
                        for (int q = 0; q < (ROWWISE ? CB : 4) / 4; ++q) {
                            if (4 * q < R) {
                                const float4 b = b4[q];
                                acc[4 * q] = fmaf(zu, b.x, acc[4 * q]);
                                acc[4 * q + 1] = fmaf(zu, b.y, acc[4 * q + 1]);
                                acc[4 * q + 2] = fmaf(zu, b.z, acc[4 * q + 2]);
                                acc[4 * q + 3] = fmaf(zu, b.w, acc[4 * q + 3]);
                            }
                        }
                    }
                    float *m3r = M3p + lane * RS;
#pragma unroll
                    for (int c = 0; c < (ROWWISE ? CB : 1); ++c)
                        if (c < R) m3r[c] = fmaf(zpi[c], acc[c], m3r[c]);
                }
            } else if (MODE3) {
                RowCol rs(lane, R);
                for (int e = lane; e < R * R; e += 32, rs.next(R)) {
                    float acc = 0.f;
#pragma unroll 4
                    for (int i = 0; i < nr; ++i) acc = fmaf(zo[i * RS + rs.r], zn[i * RS + rs.c], acc);
                    Cacc[e] += acc;
                }
            }
            // a lane's two packed entries p and p + 32 accumulated together (two
            // independent chains; a lane without a second entry repeats the
            // first and discards it), each with its own terms in row order
            for (int p = lane; p < P; p += 64) {
                const bool two = p + 32 < P;
                const int q = two ? p + 32 : p;
                const int r = pr[p], s = pc[p], r1 = pr[q], s1 = pc[q];
                float sh = Ghi[p], sl = Glo[p], sh1 = Ghi[q], sl1 = Glo[q];
#pragma unroll 4
                for (int i = 0; i < nr; ++i) {
                    const float a = zn[i * RS + r], b = zn[i * RS + s];
                    const float a1 = zn[i * RS + r1], b1 = zn[i * RS + s1];
                    // TwoProduct and TwoSum with uncontracted roundings (see two_sum)
                    const float pa = f_mul(a, b), pa1 = f_mul(a1, b1);
                    const float pe = f_fma(a, b, -pa);          // a*b = pa + pe exactly
                    const float pe1 = f_fma(a1, b1, -pa1);
                    const float t = f_add(sh, pa), t1 = f_add(sh1, pa1);   // TwoSum(sh, pa)
                    const float bv = f_sub(t, sh), bv1 = f_sub(t1, sh1);
                    const float er = f_add(f_sub(sh, f_sub(t, bv)), f_sub(pa, bv));
                    const float er1 = f_add(f_sub(sh1, f_sub(t1, bv1)), f_sub(pa1, bv1));
                    sh = t;
                    sh1 = t1;
                    sl = f_add(sl, f_add(er, pe));
                    sl1 = f_add(sl1, f_add(er1, pe1));
                }
                Ghi[p] = sh;
                Glo[p] = sl;
                if (two) {
                    Ghi[q] = sh1;
                    Glo[q] = sl1;
                }
            }
            __syncwarp();
            base += tot;
        }
        dw *Gk = G + (size_t)k * P;
        for (int p = lane; p < P; p += 32) Gk[p] = two_sum(Ghi[p], Glo[p]);   // normalised pair
        if (Gf) {
            float *Gfk = Gf + (size_t)k * P;
            for (int p = lane; p < P; p += 32) Gfk[p] = Ghi[p] + Glo[p];
        }
        if (MODE3 && ROWWISE) {
            __syncwarp();
            for (int s = lane; s < R; s += 32) {
                float m = 0.f;
                for (int l = 0; l < 32; ++l) m += M3p[l * RS + s];
                M3[(size_t)k * R + s] = m;
                Tk[s] = m;
            }
        } else if (MODE3) {
            const float *Tg = T + (size_t)k * R * R;
            for (int e = lane; e < R * R; e += 32) Tk[e] = Tg[e];
            __syncwarp();
            float *scr = zo;   // 64 RS >= R R floats of scratch
            RowCol rs(lane, R);
            for (int e = lane; e < R * R; e += 32, rs.next(R)) {
                float b = 0.f;
                for (int u = 0; u < R; ++u) b = fmaf(Tk[rs.r * R + u], Cacc[u * R + rs.c], b);
                scr[e] = Hs[e] * b;
            }
            __syncwarp();
            for (int s = lane; s < R; s += 32) {
                float m = 0.f;
                for (int r = 0; r < R; ++r) m += scr[r * R + s];
                M3[(size_t)k * R + s] = m;
                Tk[s] = m;
            }
        }
        if (MODE3) {
            __syncwarp();
            // W(k,:) = M3(k,:) G3inv with G3inv as a float pair and the
            // products accumulated error-free (TwoProduct + TwoSum): FP64-class
            // accuracy without FP64 instructions, whose issue rate on this
            // GPU would make these R^2 products the pass's largest cost.
            for (int s = lane; s < R; s += 32) {
                float hi = 0.f, lo = 0.f;
                for (int u = 0; u < R; ++u) {
                    const float m = Tk[u];
                    pair_fma(hi, lo, m, G3h[u * R + s]);
                    lo = fmaf(m, G3l[u * R + s], lo);
                }
                W[(size_t)k * R + s] = hi + lo;
            }
            __syncwarp();
        }
    }
}

// ---------------------------------------------------------------------------
// Pass beta, part 1: rows of P_k = Z_k F_k with F_k = T_k^T H S_k, so that
// mode 2 (Eq. mttkrp2_3) is M2 = sum_k Y_k^T H S_k = sum_k X_k^T P_k.
// One warp per subject; the rows go to P (N x R) in stacked-row order.
// ---------------------------------------------------------------------------
// bfloat16 bit pattern of v, rounded to nearest even (as Stor<bf16_t>::st)
static __device__ __forceinline__ uint32_t bf16_bits(float v) {
    const bf16_t h = __float2bfloat16_rn(v);
    uint16_t u;
    memcpy(&u, &h, sizeof u);
    return u;
}

// a[0 .. CB) to a 16-byte aligned row segment p as 16-byte vectors: the
// first lim values, zeros up to len (len <= CB, a multiple of the vector)
template <int CB>
static __device__ __forceinline__ void vec_store_row(float *p, const float *a, int lim, int len) {
#pragma unroll
    for (int q = 0; q < CB / 4; ++q) {
        if (4 * q < len) {
            float4 v;
            v.x = 4 * q < lim ? a[4 * q] : 0.f;
            v.y = 4 * q + 1 < lim ? a[4 * q + 1] : 0.f;
            v.z = 4 * q + 2 < lim ? a[4 * q + 2] : 0.f;
            v.w = 4 * q + 3 < lim ? a[4 * q + 3] : 0.f;
            *reinterpret_cast<float4 *>(p + 4 * q) = v;
        }
    }
}
template <int CB>
static __device__ __forceinline__ void vec_store_row(bf16_t *p, const float *a, int lim, int len) {
#pragma unroll
    for (int q = 0; q < CB / 8; ++q) {
        if (8 * q < len) {
            uint32_t w[4];
#pragma unroll
            for (int h = 0; h < 4; ++h) {
                const int c = 8 * q + 2 * h;
                const uint32_t lo = c < lim ? bf16_bits(a[c]) : 0u;
                const uint32_t hi = c + 1 < lim ? bf16_bits(a[c + 1]) : 0u;
                w[h] = lo | (hi << 16);
            }
            *reinterpret_cast<uint4 *>(p + 8 * q) = make_uint4(w[0], w[1], w[2], w[3]);
        }
    }
}

static __host__ __device__ size_t beta_warp_bytes(int R) {
    const size_t b = ((size_t)32 * row_stride(R) + (size_t)R * f_stride(R) + (size_t)R * R + R) * 4;
    return (b + 15) & ~(size_t)15;
}

// The same kernel serves p2_get_U (U_k = Q_k H = Z_k T_k^T H): W == NULL
// stands for S_k = I, the output type O may differ from the storage type S,
// and row r of the view is written at Pout[(r - out_row0) ldo].  With ldo =
// v_stride<O>(R) (the mode-2 rows) every row is a whole number of 16-byte
// vectors, written with vector stores, the padding zero.
template <int CB, class S, class O = S, int RT = 0>
__global__ void __launch_bounds__(256, CB >= 32 ? 1 : 4) k_beta_p(XView X, const S *__restrict__ V,
                                                const float *__restrict__ H,
                                                const float *__restrict__ T,
                                                const float *__restrict__ W, O *Pout, int R_rt,
                                                int64_t out_row0, int ldo) {
    const int R = RT > 0 ? RT : R_rt;   // RT > 0: the rank fixed at compile time
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int RS = row_stride(R);
    float *Hs = reinterpret_cast<float *>(smem_raw);
    const size_t cta_bytes = ((size_t)R * R * 4 + 15) & ~(size_t)15;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int FS = f_stride(R);
    float *zo = reinterpret_cast<float *>(smem_raw + cta_bytes + warp * beta_warp_bytes(R));
    float *Fk = zo + 32 * RS;                   // 16-byte aligned: 32 RS floats = 128 RS bytes
    float *Tk = Fk + R * FS;
    float *wk = Tk + R * R;
    for (int i = threadIdx.x; i < R * R; i += blockDim.x) Hs[i] = H[i];
    __syncthreads();
    const int64_t nwarps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t ki = (int64_t)blockIdx.x * (blockDim.x >> 5) + warp; ki < X.K; ki += nwarps) {
        const int64_t k = X.order ? (int64_t)X.order[ki] : ki;
        const int64_t r0 = X.subj_row[k], r1 = X.subj_row[k + 1];
        if (r1 == r0) continue;
        int64_t base = X.subj_nnz[k];
        const float *Tg = T + (size_t)k * R * R;
        for (int e = lane; e < R * R; e += 32) Tk[e] = Tg[e];
        for (int s = lane; s < R; s += 32) wk[s] = W ? W[(size_t)k * R + s] : 1.f;
        __syncwarp();
        RowCol us(lane, R);
        for (int e = lane; e < R * R; e += 32, us.next(R)) {
            float f = 0.f;
            for (int r = 0; r < R; ++r) f = fmaf(Tk[r * R + us.r], Hs[r * R + us.c], f);
            Fk[us.r * FS + us.c] = f * wk[us.c];
        }
        for (int e = lane; e < R * (FS - R); e += 32) {          // zero padding columns
            const int u = e / (FS - R);
            Fk[u * FS + R + (e - u * (FS - R))] = 0.f;
        }
        __syncwarp();
        for (int64_t cr = r0; cr < r1; cr += 32) {
            const int nr = (int)((r1 - cr) < 32 ? (r1 - cr) : 32);
            const int len = (lane < nr) ? (int)X.row_len[cr + lane] : 0;
            const int off = warp_excl_scan(len, lane);
            const int tot = __shfl_sync(FULLMASK, off + len, 31);
            gather_rows<CB, false, S>(X, nr, base, len, off, V, nullptr, zo, nullptr, R, RS, lane);
            __syncwarp();
            O *Pr = Pout + (size_t)(cr - out_row0) * ldo;
            const bool vec = ldo == v_stride<O>(R);
            // lane i computes row i of Z_k F_k; all lanes read the same F_k row
            // (a shared-memory broadcast) four columns at a time
            if (lane < nr) {
                const float *zr = zo + lane * RS;
                O *Prow = Pr + (size_t)lane * ldo;
                for (int cb = 0; cb < R; cb += CB) {
                    float acc[CB];
#pragma unroll
                    for (int c = 0; c < CB; ++c) acc[c] = 0.f;
                    for (int u = 0; u < R; ++u) {
                        const float a = zr[u];
                        const float4 *f4 = reinterpret_cast<const float4 *>(Fk + u * FS + cb);
#pragma unroll
                        for (int q = 0; q < CB / 4; ++q) {
                            if (cb + 4 * q < R) {
                                const float4 f = f4[q];
                                acc[4 * q] = fmaf(a, f.x, acc[4 * q]);
                                acc[4 * q + 1] = fmaf(a, f.y, acc[4 * q + 1]);
                                acc[4 * q + 2] = fmaf(a, f.z, acc[4 * q + 2]);
                                acc[4 * q + 3] = fmaf(a, f.w, acc[4 * q + 3]);
                            }
                        }
                    }
                    if (vec) {
                        vec_store_row<CB>(Prow + cb, acc, R - cb, ldo - cb);
                    } else {
#pragma unroll
                        for (int c = 0; c < CB; ++c)
                            if (cb + c < R) Stor<O>::st(Prow + cb + c, acc[c]);
                    }
                }
            }
            __syncwarp();
            base += tot;
        }
    }
}

// v[0 .. CB) from a 16-byte aligned row segment p with 16-byte loads (the
// vectors that hold the first lim values)
template <int CB>
static __device__ __forceinline__ void vec_load_row(float *v, const float *__restrict__ p, int lim) {
#pragma unroll
    for (int q = 0; q < CB / 4; ++q) {
        if (4 * q < lim) {
            const float4 t = __ldg(reinterpret_cast<const float4 *>(p) + q);
            v[4 * q] = t.x;
            v[4 * q + 1] = t.y;
            v[4 * q + 2] = t.z;
            v[4 * q + 3] = t.w;
        }
    }
}
template <int CB>
static __device__ __forceinline__ void vec_load_row(float *v, const bf16_t *__restrict__ p, int lim) {
#pragma unroll
    for (int q = 0; q < CB / 8; ++q) {
        if (8 * q < lim) {
            const uint4 t = __ldg(reinterpret_cast<const uint4 *>(p) + q);
            const unsigned w[4] = {t.x, t.y, t.z, t.w};
#pragma unroll
            for (int h = 0; h < 4; ++h) {       // two bfloat16 per word, low half first
                v[8 * q + 2 * h] = __int_as_float((int)(w[h] << 16));
                v[8 * q + 2 * h + 1] = __int_as_float((int)(w[h] & 0xffff0000u));
            }
        }
    }
}

// ---------------------------------------------------------------------------
// Pass beta, part 2: M2(j, :) = sum over the non-zeros x of column j of
// x * P(row, :), read column-major.  One warp per column segment (at most
// P2_SEG non-zeros), one lane per non-zero (32 rows of P in flight per
// warp); each lane accumulates CB components with Kahan-compensated FP32 and
// the lanes are combined by a fixed xor-butterfly in FP64.  No atomics:
// deterministic.
// ---------------------------------------------------------------------------
template <int CB, class S>
__global__ void __launch_bounds__(256) k_m2_segments(const uint32_t *__restrict__ csc_row,
                                                     const float *__restrict__ csc_val,
                                                     const int64_t *__restrict__ seg_start,
                                                     const int64_t *__restrict__ seg_end,
                                                     int64_t sg0, int64_t sg1,
                                                     const S *__restrict__ Pin, int64_t row0,
                                                     double *segpart, int R) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int PS = v_stride<S>(R);              // P rows padded to 16-byte vectors
    const int64_t nwarps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t sg = sg0 + (int64_t)blockIdx.x * (blockDim.x >> 5) + warp; sg < sg1; sg += nwarps) {
        const int64_t a = seg_start[sg], b = seg_end[sg];
        for (int cb = 0; cb < R; cb += CB) {
            float hi[CB], cp[CB];
#pragma unroll
            for (int c = 0; c < CB; ++c) {
                hi[c] = 0.f;
                cp[c] = 0.f;
            }
            for (int64_t e = a + lane; e < b; e += 32) {
                const uint32_t row = csc_row[e];
                const float x = csc_val[e];
                const S *pr = Pin + (size_t)((int64_t)row - row0) * PS + cb;  // the block's P rows
                float pv[CB];
                vec_load_row<CB>(pv, pr, R - cb);
#pragma unroll
                for (int c = 0; c < CB; ++c) {
                    if (cb + c < R) {
                        const float y = x * pv[c] - cp[c];
                        const float tt = hi[c] + y;
                        cp[c] = (tt - hi[c]) - y;
                        hi[c] = tt;
                    }
                }
            }
#pragma unroll
            for (int c = 0; c < CB; ++c) {
                if (cb + c < R) {
                    double v = (double)hi[c] - (double)cp[c];
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULLMASK, v, o);
                    if (lane == 0) segpart[(size_t)sg * R + cb + c] = v;
                }
            }
        }
    }
}

// M2(j, :) = sum of column j's segment partials (FP64), blocks in order: one
// warp per column, lanes take each block's segments in a fixed stride,
// combined by a fixed xor-butterfly.
__global__ void k_m2_columns(const double *__restrict__ segpart, const int64_t *__restrict__ col_seg,
                             double *M2, int32_t J, int nblk, int R) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t nwarps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t j = (int64_t)blockIdx.x * (blockDim.x >> 5) + warp; j < J; j += nwarps) {
        for (int c = 0; c < R; ++c) {
            double acc = 0.0;
            for (int bk = 0; bk < nblk; ++bk) {
                const int64_t v = (int64_t)bk * J + j;
                for (int64_t sg = col_seg[v] + lane; sg < col_seg[v + 1]; sg += 32)
                    acc += segpart[(size_t)sg * R + c];
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(FULLMASK, acc, o);
            if (lane == 0) M2[(size_t)j * R + c] = acc;
        }
    }
}

// ---------------------------------------------------------------------------
// Per-subject statistics after the Q-step, in one pass over the subjects:
//   mode 1 (Eq. mttkrp1_3): M1 = sum_k (T_k G_k) * 1 W(k,:)   (Y_k V = T_k G_k),
//   W^TW and <W, M3>.
// One block per fixed contiguous subject range and one warp per subject at a
// time (no block barriers in the loop).  M1 products in FP32; the sums over
// subjects (and W^TW's products, split exactly) accumulate as float pairs.
// Block partials in FP64, layout [R*R M1][R*R WtW][1 wm3], summed later in
// block order.
// ---------------------------------------------------------------------------
// Body of the statistics kernels; G is the packed Gram as float (the copy the
// alpha pass writes for this kernel) or double (the allocation-free entry
// point's interface).  Accumulations use float pairs: ~2^-48 relative error
// and no FP64 instruction per subject.
template <class GT, int RT = 0>
static __device__ __forceinline__ void subject_stats(const float *__restrict__ T,
                                                     const GT *__restrict__ G,
                                                     const float *__restrict__ W,
                                                     const float *__restrict__ M3, double *part,
                                                     int64_t K, int R_rt, int with_m3) {
    const int R = RT > 0 ? RT : R_rt;   // RT > 0: the rank fixed at compile time
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ double red_wm3[16];
    const int P = R * (R + 1) / 2;
    const int RR = R * R;
    const int nw = blockDim.x >> 5, warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    uint8_t *pr = smem_raw;
    uint8_t *pc = pr + P;
    const size_t cta_bytes = (2 * (size_t)P + 15) & ~(size_t)15;
    const size_t wbytes = stats_warp_bytes(R);
    unsigned char *wb = smem_raw + cta_bytes + warp * wbytes;
    float *m1h = reinterpret_cast<float *>(wb);     // R*R each: M1 and W^TW pairs
    float *m1l = m1h + RR;
    float *wth = m1l + RR;
    float *wtl = wth + RR;
    float *Ts = wtl + RR;
    float *Gs = Ts + RR;
    float *ws = Gs + RR;
    for (int p = threadIdx.x; p < P; p += blockDim.x) {
        int r = (int)((sqrt(8.0 * p + 1.0) - 1.0) * 0.5);
        while ((r + 1) * (r + 2) / 2 <= p) ++r;
        while (r * (r + 1) / 2 > p) --r;
        pr[p] = (uint8_t)r;
        pc[p] = (uint8_t)(p - r * (r + 1) / 2);
    }
    for (int e = lane; e < RR; e += 32) {
        m1h[e] = 0.f;
        m1l[e] = 0.f;
        wth[e] = 0.f;
        wtl[e] = 0.f;
    }
    __syncthreads();
    const int64_t per = (K + gridDim.x - 1) / gridDim.x;
    const int64_t k0 = (int64_t)blockIdx.x * per;
    const int64_t k1 = (k0 + per < K) ? (k0 + per) : K;
    float wm3h = 0.f, wm3l = 0.f;
    const int r0 = lane / R, c0 = lane - (lane / R) * R;   // first entry of this lane
    for (int64_t k = k0 + warp; k < k1; k += nw) {
        const float *Tg = T + (size_t)k * RR;
        const GT *Gg = G + (size_t)k * P;
        for (int e = lane; e < RR; e += 32) Ts[e] = Tg[e];
        for (int p = lane; p < P; p += 32) {
            const float g = (float)Gg[p];
            const int r = pr[p], c = pc[p];
            Gs[r * R + c] = g;
            Gs[c * R + r] = g;
        }
#pragma unroll
        for (int t = 0; t < 2; ++t) {
            const int s = lane + 32 * t;
            if (s < R) {
                const float v = W[(size_t)k * R + s];
                ws[s] = v;
                if (with_m3) pair_fma(wm3h, wm3l, v, M3[(size_t)k * R + s]);
            }
        }
        __syncwarp();
        int r = r0, c = c0;
        for (int e = lane; e < RR; e += 32) {
            float sacc = 0.f;
            for (int u = 0; u < R; ++u) sacc = fmaf(Ts[r * R + u], Gs[u * R + c], sacc);
            pair_add(m1h[e], m1l[e], sacc * ws[c]);
            pair_fma(wth[e], wtl[e], ws[r], ws[c]);
            c += 32;                                   // next entry e + 32
            while (c >= R) {
                c -= R;
                ++r;
            }
        }
        __syncwarp();
    }
    // fixed-order reductions: lanes, then warps in index order
    double wm3 = (double)wm3h + (double)wm3l;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) wm3 += __shfl_down_sync(FULLMASK, wm3, o);
    if (lane == 0) red_wm3[warp] = wm3;
    __syncthreads();
    const size_t stride = stats_part_stride(R);
    double *out = part + (size_t)blockIdx.x * stride;
    for (int e = threadIdx.x; e < RR; e += blockDim.x) {
        double m = 0.0, w2 = 0.0;
        for (int q = 0; q < nw; ++q) {
            const float *aq = reinterpret_cast<const float *>(smem_raw + cta_bytes + q * wbytes);
            m += (double)aq[e] + (double)aq[RR + e];
            w2 += (double)aq[2 * RR + e] + (double)aq[3 * RR + e];
        }
        out[e] = m;
        out[RR + e] = w2;
    }
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int q = 0; q < nw; ++q) t += red_wm3[q];
        out[2 * RR] = t;
    }
}

__global__ void __launch_bounds__(256) k_subject_stats(const float *__restrict__ T,
                                                       const double *__restrict__ G,
                                                       const float *__restrict__ W,
                                                       const float *__restrict__ M3, double *part,
                                                       int64_t K, int R, int with_m3) {
    subject_stats<double>(T, G, W, M3, part, K, R, with_m3);
}

template <int RT>
__global__ void __launch_bounds__(512, 2) k_subject_stats_gf(const float *__restrict__ T,
                                                          const float *__restrict__ Gf,
                                                          const float *__restrict__ W,
                                                          const float *__restrict__ M3,
                                                          double *part, int64_t K, int R,
                                                          int with_m3) {
    subject_stats<float, RT>(T, Gf, W, M3, part, K, R, with_m3);
}


// Partials of V^T V (V stored FP32, products exact in FP64) over row ranges.
template <class S>
__global__ void __launch_bounds__(256) k_gram_v(const S *__restrict__ V, double *part,
                                                int64_t J, int R) {
    const int64_t per = (J + gridDim.x - 1) / gridDim.x;
    const int64_t j0 = (int64_t)blockIdx.x * per;
    const int64_t j1 = (j0 + per < J) ? (j0 + per) : J;
    double acc[16];
#pragma unroll
    for (int q = 0; q < 16; ++q) acc[q] = 0.0;
    for (int64_t j = j0; j < j1; ++j) {
        const S *vj = V + (size_t)j * v_stride<S>(R);
#pragma unroll
        for (int q = 0; q < 16; ++q) {
            const int e = threadIdx.x + q * blockDim.x;
            if (e < R * R) {
                const int r = e / R, s = e - r * R;
                acc[q] = fma((double)Stor<S>::ldp(vj + r), (double)Stor<S>::ldp(vj + s), acc[q]);
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
// and U the eigenvectors (columns).  A pair is rotated while |a_pq| exceeds
// eps sqrt(|a_pp a_qq|) and abs_floor (a floor of the order of eps ||A||
// ends the sweeps on a block of rounding noise, such as a null space).
static __device__ void cta_jacobi(double *A, double *U, int n, int *flags, double abs_floor = 0.0) {
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
                    if (fabs(apq) > eps * sqrt(fabs(app * aqq)) && fabs(apq) > fmax(1e-300, abs_floor)) {
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

// out = A^-1 by a Cholesky factorisation A = L L^T (in C), L^-1 (in U) and
// A^-1 = L^-T L^-1, when that provably equals A^+ as cta_pinv defines it:
// every eigenvalue above the cut n 2^-52 lambda_max.  lambda_min >=
// 1 / trace(A^-1) and lambda_max <= trace(A), so a margin of 2^10 between
// 1 / trace(A^-1) and n 2^-52 trace(A) leaves no eigenvalue near the cut.
// Returns false (out untouched, A untouched) when the factorisation breaks
// down or the bound does not hold.  A chain of ~2n FP64 square roots and
// divisions instead of the Jacobi sweeps' ~6n rounds of them.
static __device__ bool cta_inv_chol(const double *A, double *C, double *U, double *out, int n) {
    __shared__ double rinv[P2_RMAX];
    __shared__ int ok;
    __shared__ double tra, trinv;
    const int tid = threadIdx.x, nt = blockDim.x;
    for (int e = tid; e < n * n; e += nt) {
        C[e] = A[e];
        U[e] = 0.0;
    }
    if (tid == 0) {
        ok = 1;
        double t = 0.0;
        for (int i = 0; i < n; ++i) t += A[i * n + i];
        tra = t;
    }
    __syncthreads();
    for (int k = 0; k < n; ++k) {                        // right-looking, lower triangle
        if (tid == 0) {
            const double d = C[k * n + k];
            if (!(d > 0.0) || !ok) {
                ok = 0;
            } else {
                const double l = sqrt(d);
                C[k * n + k] = l;
                rinv[k] = 1.0 / l;
            }
        }
        __syncthreads();
        if (!ok) return false;
        for (int i = k + 1 + tid; i < n; i += nt) C[i * n + k] *= rinv[k];
        __syncthreads();
        for (int e = tid; e < (n - k - 1) * (n - k - 1); e += nt) {
            const int i = k + 1 + e / (n - k - 1), j = k + 1 + e % (n - k - 1);
            if (j <= i) C[i * n + j] = fma(-C[i * n + k], C[j * n + k], C[i * n + j]);
        }
        __syncthreads();
    }
    for (int j = tid; j < n; j += nt) {                  // column j of L^-1 (lower)
        for (int i = j; i < n; ++i) {
            double s = (i == j) ? 1.0 : 0.0;
            for (int m = j; m < i; ++m) s = fma(-C[i * n + m], U[m * n + j], s);
            U[i * n + j] = s * rinv[i];
        }
    }
    __syncthreads();
    for (int e = tid; e < n * n; e += nt) {              // (L^-T L^-1)_{ij}
        const int i = e / n, j = e - (e / n) * n;
        double s = 0.0;
        for (int m = (i > j ? i : j); m < n; ++m) s = fma(U[m * n + i], U[m * n + j], s);
        C[e] = s;
    }
    __syncthreads();
    if (tid == 0) {
        double t = 0.0;
        for (int i = 0; i < n; ++i) t += C[i * n + i];
        trinv = t;
    }
    __syncthreads();
    const double cut = (double)n * 2.220446049250313e-16 * tra;
    if (!(trinv > 0.0) || !(1.0 / trinv > 1024.0 * cut) || !isfinite(trinv)) return false;
    for (int e = tid; e < n * n; e += nt) out[e] = C[e];
    __syncthreads();
    return true;
}

// out = A^+ for the symmetric PSD n x n matrix in A (destroyed); U and C are
// n x n scratch.  Eigenvalues <= n * 2^-52 * lambda_max are dropped (by the
// Jacobi eigen-decomposition; the Cholesky inverse where it provably gives
// the same matrix, up to rounding).
static __device__ void cta_pinv(double *A, double *U, double *C, double *out, int n, int *flags) {
    __shared__ double f[P2_RMAX];
    if (cta_inv_chol(A, C, U, out, n)) return;
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

// ---------------------------------------------------------------------------
// Rational start (Kiers, ten Berge & Bro, J. Chemometrics 13, 1999): H = I,
// S_k = I and V = the R leading eigenvectors of A = sum_k X_k^T X_k.  They
// come from subspace iteration with a Rayleigh-Ritz step on every product
// (Golub & Van Loan, "Matrix Computations", 4th ed., Section 8.2.4; Stewart,
// Numer. Math. 25, 1976) over a block of b >= R columns, so the leading R
// Ritz vectors converge at the rate lambda_{b+1} / lambda_R.  A V is formed
// as X^T (X V) without the J x J matrix.  One-time work, all in FP64: the
// eigenvalues of A are often close (adjacent ratios of 0.98 on the synthetic
// workloads) and an eigenvector's error is the product's relative error
// times lambda_1 over its gap.
// ---------------------------------------------------------------------------

// Sum of v over the CTA in a fixed order (lanes by a butterfly, then the
// warps in order), returned to every thread; red holds one double per warp.
static __device__ double cta_sum(double v, double *red) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULLMASK, v, o);
    __syncthreads();                       // red is free from its previous use
    if (lane == 0) red[warp] = v;
    __syncthreads();
    double s = 0.0;
    for (int w = 0; w < nw; ++w) s += red[w];
    return s;
}

// out[q] = sum_j A(j, ca[q]) B(j, cb[q]) for q < nq <= 8 (A, B: J rows of
// strides lda, ldb), by the whole CTA: threads over rows, the partial sums
// in shared memory (8 blockDim.x doubles at part) added in thread order.
static __device__ void cta_dots8(const double *__restrict__ A, int lda,
                                 const double *__restrict__ B, int ldb, const int *ca,
                                 const int *cb, int nq, int32_t J, double *part, double *out) {
    const int tid = threadIdx.x, nt = blockDim.x;
    double acc[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) acc[q] = 0.0;
    for (int32_t j = tid; j < J; j += nt) {
        const double *a = A + (size_t)j * lda, *bb = B + (size_t)j * ldb;
#pragma unroll
        for (int q = 0; q < 8; ++q)
            if (q < nq) acc[q] = fma(a[ca[q]], bb[cb[q]], acc[q]);
    }
#pragma unroll
    for (int q = 0; q < 8; ++q) part[q * nt + tid] = acc[q];
    __syncthreads();
    if (tid < nq) {
        double v = 0.0;
        for (int t = 0; t < nt; ++t) v += part[tid * nt + t];
        out[tid] = v;
    }
    __syncthreads();
}

// Columns c0 .. c0+CW-1 of Z = X Vd in FP64 (stacked rows, N x CW; Vd is
// J x b): one warp per subject, one lane per row of a 32-row chunk, row
// offsets from a warp scan of the row lengths.
__global__ void __launch_bounds__(256) k_eig_z(XView X, const double *__restrict__ Vd, int b,
                                               int c0, int CW, double *Z) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t nwarps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t k = (int64_t)blockIdx.x * (blockDim.x >> 5) + warp; k < X.K; k += nwarps) {
        const int64_t r0 = X.subj_row[k], r1 = X.subj_row[k + 1];
        int64_t base = X.subj_nnz[k];
        for (int64_t cr = r0; cr < r1; cr += 32) {
            const int nr = (int)((r1 - cr) < 32 ? (r1 - cr) : 32);
            const int len = (lane < nr) ? (int)X.row_len[cr + lane] : 0;
            const int off = warp_excl_scan(len, lane);
            const int tot = __shfl_sync(FULLMASK, off + len, 31);
            if (lane < nr) {
                const int64_t b0 = base + off;
                double *zr = Z + (size_t)(cr + lane) * CW;
                for (int c8 = 0; c8 < CW; c8 += 8) {     // eight components per pass over the row
                    double a[8];
#pragma unroll
                    for (int q = 0; q < 8; ++q) a[q] = 0.0;
                    for (int e = 0; e < len; ++e) {
                        const double x = (double)X.val[b0 + e];
                        const double *v = Vd + (size_t)X.col[b0 + e] * b + c0 + c8;
#pragma unroll
                        for (int q = 0; q < 8; ++q)
                            if (c8 + q < CW) a[q] = fma(x, v[q], a[q]);
                    }
#pragma unroll
                    for (int q = 0; q < 8; ++q)
                        if (c8 + q < CW) zr[c8 + q] = a[q];
                }
            }
            base += tot;
        }
    }
}

// Segment partials of X^T Z in FP64 (Z: N x CW), segpart rows CW wide: one
// thread per (segment, component), summing the segment's non-zeros in order.
__global__ void __launch_bounds__(256) k_eig_m2_segments(const uint32_t *__restrict__ csc_row,
                                                         const float *__restrict__ csc_val,
                                                         const int64_t *__restrict__ seg_start,
                                                         const int64_t *__restrict__ seg_end,
                                                         int64_t nseg, const double *__restrict__ Z,
                                                         int CW, double *segpart) {
    const int64_t n = nseg * CW, stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += stride) {
        const int64_t sg = t / CW;
        const int c = (int)(t - sg * CW);
        double v = 0.0;
        for (int64_t e = seg_start[sg]; e < seg_end[sg]; ++e)
            v = fma((double)csc_val[e], Z[(size_t)csc_row[e] * CW + c], v);
        segpart[t] = v;
    }
}

// Y(j, c0 + c) = sum of column j's segment partials in order (rows CW wide),
// blocks in order: Y J x b, one thread per (column, component).
__global__ void k_eig_m2_columns(const double *__restrict__ segpart,
                                 const int64_t *__restrict__ col_seg, int32_t J, int nblk, int CW,
                                 double *Y, int b, int c0) {
    const int64_t n = (int64_t)J * CW, stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += stride) {
        const int64_t j = t / CW;
        const int c = (int)(t - j * CW);
        double acc = 0.0;
        for (int bk = 0; bk < nblk; ++bk) {
            const int64_t v = (int64_t)bk * J + j;
            for (int64_t sg = col_seg[v]; sg < col_seg[v + 1]; ++sg)
                acc += segpart[(size_t)sg * CW + c];
        }
        Y[(size_t)j * b + c0 + c] = acc;
    }
}

// H = I, W = 1
__global__ void k_eig_fill(float *H, float *W, int64_t K, int R) {
    const int64_t n = K * R, stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += stride) W[e] = 1.f;
    if (blockIdx.x == 0)
        for (int e = threadIdx.x; e < R * R; e += blockDim.x) H[e] = (e / R == e % R) ? 1.f : 0.f;
}

// Orthonormal basis Q (J x b, FP64, row-major) of the columns of Y by
// classical Gram-Schmidt with one full reorthogonalisation (CGS2, orthogonal
// to working precision while the columns are numerically independent:
// Giraud, Langou, Rozloznik & van den Eshof, Numer. Math. 101, 2005); the
// leading columns of Q span the leading columns of Y.  A column left with at
// most 2^-40 of its norm, or of the first column's norm, after both passes
// depends on the earlier ones numerically (or is rounding noise, as the
// columns of A V U for A's null space are); it is replaced by the unit vector
// e_j with the largest
// component outside their span (lowest j on ties; that component is at least
// 1/sqrt(J) when J >= b) and orthogonalised again, so Q always has b
// orthonormal columns.  With Vold (J x b), *dist = ||Q_R - Vold_R Vold_R^T
// Q_R||_F^2 over the leading R columns of both: the sum of the squared sines
// of the principal angles between the two leading subspaces.  Dynamic
// shared memory: 8 blockDim.x doubles.  One CTA of whole warps.
__global__ void __launch_bounds__(256) k_eig_orth(const double *__restrict__ Y,
                                                  const double *__restrict__ Vold, double *Q,
                                                  int32_t J, int b, int R, double *dist,
                                                  int *flags) {
    extern __shared__ __align__(16) double part[];   // 8 blockDim.x doubles (cta_dots8)
    __shared__ double coef[P2_RMAX];
    __shared__ double red[32];
    __shared__ int32_t redj[32];
    __shared__ int32_t pick;
    const int tid = threadIdx.x, nt = blockDim.x;
    const int lane = tid & 31, warp = tid >> 5, nw = nt >> 5;
    double scale = 0.0;                        // norm of Y's first column
    for (int r = 0; r < b; ++r) {
        for (int32_t j = tid; j < J; j += nt) Q[(size_t)j * b + r] = Y[(size_t)j * b + r];
        __syncthreads();
        double a0 = 0.0;
        for (int32_t j = tid; j < J; j += nt) {
            const double q = Q[(size_t)j * b + r];
            a0 = fma(q, q, a0);
        }
        double ref = sqrt(cta_sum(a0, red));   // norm before the projections
        if (r == 0) scale = ref;
        for (int attempt = 0; attempt < 2; ++attempt) {
            for (int pass = 0; pass < 2; ++pass) {
                for (int s0 = 0; s0 < r; s0 += 8) {
                    int ca[8], cb[8];
#pragma unroll
                    for (int q = 0; q < 8; ++q) {
                        ca[q] = s0 + q;
                        cb[q] = r;
                    }
                    cta_dots8(Q, b, Q, b, ca, cb, r - s0 < 8 ? r - s0 : 8, J, part, coef + s0);
                }
                for (int32_t j = tid; j < J; j += nt) {
                    double q = Q[(size_t)j * b + r];
                    for (int s = 0; s < r; ++s) q = fma(-coef[s], Q[(size_t)j * b + s], q);
                    Q[(size_t)j * b + r] = q;
                }
                __syncthreads();
            }
            double a = 0.0;
            for (int32_t j = tid; j < J; j += nt) {
                const double q = Q[(size_t)j * b + r];
                a = fma(q, q, a);
            }
            const double nrm = sqrt(cta_sum(a, red));
            if (nrm > 0x1p-40 * fmax(ref, scale) && nrm > 0.0) {
                const double inv = 1.0 / nrm;
                for (int32_t j = tid; j < J; j += nt) Q[(size_t)j * b + r] *= inv;
                __syncthreads();
                break;
            }
            if (attempt == 1) {                // not reached when J >= b
                if (tid == 0) atomicOr(flags, FLAG_EIG_NOCONV);
                break;
            }
            // replacement: the e_j with the largest 1 - sum_{s<r} Q(j,s)^2
            double best = -1.0;
            int32_t bj = 0;
            for (int32_t j = tid; j < J; j += nt) {
                double w = 1.0;
                for (int s = 0; s < r; ++s) {
                    const double q = Q[(size_t)j * b + s];
                    w = fma(-q, q, w);
                }
                if (w > best) {                // j increases within a thread: first max kept
                    best = w;
                    bj = j;
                }
            }
            for (int o = 16; o > 0; o >>= 1) {
                const double ob = __shfl_xor_sync(FULLMASK, best, o);
                const int32_t oj = __shfl_xor_sync(FULLMASK, bj, o);
                if (ob > best || (ob == best && oj < bj)) {
                    best = ob;
                    bj = oj;
                }
            }
            __syncthreads();
            if (lane == 0) {
                red[warp] = best;
                redj[warp] = bj;
            }
            __syncthreads();
            if (tid == 0) {
                double bb = red[0];
                int32_t jb = redj[0];
                for (int w = 1; w < nw; ++w)
                    if (red[w] > bb || (red[w] == bb && redj[w] < jb)) {
                        bb = red[w];
                        jb = redj[w];
                    }
                pick = jb;
            }
            __syncthreads();
            const int32_t jp = pick;
            for (int32_t j = tid; j < J; j += nt) Q[(size_t)j * b + r] = (j == jp) ? 1.0 : 0.0;
            __syncthreads();
            ref = 1.0;
            if (r == 0) scale = 1.0;
        }
    }
    if (Vold) {
        // C = Vold_R^T Q_R, then ||Q_R - Vold_R C||_F^2 (no cancellation
        // against R, so the distance resolves well below eps)
        __shared__ double C[P2_RMAX * P2_RMAX];
        for (int e0 = 0; e0 < R * R; e0 += 8) {
            int ca[8], cb[8];
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                const int e = e0 + q < R * R ? e0 + q : 0;
                ca[q] = e / R;
                cb[q] = e - (e / R) * R;
            }
            cta_dots8(Vold, b, Q, b, ca, cb, R * R - e0 < 8 ? R * R - e0 : 8, J, part, C + e0);
        }
        double a = 0.0;
        for (int32_t j = tid; j < J; j += nt)
            for (int t = 0; t < R; ++t) {
                double res = Q[(size_t)j * b + t];
                for (int s = 0; s < R; ++s) res = fma(-Vold[(size_t)j * b + s], C[s * R + t], res);
                a = fma(res, res, a);
            }
        const double tot = cta_sum(a, red);
        if (tid == 0) *dist = tot;
    }
}

// Rayleigh-Ritz step on the orthonormal Vd (J x b) with Y = A Vd:
// B = Vd^T Y (symmetrised) = U diag(l) U^T by the CTA Jacobi, the columns of
// U in decreasing order of l (lower index first on ties).  Not final:
// Out = Y U, the next block before orthonormalisation.  Final: Out = Vd U
// (the Ritz vectors), each column's entry of largest magnitude made positive
// (lowest row on ties), and the leading R columns stored to V (storage type
// S, row stride VS, zero padding).  Dynamic shared memory: 2 b^2 doubles.
// Dynamic shared memory: 2 b^2 + 8 blockDim.x doubles.  One CTA of whole
// warps.
template <class S>
__global__ void __launch_bounds__(256) k_eig_ritz(const double *__restrict__ Y,
                                                  const double *__restrict__ Vd, double *Out,
                                                  S *V, int VS, int32_t J, int b, int R,
                                                  int final_step, int *flags) {
    extern __shared__ __align__(16) double sd[];
    double *A = sd, *U = A + b * b, *part = U + b * b;   // part: 8 blockDim.x doubles
    __shared__ int perm[P2_RMAX];
    __shared__ double sgn[P2_RMAX];
    const int tid = threadIdx.x, nt = blockDim.x;
    for (int e0 = 0; e0 < b * b; e0 += 8) {
        int ca[8], cb[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const int e = e0 + q < b * b ? e0 + q : 0;
            ca[q] = e / b;
            cb[q] = e - (e / b) * b;
        }
        cta_dots8(Vd, b, Y, b, ca, cb, b * b - e0 < 8 ? b * b - e0 : 8, J, part, U + e0);
    }
    __shared__ double fro;
    for (int e = tid; e < b * b; e += nt) {
        const int s = e / b, t = e - s * b;
        A[e] = 0.5 * (U[s * b + t] + U[t * b + s]);
    }
    __syncthreads();
    if (tid == 0) {
        double f = 0.0;
        for (int e = 0; e < b * b; ++e) f = fma(A[e], A[e], f);
        fro = sqrt(f);
    }
    __syncthreads();
    cta_jacobi(A, U, b, flags, 2.220446049250313e-16 * fro);
    if (tid == 0) {
        for (int i = 0; i < b; ++i) perm[i] = i;
        for (int i = 1; i < b; ++i) {          // stable insertion sort, decreasing l
            const int p = perm[i];
            const double lp = A[p * b + p];
            int l = i;
            while (l > 0 && A[perm[l - 1] * b + perm[l - 1]] < lp) {
                perm[l] = perm[l - 1];
                --l;
            }
            perm[l] = p;
        }
    }
    __syncthreads();
    const double *Src = final_step ? Vd : Y;
    for (int32_t j = tid; j < J; j += nt)
        for (int col = 0; col < b; ++col) {
            double a = 0.0;
            for (int u = 0; u < b; ++u) a = fma(Src[(size_t)j * b + u], U[u * b + perm[col]], a);
            Out[(size_t)j * b + col] = a;
        }
    __syncthreads();
    if (!final_step) return;
    for (int col = tid; col < R; col += nt) {
        double best = -1.0, val = 0.0;
        for (int32_t j = 0; j < J; ++j) {      // first maximum: lowest row on ties
            const double v = Out[(size_t)j * b + col];
            if (fabs(v) > best) {
                best = fabs(v);
                val = v;
            }
        }
        sgn[col] = val < 0.0 ? -1.0 : 1.0;
    }
    __syncthreads();
    for (size_t e = tid; e < (size_t)J * VS; e += nt) {
        const size_t j = e / VS;
        const int col = (int)(e - j * VS);
        double v = 0.0;
        if (col < R) {
            v = sgn[col] * Out[j * b + col];
            Out[j * b + col] = v;
        }
        Stor<S>::st(V + e, (float)v);
    }
}

// H solve: M1 = sum of partials; H = normalize(M1 (W^TW * V^TV)^+); H64, HtH.
__global__ void __launch_bounds__(256) k_solve_h(const double *__restrict__ part, int nparts,
                                                 SmallState *st, float *H, int R) {
    extern __shared__ __align__(16) double sd[];
    double *A = sd, *U = A + R * R, *Pi = U + R * R, *Hn = Pi + R * R;
    __shared__ double nrm[P2_RMAX];
    for (int e = threadIdx.x; e < R * R; e += blockDim.x) {
        double s = 0.0;
        for (int b = 0; b < nparts; ++b) s += part[(size_t)b * stats_part_stride(R) + e];
        st->M1[e] = s;
        A[e] = st->WtW[e] * st->VtV[e];
    }
    __syncthreads();
    cta_pinv(A, U, Hn, Pi, R, &st->flags);            // Hn: scratch until written below
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
    double *A = sd, *U = A + R * R, *C = U + R * R;
    for (int e = threadIdx.x; e < R * R; e += blockDim.x) A[e] = st->WtW[e] * st->HtH[e];
    __syncthreads();
    cta_pinv(A, U, C, st->P2inv, R, &st->flags);
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
template <class S>
__global__ void k_solve_v_store(const double *__restrict__ Vun, const SmallState *st, S *V,
                                S *Vprev, int64_t n, int R) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t j = e / R;
        const int s = (int)(e - j * R);
        const int64_t d = j * v_stride<S>(R) + s;   // V rows are padded (see v_stride)
        const double nr = st->colnorm[s];
        Vprev[d] = V[d];
        Stor<S>::st(V + d, nr > 0.0 ? (float)(Vun[e] / nr) : 0.f);
    }
}

// Sum V^TV partials; G3inv = (V^TV * H^TH)^+.
__global__ void __launch_bounds__(256) k_fin_v(const double *__restrict__ part, int nparts,
                                               SmallState *st, int R, int with_g3) {
    extern __shared__ __align__(16) double sd[];
    double *A = sd, *U = A + R * R, *C = U + R * R;     // C: with_g3 only (4 R^2 doubles)
    for (int e = threadIdx.x; e < R * R; e += blockDim.x) {
        double s = 0.0;
        for (int b = 0; b < nparts; ++b) s += part[(size_t)b * R * R + e];
        st->VtV[e] = s;
        A[e] = s * st->HtH[e];
    }
    __syncthreads();
    if (with_g3) cta_pinv(A, U, C, st->G3inv, R, &st->flags);
}

// The exchange hook of a sharded context: sums buf over the shards in place
// (see p2_set_exchange).
int exchange(p2_ctx *c, double *buf, int64_t count) {
    if (!c->xfn) return P2_OK;
    const int r = c->xfn(buf, count, (void *)c->stream, c->xuser);
    if (r != 0) {
        set_error("the exchange hook returned %d (%lld values)", r, (long long)count);
        return P2_EEXCHANGE;
    }
    return P2_OK;
}

// out[e] = sum of the nparts rows of part (row stride `stride`), in row
// order: the one-row statistics a sharded context exchanges.
__global__ void k_part_rows_sum(const double *__restrict__ part, int nparts, int64_t stride,
                                double *out) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < stride;
         e += (int64_t)gridDim.x * blockDim.x) {
        double s = 0.0;
        for (int b = 0; b < nparts; ++b) s += part[(size_t)b * stride + e];
        out[e] = s;
    }
}

// Sum the subject-statistics partials: W^TW, <W, M3>; loss / fit.
// (M1 stays in the partials; the H solve sums it.)
__global__ void k_fin_w(const double *__restrict__ part, int nparts, SmallState *st, int R,
                        int with_fit) {
    const size_t stride = stats_part_stride(R);
    __shared__ double red[256];
    double lsum = 0.0;
    for (int e = threadIdx.x; e < R * R; e += blockDim.x) {
        double s = 0.0;
        for (int b = 0; b < nparts; ++b) s += part[(size_t)b * stride + R * R + e];
        st->WtW[e] = s;
        lsum += s * st->HtH[e] * st->VtV[e];
    }
    red[threadIdx.x] = lsum;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int i = 0; i < (int)blockDim.x; ++i) t += red[i];
        if (with_fit) {
            double wm3 = 0.0;
            for (int b = 0; b < nparts; ++b) wm3 += part[(size_t)b * stride + 2 * R * R];
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
static size_t alpha_warp_bytes(int R) { return alpha_warp_bytes_dev(R); }

// register block of components in the sparse passes: 8, 16 or 32
static int comp_block(int R) { return R <= 8 ? 8 : (R <= 16 ? 16 : 32); }

// V, Vprev, T and P of the context in storage type S
template <class S> struct Bufs;
template <> struct Bufs<float> {
    static float *V(const p2_ctx *c) { return c->d_V; }
    static float *Vprev(const p2_ctx *c) { return c->d_Vprev; }
    static float *P(const p2_ctx *c) { return c->d_P; }
};
template <> struct Bufs<bf16_t> {
    static bf16_t *V(const p2_ctx *c) { return c->d_Vh; }
    static bf16_t *Vprev(const p2_ctx *c) { return c->d_Vprevh; }
    static bf16_t *P(const p2_ctx *c) { return c->d_Ph; }
};

struct Launch {
    int alpha_warps, beta_warps, alpha_blocks, beta_blocks;
    size_t alpha_smem, beta_smem;
};

// CTAs of this shape that fit on one SM (shared memory and 2048 threads).
static int blocks_per_sm(const p2_ctx *c, size_t smem, int threads) {
    const size_t usable = 233472;   // per-SM shared memory (228 KB) on this GPU
    int b = smem > 0 ? (int)(usable / (smem + 1024)) : 32;
    if (b > 2048 / threads) b = 2048 / threads;
    if (b > (int)((size_t)c->geo.smem_optin / (smem > 0 ? smem : 1))) b = (int)((size_t)c->geo.smem_optin / (smem > 0 ? smem : 1));
    return b < 1 ? 1 : b;
}

// Blocks of this kernel resident on one SM (registers, shared memory,
// threads), from the occupancy calculator; the persistent passes launch
// exactly that many per SM.
template <class Kern>
static int resident_blocks(const p2_ctx *c, Kern kern, int threads, size_t smem) {
    int b = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, kern, threads, smem) != cudaSuccess ||
        b < 1) {
        cudaGetLastError();
        b = blocks_per_sm(c, smem, threads);
    }
    return b;
}

static Launch plan(const p2_ctx *c) {
    Launch L{};
    const int R = c->R;
    const size_t cap = (size_t)c->geo.smem_optin;
    const int wmax = 8;                                 // the passes' launch bounds (256 threads)
    int aw = wmax;
    while (aw > 1 && alpha_cta_bytes(R) + aw * alpha_warp_bytes(R) > cap) --aw;
    L.alpha_warps = aw;
    L.alpha_smem = alpha_cta_bytes(R) + aw * alpha_warp_bytes(R);
    int bw = wmax;
    const size_t bcta = ((size_t)R * R * 4 + 15) & ~(size_t)15;
    while (bw > 1 && bcta + bw * beta_warp_bytes(R) > cap) --bw;
    L.beta_warps = bw;
    L.beta_smem = bcta + bw * beta_warp_bytes(R);
    L.alpha_blocks = blocks_per_sm(c, L.alpha_smem, L.alpha_warps * 32);
    L.beta_blocks = blocks_per_sm(c, L.beta_smem, L.beta_warps * 32);
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

// Ranks 1 .. 16 and the multiples of 8 up to 64 run kernels compiled for
// that rank (loop bounds, strides and shared-memory offsets constant: alpha
// pass -27% at R = 10); other ranks the generic kernels with CB = 32.
using RankList = std::integer_sequence<int, 1, 2, 3, 4, 5, 6, 7, 8, 9, 10, 11, 12, 13, 14, 15, 16,
                                       24, 32, 40, 48, 56, 64>;
template <int R>
struct RankBlock {
    // above 32 the whole row (R rounded up to 8) in one block, so that a
    // row's non-zeros are walked once per operand
    static constexpr int cb = R <= 8 ? 8 : R <= 16 ? 16 : R <= 32 ? 32 : (R + 7) / 8 * 8;
};

template <class S, int... Rs>
static int allow_rank_kernels(int cap, std::integer_sequence<int, Rs...>) {
    int rc = P2_OK;
    ((rc = rc != P2_OK ? rc
                       : allow_dynamic_smem(k_alpha<RankBlock<Rs>::cb, true, S, Rs>, cap,
                                            "k_alpha")),
     ...);
    ((rc = rc != P2_OK ? rc
                       : allow_dynamic_smem(k_alpha<RankBlock<Rs>::cb, false, S, Rs>, cap,
                                            "k_alpha")),
     ...);
    ((rc = rc != P2_OK ? rc
                       : allow_dynamic_smem(k_beta_p<RankBlock<Rs>::cb, S, S, Rs>, cap,
                                            "k_beta_p")),
     ...);
    return rc;
}

template <int... Rs>
static int allow_rank_stats(int cap, std::integer_sequence<int, Rs...>) {
    int rc = P2_OK;
    ((rc = rc != P2_OK ? rc
                       : allow_dynamic_smem(k_subject_stats_gf<Rs>, cap, "k_subject_stats_gf")),
     ...);
    return rc;
}

template <class S>
static int configure_sparse(int cap) {
    int rc = allow_rank_kernels<S>(cap, RankList{});
    if (rc == P2_OK) rc = allow_dynamic_smem(k_alpha<32, true, S>, cap, "k_alpha");
    if (rc == P2_OK) rc = allow_dynamic_smem(k_alpha<32, false, S>, cap, "k_alpha");
    if (rc == P2_OK) rc = allow_dynamic_smem(k_beta_p<32, S>, cap, "k_beta_p");
    if (rc == P2_OK) rc = allow_dynamic_smem(k_beta_p<8, S, float>, cap, "k_beta_p");
    if (rc == P2_OK) rc = allow_dynamic_smem(k_beta_p<16, S, float>, cap, "k_beta_p");
    if (rc == P2_OK) rc = allow_dynamic_smem(k_beta_p<32, S, float>, cap, "k_beta_p");
    return rc;
}

int configure_kernels(p2_ctx *c) {
    const int cap = c->geo.smem_optin;
    int rc = P2_OK;
    if (rc == P2_OK) rc = configure_sparse<float>(cap);
    if (rc == P2_OK) rc = configure_sparse<bf16_t>(cap);
    if (rc == P2_OK) rc = allow_rank_stats(cap, RankList{});
    if (rc == P2_OK) rc = polar_configure(c);
    if (rc == P2_OK) rc = allow_dynamic_smem(k_solve_h, cap, "k_solve_h");
    if (rc == P2_OK) rc = allow_dynamic_smem(k_solve_v_pinv, cap, "k_solve_v_pinv");
    if (rc == P2_OK) rc = allow_dynamic_smem(k_fin_v, cap, "k_fin_v");
    if (rc == P2_OK) rc = allow_dynamic_smem(k_subject_stats, cap, "k_subject_stats");
    if (rc == P2_OK) rc = allow_dynamic_smem(k_subject_stats_gf<0>, cap, "k_subject_stats_gf");
    if (rc == P2_OK) rc = allow_dynamic_smem(k_eig_orth, cap, "k_eig_orth");
    if (rc == P2_OK) rc = allow_dynamic_smem(k_eig_ritz<float>, cap, "k_eig_ritz");
    if (rc == P2_OK) rc = allow_dynamic_smem(k_eig_ritz<bf16_t>, cap, "k_eig_ritz");
    if (rc == P2_OK && c->opt.nonneg) {
        const cudaError_t e = nnls_configure(cap);
        if (e != cudaSuccess) {
            set_error("configuring the NNLS kernels: %s", cudaGetErrorString(e));
            rc = P2_ECUDA;
        }
    }
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
    if (!c->opt.timing) return;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    cudaStreamIsCapturing(c->stream, &cs);
    if (cs == cudaStreamCaptureStatusActive)
        cudaEventRecordWithFlags(c->ev[i], c->stream, cudaEventRecordExternal);
    else
        cudaEventRecord(c->ev[i], c->stream);
}

// Gram G_k of Z_k = X_k V for an arbitrary batch X (projection of new
// subjects onto the model's V).
template <int CB, class S, int RT>
static void launch_gram_k(const p2_ctx *c, const XView &X, const SmallState *st, dw *G,
                          cudaStream_t s) {
    const Launch L = plan(c);
    const int nt = L.alpha_warps * 32;
    dim3 grid(c->geo.nsm * resident_blocks(c, k_alpha<CB, false, S, RT>, nt, L.alpha_smem));
    k_alpha<CB, false, S, RT><<<grid, dim3(nt), L.alpha_smem, s>>>(
        X, nullptr, Bufs<S>::V(c), c->d_H, nullptr, st, G, nullptr, nullptr, nullptr, c->R);
}

template <class S, int... Rs>
static void launch_gram_ranks(const p2_ctx *c, const XView &X, const SmallState *st, dw *G,
                              cudaStream_t s, std::integer_sequence<int, Rs...>) {
    bool done = false;
    ((c->R == Rs && !done
          ? (launch_gram_k<RankBlock<Rs>::cb, S, Rs>(c, X, st, G, s), done = true)
          : false),
     ...);
    if (!done) launch_gram_k<32, S, 0>(c, X, st, G, s);
}

template <class S>
static void launch_gram_t(const p2_ctx *c, const XView &X, const SmallState *st, dw *G,
                          cudaStream_t s) {
    launch_gram_ranks<S>(c, X, st, G, s, RankList{});
}

// Gram G_k of Z_k = X_k V for an arbitrary batch X (projection of new
// subjects onto the model's V).
cudaError_t launch_gram(const p2_ctx *c, const XView &X, const SmallState *st, dw *G,
                        cudaStream_t s) {
    if (c->bf16)
        launch_gram_t<bf16_t>(c, X, st, G, s);
    else
        launch_gram_t<float>(c, X, st, G, s);
    return cudaGetLastError();
}

template <int CB, bool MODE3, class S, int RT>
static void launch_alpha_k(p2_ctx *c, const Launch &L, const S *Vprev) {
    const int nt = L.alpha_warps * 32;
    dim3 grid(c->geo.nsm * resident_blocks(c, k_alpha<CB, MODE3, S, RT>, nt, L.alpha_smem));
    k_alpha<CB, MODE3, S, RT><<<grid, dim3(nt), L.alpha_smem, c->stream>>>(
        xview(c), Vprev, Bufs<S>::V(c), c->d_H, c->d_T, c->d_s, c->d_G, c->d_Gf, c->d_W, c->d_M3,
        c->R);
}

template <bool MODE3, class S, int... Rs>
static void launch_alpha_ranks(p2_ctx *c, const Launch &L, const S *Vprev,
                               std::integer_sequence<int, Rs...>) {
    bool done = false;
    ((c->R == Rs && !done
          ? (launch_alpha_k<RankBlock<Rs>::cb, MODE3, S, Rs>(c, L, Vprev), done = true)
          : false),
     ...);
    if (!done) launch_alpha_k<32, MODE3, S, 0>(c, L, Vprev);
}

template <bool MODE3, class S>
static void launch_alpha_t(p2_ctx *c, const Launch &L, const S *Vprev) {
    launch_alpha_ranks<MODE3, S>(c, L, Vprev, RankList{});
}

// pass alpha: with MODE3 Z_k from Vprev and Z'_k from V (the iteration), else
// the Gram of Z_k = X_k V only (prologue)
template <bool MODE3>
static void launch_alpha(p2_ctx *c, const Launch &L) {
    if (c->bf16)
        launch_alpha_t<MODE3, bf16_t>(c, L, MODE3 ? c->d_Vprevh : nullptr);
    else
        launch_alpha_t<MODE3, float>(c, L, MODE3 ? c->d_Vprev : nullptr);
}

// Mode-2 rows of row block b (its subjects, P rows relative to the block's
// first row, into the P buffer that holds one block); one block: the whole
// collection, in the subject order of xview.
template <int CB, class S, int RT>
static void launch_beta_k(p2_ctx *c, const Launch &L, int b) {
    const int nt = L.beta_warps * 32;
    XView X = xview(c);
    int64_t row0 = 0, k0 = 0;
    if (c->X.nblk > 1) {
        k0 = c->X.blk_subj[b];
        X.subj_row += k0;
        X.subj_nnz += k0;
        X.K = c->X.blk_subj[b + 1] - k0;
        X.order = nullptr;
        row0 = c->X.blk_row[b];
    }
    const int64_t want = (X.K + L.beta_warps - 1) / L.beta_warps;
    const int64_t full = (int64_t)c->geo.nsm * resident_blocks(c, k_beta_p<CB, S, S, RT>, nt, L.beta_smem);
    dim3 grid((unsigned)std::max<int64_t>(1, std::min(want, full)));
    k_beta_p<CB, S, S, RT><<<grid, dim3(nt), L.beta_smem, c->stream>>>(
        X, Bufs<S>::V(c), c->d_H, c->d_T + (size_t)k0 * c->R * c->R, c->d_W + (size_t)k0 * c->R,
        Bufs<S>::P(c), c->R, row0, v_stride<S>(c->R));
}

template <class S, int... Rs>
static void launch_beta_ranks(p2_ctx *c, const Launch &L, int b, std::integer_sequence<int, Rs...>) {
    bool done = false;
    ((c->R == Rs && !done ? (launch_beta_k<RankBlock<Rs>::cb, S, Rs>(c, L, b), done = true)
                              : false),
     ...);
    if (!done) launch_beta_k<32, S, 0>(c, L, b);
}

template <class S>
static void launch_beta_p_t(p2_ctx *c, const Launch &L, int b) {
    launch_beta_ranks<S>(c, L, b, RankList{});
}

// mode-1 statistics (k_subject_stats_gf) compiled for the rank when it is in RankList
template <int... Rs>
static void launch_stats_ranks(p2_ctx *c, int nb, int nt, size_t ssm, int with_fit,
                               std::integer_sequence<int, Rs...>) {
    bool done = false;
    ((c->R == Rs && !done
          ? (k_subject_stats_gf<Rs><<<nb, nt, ssm, c->stream>>>(
                 c->d_T, c->d_Gf, c->d_W, c->d_M3, c->d_part, c->X.K, c->R, with_fit),
             done = true)
          : false),
     ...);
    if (!done)
        k_subject_stats_gf<0><<<nb, nt, ssm, c->stream>>>(c->d_T, c->d_Gf, c->d_W, c->d_M3,
                                                          c->d_part, c->X.K, c->R, with_fit);
}

static void launch_beta_p(p2_ctx *c, const Launch &L, int b) {
    if (c->bf16)
        launch_beta_p_t<bf16_t>(c, L, b);
    else
        launch_beta_p_t<float>(c, L, b);
}

// U rows of subjects k0 .. k1-1 (rows r0 .. of the stacked order) into the
// FP32 device buffer U: U_k = Z_k T_k^T H, the beta kernel with S_k = I.
template <class S>
static void launch_get_u_t(p2_ctx *c, const Launch &L, int64_t k0, int64_t k1, int64_t r0,
                           float *U) {
    const int nt = L.beta_warps * 32;
    XView X = xview(c);
    X.subj_row += k0;
    X.subj_nnz += k0;
    X.K = k1 - k0;
    X.order = nullptr;
    const S *V = Bufs<S>::V(c);
    const float *T = c->d_T + (size_t)k0 * c->R * c->R;
    const int64_t want = (k1 - k0 + L.beta_warps - 1) / L.beta_warps;
    switch (comp_block(c->R)) {
        case 8: {
            const int g = (int)std::min<int64_t>(want, c->geo.nsm * resident_blocks(c, k_beta_p<8, S, float>, nt, L.beta_smem));
            k_beta_p<8, S, float><<<g, nt, L.beta_smem, c->stream>>>(X, V, c->d_H, T, nullptr, U, c->R, r0, c->R);
            break;
        }
        case 16: {
            const int g = (int)std::min<int64_t>(want, c->geo.nsm * resident_blocks(c, k_beta_p<16, S, float>, nt, L.beta_smem));
            k_beta_p<16, S, float><<<g, nt, L.beta_smem, c->stream>>>(X, V, c->d_H, T, nullptr, U, c->R, r0, c->R);
            break;
        }
        default: {
            const int g = (int)std::min<int64_t>(want, c->geo.nsm * resident_blocks(c, k_beta_p<32, S, float>, nt, L.beta_smem));
            k_beta_p<32, S, float><<<g, nt, L.beta_smem, c->stream>>>(X, V, c->d_H, T, nullptr, U, c->R, r0, c->R);
            break;
        }
    }
}

cudaError_t launch_get_u(p2_ctx *c, int64_t k0, int64_t k1, int64_t r0, float *U) {
    if (k1 <= k0) return cudaSuccess;
    const Launch L = plan(c);
    if (c->bf16)
        launch_get_u_t<bf16_t>(c, L, k0, k1, r0, U);
    else
        launch_get_u_t<float>(c, L, k0, k1, r0, U);
    return cudaGetLastError();
}

// Mode-2 segment partials of row block b (segments blk_seg[b] .. blk_seg[b+1]).
template <class S>
static void launch_m2_segments_t(p2_ctx *c, int b) {
    const int64_t sg0 = c->X.blk_seg[b], sg1 = c->X.blk_seg[b + 1];
    if (sg1 <= sg0) return;
    const int64_t want = (sg1 - sg0 + 7) / 8;
    const int sb = (int)(want < 64 * (int64_t)c->geo.nsm ? want : 64 * (int64_t)c->geo.nsm);
    const S *P = Bufs<S>::P(c);
    const int64_t row0 = c->X.nblk > 1 ? c->X.blk_row[b] : 0;
    switch (comp_block(c->R)) {
        case 8:
            k_m2_segments<8, S><<<sb, 256, 0, c->stream>>>(c->X.csc_row, c->X.csc_val, c->X.seg_start,
                                                           c->X.seg_end, sg0, sg1, P, row0,
                                                           c->d_segpart, c->R);
            break;
        case 16:
            k_m2_segments<16, S><<<sb, 256, 0, c->stream>>>(c->X.csc_row, c->X.csc_val, c->X.seg_start,
                                                            c->X.seg_end, sg0, sg1, P, row0,
                                                            c->d_segpart, c->R);
            break;
        default:
            k_m2_segments<32, S><<<sb, 256, 0, c->stream>>>(c->X.csc_row, c->X.csc_val, c->X.seg_start,
                                                            c->X.seg_end, sg0, sg1, P, row0,
                                                            c->d_segpart, c->R);
            break;
    }
}

static void launch_m2_segments(p2_ctx *c, int b) {
    if (c->bf16)
        launch_m2_segments_t<bf16_t>(c, b);
    else
        launch_m2_segments_t<float>(c, b);
}

// The mode-2 pass's kernels, row block by row block: each block's P rows are
// written and then read back while they are in L2.
static int enqueue_mode2_blocks(p2_ctx *c, const Launch &L) {
    for (int b = 0; b < c->X.nblk; ++b) {
        launch_beta_p(c, L, b);
        P2_LAUNCH_CHECK("k_beta_p");
        if (c->X.blk_seg[b + 1] > c->X.blk_seg[b]) {
            launch_m2_segments(c, b);
            P2_LAUNCH_CHECK("k_m2_segments");
        }
    }
    return P2_OK;
}

// Q-step for the current (H, V, W) (Algorithm 2's SVD loop), then the
// per-subject statistics that need it: mode-1 MTTKRP partials, W^TW,
// max |W|, <W, M3>, and (with_fit) the loss of the completed iteration.
static int enqueue_qstep(p2_ctx *c, int with_fit) {
    const int R = c->R;
    cudaStream_t s = c->stream;
    const int nb = c->geo.red_blocks;
    const int64_t K = c->X.K;
    mark(c, 4);
    {
        cudaError_t e = launch_polar(c);
        if (e != cudaSuccess) {
            set_error("launch of the Procrustes kernel failed: %s", cudaGetErrorString(e));
            return P2_ECUDA;
        }
        c->enqueued += polar_launches(c);
    }
    mark(c, 5);
    const int P = R * (R + 1) / 2;
    const size_t cta = (2 * (size_t)P + 15) & ~(size_t)15;
    int nw = 16;                            // up to 16 warps (k_subject_stats_gf's bound)
    const size_t scap = (size_t)c->geo.smem_optin - 16 * sizeof(double) - 16 * P2_RMAX * sizeof(float);
    while (nw > 1 && cta + nw * stats_warp_bytes(R) > scap) --nw;
    const size_t ssm = cta + nw * stats_warp_bytes(R);
    launch_stats_ranks(c, nb, nw * 32, ssm, with_fit, RankList{});
    P2_LAUNCH_CHECK("k_subject_stats");
    mark(c, 6);
    if (c->xfn) {
        // sharded: this shard's statistics as one row, summed over the shards
        const int64_t stride = (int64_t)stats_part_stride(R);
        k_part_rows_sum<<<(int)((stride + 255) / 256), 256, 0, s>>>(c->d_part, nb, stride,
                                                                  c->d_red);
        P2_LAUNCH_CHECK("k_part_rows_sum");
        const int xrc = exchange(c, c->d_red, stride);
        if (xrc != P2_OK) return xrc;
        k_fin_w<<<1, 256, 0, s>>>(c->d_red, 1, c->d_s, R, with_fit);
    } else {
        k_fin_w<<<1, 256, 0, s>>>(c->d_part, nb, c->d_s, R, with_fit);
    }
    P2_LAUNCH_CHECK("k_fin_w");
    return P2_OK;
}

int enqueue_factor_stats(p2_ctx *c) {
    const int R = c->R;
    cudaStream_t s = c->stream;
    const int nb = c->geo.red_blocks;
    k_init_h<<<1, 256, 0, s>>>(c->d_H, c->d_s, R);
    P2_LAUNCH_CHECK("k_init_h");
    if (c->bf16)
        k_gram_v<bf16_t><<<nb, 256, 0, s>>>(c->d_Vh, c->d_part2, c->X.J, R);
    else
        k_gram_v<float><<<nb, 256, 0, s>>>(c->d_V, c->d_part2, c->X.J, R);
    P2_LAUNCH_CHECK("k_gram_v");
    k_fin_v<<<1, 256, (size_t)2 * R * R * 8, s>>>(c->d_part2, nb, c->d_s, R, 0);
    P2_LAUNCH_CHECK("k_fin_v");
    return P2_OK;
}

int enqueue_prologue(p2_ctx *c) {
    const Launch L = plan(c);
    launch_alpha<false>(c, L);
    P2_LAUNCH_CHECK("k_alpha<false>");
    return enqueue_qstep(c, 0);
}

// Autotuner trials.
template <class F>
static int tune_time(p2_ctx *c, int reps, float *ms, F &&enqueue) {
    cudaEvent_t a = nullptr, b = nullptr;
    P2_CUDA_TRY(cudaEventCreate(&a));
    cudaError_t e = cudaEventCreate(&b);
    if (e != cudaSuccess) {
        cudaEventDestroy(a);
        P2_CUDA_TRY(e);
    }
    float best = -1.f;
    int rc = P2_OK;
    for (int r = 0; r < reps && rc == P2_OK; ++r) {
        cudaEventRecord(a, c->stream);
        rc = enqueue();
        cudaEventRecord(b, c->stream);
        e = cudaEventSynchronize(b);
        float t = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&t, a, b);
        if (e != cudaSuccess && rc == P2_OK) {
            set_error("autotuner timing: %s", cudaGetErrorString(e));
            rc = P2_ECUDA;
        }
        if (rc == P2_OK && (best < 0.f || t < best)) best = t;
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    *ms = best;
    return rc;
}

int tune_time_qstep(p2_ctx *c, int reps, float *ms) {
    return tune_time(c, reps, ms, [c]() -> int {
        const cudaError_t e = launch_polar(c);
        if (e != cudaSuccess) {
            set_error("autotuner: Procrustes launch failed: %s", cudaGetErrorString(e));
            return P2_ECUDA;
        }
        c->enqueued += polar_launches(c);
        return P2_OK;
    });
}

int tune_time_mode2(p2_ctx *c, int reps, float *ms) {
    return tune_time(c, reps, ms, [c]() -> int {
        const Launch L = plan(c);
        return enqueue_mode2_blocks(c, L);
    });
}

int enqueue_iteration(p2_ctx *c) {
    const Launch L = plan(c);
    const int R = c->R;
    cudaStream_t s = c->stream;
    const int nsm = c->geo.nsm;
    const int nb = c->geo.red_blocks;
    const int64_t J = c->X.J;
    const size_t sm_pinv = (size_t)4 * R * R * 8;
    // H step (Algorithm 1 line 3 with U = H; mode-1 MTTKRP from the previous pass)
    mark(c, 0);
    k_solve_h<<<1, 256, sm_pinv, s>>>(c->xfn ? c->d_red : c->d_part, c->xfn ? 1 : nb, c->d_s,
                                      c->d_H, R);
    P2_LAUNCH_CHECK("k_solve_h");
    // pass beta: mode-2 MTTKRP
    mark(c, 1);
    {
        const int rc = enqueue_mode2_blocks(c, L);
        if (rc != P2_OK) return rc;
    }
    const int64_t nJR = J * R;
    const int fb = (int)((nJR + 255) / 256 < 4 * nsm ? (nJR + 255) / 256 : 4 * nsm);
    const int cb_blocks = (int)((J + 7) / 8 < 8 * nsm ? (J + 7) / 8 : 8 * nsm);
    k_m2_columns<<<cb_blocks, 256, 0, s>>>(c->d_segpart, c->X.col_seg, c->d_M2, (int32_t)J,
                                           c->X.nblk, R);
    P2_LAUNCH_CHECK("k_m2_columns");
    {                                           // sharded: M2 summed over the shards
        const int xrc = exchange(c, c->d_M2, nJR);
        if (xrc != P2_OK) return xrc;
    }
    // V step (Algorithm 1 line 5)
    mark(c, 2);
    if (c->opt.nonneg) {
        // Section 5.1's variant: V rows by non-negative least squares
        const cudaError_t e = launch_nnls_v(c, c->d_part2, nb);
        if (e != cudaSuccess) {
            set_error("launch of the V NNLS kernels failed: %s", cudaGetErrorString(e));
            return P2_ECUDA;
        }
        c->enqueued += 2;
    } else {
        k_solve_v_pinv<<<1, 256, sm_pinv, s>>>(c->d_s, R);
        P2_LAUNCH_CHECK("k_solve_v_pinv");
        k_solve_v_rows<<<nb, 256, ((size_t)R * R + 256) * 8, s>>>(c->d_M2, c->d_s, c->d_Vun,
                                                                   c->d_part2, J, R);
        P2_LAUNCH_CHECK("k_solve_v_rows");
    }
    k_solve_v_norm<<<1, 64, 0, s>>>(c->d_part2, nb, c->d_s, R);
    P2_LAUNCH_CHECK("k_solve_v_norm");
    if (c->bf16)
        k_solve_v_store<bf16_t><<<fb, 256, 0, s>>>(c->d_Vun, c->d_s, c->d_Vh, c->d_Vprevh, nJR, R);
    else
        k_solve_v_store<float><<<fb, 256, 0, s>>>(c->d_Vun, c->d_s, c->d_V, c->d_Vprev, nJR, R);
    P2_LAUNCH_CHECK("k_solve_v_store");
    if (c->bf16)
        k_gram_v<bf16_t><<<nb, 256, 0, s>>>(c->d_Vh, c->d_part2, J, R);
    else
        k_gram_v<float><<<nb, 256, 0, s>>>(c->d_V, c->d_part2, J, R);
    P2_LAUNCH_CHECK("k_gram_v");
    k_fin_v<<<1, 256, sm_pinv, s>>>(c->d_part2, nb, c->d_s, R, 1);
    P2_LAUNCH_CHECK("k_fin_v");
    // pass alpha: mode-3 MTTKRP + W step (Algorithm 1 line 7) + Gram for the next Q-step
    mark(c, 3);
    launch_alpha<true>(c, L);
    P2_LAUNCH_CHECK("k_alpha<true>");
    if (c->opt.nonneg) {
        // W rows by non-negative least squares over the M3 rows pass alpha wrote
        const cudaError_t e = launch_nnls_w(c);
        if (e != cudaSuccess) {
            set_error("launch of the W NNLS kernel failed: %s", cudaGetErrorString(e));
            return P2_ECUDA;
        }
        c->enqueued += 1;
    }
    // next Q-step (Algorithm 2's SVD loop), mode-1 MTTKRP, W statistics, fit
    int rc = enqueue_qstep(c, 1);
    mark(c, 7);
    return rc;
}

// Rational start pieces (driven by p2_init_eig).
int enqueue_eig_fill(p2_ctx *c) {
    const int64_t n = c->X.K * c->R;
    const int nb = (int)((n + 255) / 256 < 4 * c->geo.nsm ? (n + 255) / 256 : 4 * c->geo.nsm);
    k_eig_fill<<<nb > 0 ? nb : 1, 256, 0, c->stream>>>(c->d_H, c->d_W, c->X.K, c->R);
    P2_LAUNCH_CHECK("k_eig_fill");
    return P2_OK;
}

int enqueue_eig_product(p2_ctx *c, const double *Vd, int b, int CW, double *Z, double *seg,
                        double *Y) {
    const int32_t J = c->X.J;
    const int nsm = c->geo.nsm;
    const int64_t zw = (c->X.K + 7) / 8, sw = (c->X.nseg * CW + 255) / 256,
                  cw = ((int64_t)J * CW + 255) / 256;
    const int zb = (int)(zw < 16 * nsm ? (zw > 0 ? zw : 1) : 16 * nsm);
    const int sb = (int)(sw < 64 * nsm ? (sw > 0 ? sw : 1) : 64 * nsm);
    const int cb = (int)(cw < 8 * nsm ? (cw > 0 ? cw : 1) : 8 * nsm);
    for (int c0 = 0; c0 < b; c0 += CW) {
        const int w = (b - c0) < CW ? (b - c0) : CW;
        k_eig_z<<<zb, 256, 0, c->stream>>>(xview(c), Vd, b, c0, w, Z);
        P2_LAUNCH_CHECK("k_eig_z");
        if (c->X.nseg > 0) {
            k_eig_m2_segments<<<sb, 256, 0, c->stream>>>(c->X.csc_row, c->X.csc_val, c->X.seg_start,
                                                         c->X.seg_end, c->X.nseg, Z, w, seg);
            P2_LAUNCH_CHECK("k_eig_m2_segments");
        }
        k_eig_m2_columns<<<cb, 256, 0, c->stream>>>(seg, c->X.col_seg, J, c->X.nblk, w, Y, b, c0);
        P2_LAUNCH_CHECK("k_eig_m2_columns");
    }
    return P2_OK;
}

int enqueue_eig_orth(p2_ctx *c, const double *Y, const double *Vold, double *Q, int b,
                     double *dist) {
    k_eig_orth<<<1, 256, (size_t)8 * 256 * 8, c->stream>>>(Y, Vold, Q, (int32_t)c->X.J, b, c->R, dist,
                                                           &c->d_s->flags);
    P2_LAUNCH_CHECK("k_eig_orth");
    return P2_OK;
}

int enqueue_eig_ritz(p2_ctx *c, const double *Y, const double *Vd, double *Out, int b,
                     int final_step) {
    const int32_t J = (int32_t)c->X.J;
    const size_t sm = ((size_t)2 * b * b + 8 * 256) * 8;
    if (c->bf16)
        k_eig_ritz<bf16_t><<<1, 256, sm, c->stream>>>(Y, Vd, Out, c->d_Vh, v_stride<bf16_t>(c->R), J,
                                                      b, c->R, final_step, &c->d_s->flags);
    else
        k_eig_ritz<float><<<1, 256, sm, c->stream>>>(Y, Vd, Out, c->d_V, v_stride<float>(c->R), J, b,
                                                     c->R, final_step, &c->d_s->flags);
    P2_LAUNCH_CHECK("k_eig_ritz");
    return P2_OK;
}

}  // namespace p2
