// M' = H' S' G' S' H'^T of the Procrustes step (Section 3.2: the matrix whose
// eigen-decomposition gives the polar factor of A_k = X_k V S_k H^T) for every
// subject, on the fifth-generation tensor cores.
//
// The Procrustes kernels form M' in double-word arithmetic on the FP32 pipe
// (~2^-46 normwise), 3 R^3 flops per subject.  Here the two products U =
// B' H'^T and M' = H' U (B' = S' G' S') run as bf16 MMAs with FP32
// accumulation in tensor memory, made exact by splitting (the Ozaki scheme:
// Ozaki, Ogita, Oishi and Rump, "Error-free transformations of matrix
// multiplication by using fast routines of matrix multiplication and its
// applications", Numer. Algorithms 59, 2012; Ootomo, Ozaki and Yokota, "DGEMM
// on integer matrix multiplication unit", IJHPCA 2024, for the integer-slice
// form on tensor cores):
//   * every row of an operand is scaled by a power of two 2^-E_row so that
//     its largest entry is below 1, and written as seven balanced base-256
//     digits, x = 2^(E+1) sum_s sigma_s 2^(-8s), |sigma_s| <= 129 (56 bits:
//     more than the 48 of a double-word); each digit is an integer that bf16
//     holds exactly;
//   * a product of two digit matrices is then a sum of integer products below
//     2^24 in magnitude (7 digit pairs x R <= 48 terms x 129 x 128 < 2^23),
//     which FP32 accumulation adds without rounding; the pairs with the same
//     weight (level d = s + t, d = 2 .. 8) share one accumulator;
//   * the seven level sums are read back and added in double-word arithmetic
//     with their weights.  The pairs with s + t > 8 are dropped: an error below
//     ~2^-48 of the row maxima's product per entry, of the order of the
//     double-word rounding.
// The scalings are those of the Procrustes kernels (G' = G 2^sg, S' = S 2^sw,
// H' = H 2^sh), so the kernels that read M' continue exactly as if they had
// formed it.
//
// One CTA of 256 threads per SM: the MMA's M = 128 rows hold Q = floor(128 /
// R) subjects' rows (row m = subject q, row i), N = K = R rounded up to 16;
// threads m and m + 128 prepare the two halves of row m of the A operand and
// read the two halves of lane m of the accumulators.  The H' digits (the B operand of both products) stay in
// shared memory for the CTA's lifetime.  Operands K-major without swizzle.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>

#include "p2_internal.cuh"
#include "p2_dw.cuh"
#include "p2_tc.cuh"

namespace p2 {

namespace {

constexpr int TC_DIGITS = 7;       // base-256 digits per value
constexpr int TC_LEVELS = 7;       // accumulators for the weights d = 2 .. 8
constexpr int TC_ROWS = 128;       // M of every MMA
constexpr int TC_THREADS = 256;    // two threads per row of the A operand
constexpr uint32_t TC_WAIT_LIMIT = 1u << 24;   // polls of an MMA completion before giving up

struct TcGeom {
    int R, Np, Q;                  // rank, R rounded up to 16, subjects per MMA
    uint32_t sbo;                  // bytes between 8-row groups of one digit slice
    uint32_t a_slice, b_slice;     // bytes per digit slice of the A and B operands
    uint32_t off_a, off_b, off_u, off_e, off_bar, bytes, ncols;
};

TcGeom tc_geom(int R) {
    TcGeom g{};
    g.R = R;
    g.Np = (R + 15) & ~15;
    g.Q = TC_ROWS / R;
    // the core matrices of an 8-row group follow each other along K (128
    // bytes apart), the groups follow each other
    g.sbo = (uint32_t)(g.Np / 8) * 128u;
    g.a_slice = (uint32_t)(TC_ROWS / 8) * g.sbo;
    g.b_slice = (uint32_t)(g.Np / 8) * g.sbo;
    auto up = [](uint32_t v, uint32_t a) { return (v + a - 1) / a * a; };
    g.off_a = 0;
    g.off_b = up(g.off_a + TC_DIGITS * g.a_slice, 128);
    g.off_u = up(g.off_b + TC_DIGITS * g.b_slice, 16);
    g.off_e = up(g.off_u + (uint32_t)g.Q * R * R * (uint32_t)sizeof(dw), 16);
    g.off_bar = up(g.off_e + 64 * sizeof(int) + 2 * TC_ROWS * sizeof(float), 16);
    g.bytes = g.off_bar + 32;
    const int cols = TC_LEVELS * g.Np;
    g.ncols = cols <= 128 ? 128 : (cols <= 256 ? 256 : 512);
    return g;
}

static __device__ __forceinline__ uint32_t f_bits(float v) {
    return (uint32_t)__float_as_int(v);
}

// The seven digits of x 2^(55 - E) (|x| < 2^E) as bf16 bit patterns, most
// significant first: the six low digits balanced in [-128, 127], the top one
// the remainder (|top| <= 129).  The 56-bit integer is assembled from the
// significands of the two floats with shifts (no conversion instruction),
// and each digit goes back to a float by adding it to 1.5 2^23.
static __device__ __forceinline__ long long tc_fixed(float v, int E) {
    const uint32_t b = f_bits(v);
    const int ex = (int)((b >> 23) & 0xFF);
    if (ex == 0) return 0;                               // zero (subnormals: below 2^(E-56))
    const long long mant = (long long)((b & 0x7FFFFFu) | 0x800000u);
    // v = mant 2^(ex - 150); v 2^(55 - E) = mant 2^(ex - 95 - E)
    const int sh = ex - 95 - E;
    long long y;
    if (sh >= 0)
        y = mant << sh;                                  // sh <= 31 since |v| < 2^E
    else if (sh > -25)
        y = (mant + (1ll << (-sh - 1))) >> (-sh);        // round half up: error <= 2^(E-56)
    else
        y = 0;
    return (b >> 31) ? -y : y;
}
static __device__ __forceinline__ uint32_t tc_small_bits(int d) {
    // d + 1.5 2^23 is exact for |d| < 2^22; subtracting 1.5 2^23 gives d
    const float f = f_sub(__int_as_float(0x4B400000 + d), 12582912.f);
    return f_bits(f) >> 16;
}
static __device__ __forceinline__ void tc_digits(dw x, int E, uint32_t *bits) {
    long long Y = tc_fixed(x.h, E) + tc_fixed(x.l, E);
#pragma unroll
    for (int s = TC_DIGITS - 1; s >= 1; --s) {
        const int d = (int)(signed char)(Y & 0xFF);
        bits[s] = tc_small_bits(d);
        Y = (Y - d) >> 8;
    }
    bits[0] = tc_small_bits((int)Y);
}

// Entries j0 <= j < j1 (j0, j1 multiples of 8) of row `row` of the seven
// digit slices at `base`: entries j < n from x(j) (row exponent E), zero
// above.  Two entries per 32-bit store; the pairs are visited starting at
// one that depends on the row's 8-row group, so that the 32 lanes of a warp
// store to 32 different banks.
template <class F>
static __device__ __forceinline__ void tc_write_row(unsigned char *base, uint32_t slice,
                                                    const TcGeom &g, int row, F x, int n, int E,
                                                    int j0, int j1) {
    const int npairs = (j1 - j0) / 2;
    int p = (row >> 3) % npairs;
#pragma unroll 1
    for (int jj = 0; jj < npairs; ++jj, p = (p + 1 == npairs) ? 0 : p + 1) {
        const int j = j0 + 2 * p;
        uint32_t b0[TC_DIGITS], b1[TC_DIGITS];
        if (j < n) {
            tc_digits(x(j), E, b0);
        } else {
#pragma unroll
            for (int s = 0; s < TC_DIGITS; ++s) b0[s] = 0;
        }
        if (j + 1 < n) {
            tc_digits(x(j + 1), E, b1);
        } else {
#pragma unroll
            for (int s = 0; s < TC_DIGITS; ++s) b1[s] = 0;
        }
        const uint32_t off = tc::kmajor_off(row, j, g.sbo);
#pragma unroll
        for (int s = 0; s < TC_DIGITS; ++s)
            *reinterpret_cast<uint32_t *>(base + s * slice + off) = b0[s] | (b1[s] << 16);
    }
}

// Exponent E with max_j |x_j| < 2^E from the largest high part.
static __device__ __forceinline__ int row_expo(float maxabs) { return f_expo(maxabs) - 126; }

// D_d = sum over digit pairs of weight d of A_s B_t^T for d = 2 .. 8, each
// level into its own Np columns of tensor memory; issued by one thread.
static __device__ __forceinline__ void tc_issue(const TcGeom &g, uint32_t a_addr, uint32_t b_addr,
                                                uint32_t tbase) {
    const uint32_t idesc = tc::idesc_bf16_f32(TC_ROWS, g.Np);
    const int ksteps = g.Np / 16;
#pragma unroll 1
    for (int d = 2; d <= TC_DIGITS + 1; ++d) {
        uint32_t acc = 0;
        const int s_lo = d - TC_DIGITS > 1 ? d - TC_DIGITS : 1;
        const int s_hi = d - 1 < TC_DIGITS ? d - 1 : TC_DIGITS;
#pragma unroll 1
        for (int s = s_lo; s <= s_hi; ++s) {
            const int t = d - s;
#pragma unroll 1
            for (int kk = 0; kk < ksteps; ++kk) {
                const uint64_t ad = tc::smem_desc(a_addr + (s - 1) * g.a_slice + kk * 256u, 128, g.sbo);
                const uint64_t bd = tc::smem_desc(b_addr + (t - 1) * g.b_slice + kk * 256u, 128, g.sbo);
                tc::mma_bf16(tbase + (uint32_t)((d - 2) * g.Np), ad, bd, idesc, acc);
                acc = 1;
            }
        }
    }
}

// sum_d L_d 2^(-8d) 2^e (L_d exact integers below 2^24): the three leading
// levels by TwoSum into the high part, the others (below 2^-40 of the
// leading level's scale) added into the low part, then normalised.
static __device__ __forceinline__ dw tc_recon(const float (*v)[8], int cc, int e) {
    float lo = 0.f;
#pragma unroll
    for (int L = TC_LEVELS - 1; L >= 3; --L) lo = f_fma(v[L][cc], f_pow2(-8 * (L + 2)), lo);
    dw acc = two_sum(f_mul(v[0][cc], f_pow2(-16)), f_mul(v[1][cc], f_pow2(-24)));
    const dw t = two_sum(acc.h, f_mul(v[2][cc], f_pow2(-32)));
    acc = two_sum(t.h, f_add(f_add(t.l, acc.l), lo));
    const int e1 = e / 2, e2 = e - e1;
    return dw_scale(dw_scale(acc, f_pow2(e1)), f_pow2(e2));
}

// Thread 0 waits (bounded) for the MMAs committed to the barrier's current
// phase; every thread returns whether they completed.
static __device__ __forceinline__ bool tc_wait_all(uint64_t *bar, uint32_t &phase, int *fail) {
    if (threadIdx.x == 0) *fail = tc::mbar_wait(bar, phase, TC_WAIT_LIMIT) ? 0 : 1;
    __syncthreads();
    const bool ok = *fail == 0;
    if (ok) phase ^= 1u;
    tc::fence_after_sync();
    return ok;
}

__global__ void __launch_bounds__(TC_THREADS, 1) k_form_m_tc(const dw *__restrict__ G,
                                                             const float *__restrict__ W,
                                                             SmallState *st, dw *Mout, int64_t K,
                                                             TcGeom g) {
    extern __shared__ __align__(128) unsigned char smt[];
    const int R = g.R, P = R * (R + 1) / 2, Np = g.Np, Q = g.Q;
    // two threads per row of the A operand and per accumulator lane (warps w
    // and w + 4 share the lanes 32 (w % 4) ..): `half` selects the columns
    const int tid = threadIdx.x, warp = tid >> 5;
    const int m = tid & (TC_ROWS - 1), half = tid >> 7;
    const int j0 = half * (Np / 2), j1 = j0 + Np / 2;
    unsigned char *Asl = smt + g.off_a;
    unsigned char *Bsl = smt + g.off_b;
    dw *Us = reinterpret_cast<dw *>(smt + g.off_u);
    int *eh = reinterpret_cast<int *>(smt + g.off_e);
    float *rmax = reinterpret_cast<float *>(smt + g.off_e + 64 * sizeof(int));   // [2][128]
    uint64_t *bar = reinterpret_cast<uint64_t *>(smt + g.off_bar);
    uint32_t *tslot = reinterpret_cast<uint32_t *>(smt + g.off_bar + 8);
    int *fail = reinterpret_cast<int *>(smt + g.off_bar + 12);
    int *ehmax = reinterpret_cast<int *>(smt + g.off_bar + 16);
    if (tid == 0) {
        *fail = 0;
        *ehmax = 0;
        tc::mbar_init(bar, 1);
    }
    __syncthreads();
    {
        int e = 0;
        for (int x = tid; x < R * R; x += blockDim.x) e = max(e, f_expo((float)st->H64[x]));
        atomicMax(ehmax, e);
    }
    __syncthreads();
    // the larger of the two halves' row maxima (both threads of a row call it)
    auto row_max = [&](float mine) {
        rmax[half * TC_ROWS + m] = mine;
        __syncthreads();
        const float v = fmaxf(rmax[m], rmax[TC_ROWS + m]);
        __syncthreads();
        return v;
    };
    // B operand: the digits of H' = H 2^(127 - max expo), row r = H' row r
    {
        const float hsc = f_pow2(127 - *ehmax);
        const bool hr = m < Np;
        auto hrow = [&](int j) { return dw{f_mul((float)st->H64[m * R + j], hsc), 0.f}; };
        float mx = 0.f;
        if (m < R)
            for (int j = j0; j < j1 && j < R; ++j) mx = fmaxf(mx, fabsf(hrow(j).h));
        const int E = row_expo(row_max(mx));
        if (hr) {
            if (half == 0) eh[m] = E;
            tc_write_row(Bsl, g.b_slice, g, m, hrow, m < R ? R : 0, E, j0, j1);
        }
    }
    if (warp == 0) {
        tc::tmem_alloc(tslot, g.ncols);
        tc::tmem_relinquish();
    }
    tc::fence_async_smem();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tbase = *tslot;
    const uint32_t tlane = tbase + ((uint32_t)(32 * (warp & 3)) << 16);
    const uint32_t a_addr = tc::smem_addr(Asl), b_addr = tc::smem_addr(Bsl);
    uint32_t phase = 0;
    const int q = m / R, i = m - q * R;
    const int64_t ngroups = (K + Q - 1) / Q;
#pragma unroll 1
    for (int64_t grp = blockIdx.x; grp < ngroups; grp += gridDim.x) {
        const int64_t k = grp * Q + q;
        const bool act = q < Q && k < K;
        // ---- U = B' H'^T: A row m = row i of subject q's B' = S' G' S'
        int EA;
        {
            const float *Wk = W + (size_t)(act ? k : 0) * R;
            const dw *Gk = G + (size_t)(act ? k : 0) * P;
            float gsc = 1.f, wsc = 1.f, wi = 0.f;
            // entry j of row i of B' (recomputed for the digits, not held)
            auto brow = [&](int j) {
                const int p = (j <= i) ? (i * (i + 1) / 2 + j) : (j * (j + 1) / 2 + i);
                return dw_mul(dw_scale(Gk[p], gsc), two_prod(wi, f_mul(Wk[j], wsc)));
            };
            float mx = 0.f;
            if (act) {
                int ew = 0, eg = 0;
                for (int j = 0; j < R; ++j) {
                    ew = max(ew, f_expo(Wk[j]));
                    eg = max(eg, f_expo(Gk[j * (j + 1) / 2 + j].h));
                }
                gsc = f_pow2(127 - eg);
                wsc = f_pow2(127 - ew);
                wi = f_mul(Wk[i], wsc);
                for (int j = j0; j < j1 && j < R; ++j) mx = fmaxf(mx, fabsf(brow(j).h));
            }
            EA = row_expo(row_max(mx));
            tc_write_row(Asl, g.a_slice, g, m, brow, act ? R : 0, EA, j0, j1);
        }
        tc::fence_async_smem();
        tc::fence_before_sync();
        __syncthreads();
        tc::fence_after_sync();
        if (tid == 0) {
            tc_issue(g, a_addr, b_addr, tbase);
            tc::mma_commit(bar);
        }
        if (!tc_wait_all(bar, phase, fail)) break;
        // lane m holds row i of subject q's U in each level's columns
#pragma unroll 1
        for (int c0 = j0; c0 < j1; c0 += 8) {
            float v[TC_LEVELS][8];
#pragma unroll
            for (int L = 0; L < TC_LEVELS; ++L) tc::tmem_ld8(tlane + (uint32_t)(L * Np + c0), v[L]);
            tc::tmem_wait_ld();
            if (act) {
#pragma unroll
                for (int cc = 0; cc < 8; ++cc) {
                    const int c = c0 + cc;
                    if (c < R) Us[(q * R + i) * R + c] = tc_recon(v, cc, EA + eh[c] + 2);
                }
            }
        }
        tc::fence_before_sync();
        __syncthreads();
        // ---- M' = H' U: A row m = column c = i of subject q's U
        int EC;
        {
            auto ucol = [&](int r) { return Us[(q * R + r) * R + i]; };
            float mx = 0.f;
            if (act)
                for (int r = j0; r < j1 && r < R; ++r) mx = fmaxf(mx, fabsf(ucol(r).h));
            EC = row_expo(row_max(mx));
            tc_write_row(Asl, g.a_slice, g, m, ucol, act ? R : 0, EC, j0, j1);
        }
        tc::fence_async_smem();
        tc::fence_before_sync();
        __syncthreads();
        tc::fence_after_sync();
        if (tid == 0) {
            tc_issue(g, a_addr, b_addr, tbase);
            tc::mma_commit(bar);
        }
        if (!tc_wait_all(bar, phase, fail)) break;
        // lane m holds M'(r, c) for c = i, all r: the lower triangle r >= c
        // goes out, packed row by row
#pragma unroll 1
        for (int c0 = j0; c0 < j1; c0 += 8) {
            float v[TC_LEVELS][8];
#pragma unroll
            for (int L = 0; L < TC_LEVELS; ++L) tc::tmem_ld8(tlane + (uint32_t)(L * Np + c0), v[L]);
            tc::tmem_wait_ld();
            if (act) {
                dw *Mk = Mout + (size_t)k * P;
#pragma unroll
                for (int cc = 0; cc < 8; ++cc) {
                    const int r = c0 + cc;
                    if (r < R && r >= i) Mk[r * (r + 1) / 2 + i] = tc_recon(v, cc, EC + eh[r] + 2);
                }
            }
        }
        tc::fence_before_sync();
        __syncthreads();
    }
    if (*fail) {
        // let MMAs still in flight finish (bounded) before the memory goes
        if (tid == 0) {
            tc::mbar_wait(bar, phase, TC_WAIT_LIMIT);
            atomicOr(&st->flags, FLAG_TC_TIMEOUT);
        }
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    if (warp == 0) tc::tmem_dealloc(tbase, g.ncols);
}

}  // namespace

bool form_m_tc_supported(int R) { return R >= 13 && R <= P2_TC_RMAX; }

cudaError_t form_m_tc_configure(int R) {
    if (!form_m_tc_supported(R)) return cudaSuccess;
    return cudaFuncSetAttribute(k_form_m_tc, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)tc_geom(R).bytes);
}

cudaError_t launch_form_m_tc(const p2_ctx *c, const dw *G, const float *W, SmallState *st,
                             dw *Mout, int64_t K, cudaStream_t s) {
    const int R = c->R;
    if (K <= 0) return cudaSuccess;
    if (!form_m_tc_supported(R)) return cudaErrorInvalidValue;
    const TcGeom g = tc_geom(R);
    const int64_t ngroups = (K + g.Q - 1) / g.Q;
    // one CTA per SM: the accumulators take up to all of an SM's tensor memory
    const unsigned grid = (unsigned)std::min<int64_t>(ngroups, c->geo.nsm);
    k_form_m_tc<<<grid, TC_THREADS, g.bytes, s>>>(G, W, st, Mout, K, g);
    return cudaGetLastError();
}

}  // namespace p2
