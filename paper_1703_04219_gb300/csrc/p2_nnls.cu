// Non-negative variant of the CP sweep (Section 5.1: the experiments
// constrain {S_k} and V to be non-negative).  The V and W updates of
// Algorithm 1 become, row by row, the non-negative least-squares problems
//   x = argmin_{x >= 0} x^T A x / 2 - b^T x
// with the Gram-Hadamard product A shared by all rows (A = W^TW * H^TH for
// the rows of V, b = M2(j,:); A = V^TV * H^TH for the rows of W, b =
// M3(k,:)); H stays unconstrained.
//
// One lane per row for R <= 16 (one warp per row above, k_nnls_warp),
// double-word arithmetic (p2_dw.cuh), the active-set method
// of Lawson and Hanson ("Solving Least Squares Problems", 1974, Chapter 23)
// with each subproblem A_PP z_P = b_P solved by a Cholesky factorisation of
// the passive block.  The method starts from the row's passive set of the
// previous iteration (warm start, made feasible by dropping the variables
// whose subproblem solution is not positive); the result does not depend on
// the start because the minimiser is unique for positive definite A.
#include <cuda_runtime.h>
#include <math.h>
#include <stddef.h>
#include <stdint.h>

#include "p2_internal.cuh"
#include "p2_num.cuh"

#define FULLMASK_NNLS 0xffffffffu

namespace p2 {

// b element as a double-word: FP32 rows (M3) exactly, FP64 rows (M2) split
static __device__ __forceinline__ dw to_dw(float v) { return dw_f(v); }
static __device__ __forceinline__ dw to_dw(double v) {
    const float h = (float)v;
    return dw{h, (float)(v - (double)h)};
}
static __device__ __forceinline__ void store_out(float *p, dw v) { *p = v.h; }
static __device__ __forceinline__ void store_out(double *p, dw v) {
    *p = (double)v.h + (double)v.l;
}

// Double-words per lane: the Cholesky factor of the passive block (packed
// lower), its reciprocal diagonal, the compact intermediate, x, z and b.
template <int R>
__host__ __device__ constexpr int nnls_lane_dws() { return R * (R + 1) / 2 + 5 * R; }

constexpr int NNLS_THREADS = 128;     // threads per block of k_nnls_rows (a constant
                                      // stride: the lanes' entries provably distinct)

template <int R>
size_t nnls_smem(int nt) {
    return (size_t)R * R * sizeof(dw) + (size_t)nt * nnls_lane_dws<R>() * sizeof(dw) +
           (size_t)nt * R;
}

// Rows r of `rows` (n x R, FP32 or FP64) -> out (n x R, FP32 or FP64);
// passive[r] holds the row's passive set (bit j: x_j > 0) in and out.
template <int R, class B, class O>
__global__ void __launch_bounds__(NNLS_THREADS, 1) k_nnls_rows(const double *__restrict__ Xa,
                                                   const double *__restrict__ Xb,
                                                   const B *__restrict__ rows, int64_t n,
                                                   uint64_t *passive, O *out) {
    constexpr int LP = R * (R + 1) / 2;
    constexpr int DWS = nnls_lane_dws<R>();
    extern __shared__ __align__(16) dw sn[];
    constexpr int NT = NNLS_THREADS;
    const int t = threadIdx.x;
    dw *As = sn;                                   // R x R, A = Xa * Xb
    for (int e = t; e < R * R; e += NT) As[e] = to_dw(Xa[e] * Xb[e]);
    __syncthreads();
    float scale_a = 0.f;
    for (int e = 0; e < R * R; ++e) scale_a = fmaxf(scale_a, fabsf(As[e].h));
    dw *lane = sn + R * R + t;
    unsigned char *ix = reinterpret_cast<unsigned char *>(sn + R * R + (size_t)DWS * NT) + t;
    auto S = [lane](int e) -> dw & { return lane[(size_t)e * NT]; };
    auto L = [&](int a, int c) -> dw & { return S(a * (a + 1) / 2 + c); };
    auto RD = [&](int a) -> dw & { return S(LP + a); };
    auto Y = [&](int a) -> dw & { return S(LP + R + a); };
    auto X = [&](int j) -> dw & { return S(LP + 2 * R + j); };
    auto Z = [&](int j) -> dw & { return S(LP + 3 * R + j); };
    auto Bv = [&](int j) -> dw & { return S(LP + 4 * R + j); };
    auto IDX = [ix](int a) -> unsigned char & { return ix[(size_t)a * NT]; };
    const dw zero = dw_f(0.f), one = dw_f(1.f);

    // z_P = A_PP^{-1} b_P (Cholesky), z = 0 off P; returns the mask of the
    // passive variables whose solution is not positive
    auto solve = [&](uint32_t Pm) -> uint32_t {
        int p = 0;
        for (int j = 0; j < R; ++j)
            if (Pm >> j & 1u) IDX(p++) = (unsigned char)j;
        for (int a = 0; a < p; ++a) {
            const int ia = IDX(a);
            for (int c = 0; c <= a; ++c) {
                dwacc s = acc_from(As[ia * R + IDX(c)]);
                for (int q = 0; q < c; ++q) acc_fma(s, dw_neg(L(a, q)), L(c, q));
                const dw sv = acc_val(s);
                if (c < a) {
                    L(a, c) = dw_mul(sv, RD(c));
                } else {
                    const bool ok = sv.h > 0.f;           // A_PP positive definite
                    const dw rt = ok ? dw_rsqrt(sv) : zero;
                    RD(a) = rt;
                    L(a, a) = ok ? dw_mul(sv, rt) : zero;
                }
            }
        }
        for (int a = 0; a < p; ++a) {                    // L y = b_P
            dwacc s = acc_from(Bv(IDX(a)));
            for (int q = 0; q < a; ++q) acc_fma(s, dw_neg(L(a, q)), Y(q));
            Y(a) = dw_mul(acc_val(s), RD(a));
        }
        for (int a = p - 1; a >= 0; --a) {               // L^T z = y, in place
            dwacc s = acc_from(Y(a));
            for (int q = a + 1; q < p; ++q) acc_fma(s, dw_neg(L(q, a)), Y(q));
            Y(a) = dw_mul(acc_val(s), RD(a));
        }
        for (int j = 0; j < R; ++j) Z(j) = zero;
        uint32_t bad = 0;
        for (int a = 0; a < p; ++a) {
            const int j = IDX(a);
            Z(j) = Y(a);
            if (!(Y(a).h > 0.f)) bad |= 1u << j;
        }
        return bad;
    };

    const int64_t nth = (int64_t)gridDim.x * NT;
    for (int64_t r = (int64_t)blockIdx.x * NT + t; r < n; r += nth) {
        float scale = scale_a;
        for (int j = 0; j < R; ++j) {
            const dw bj = to_dw(rows[(size_t)r * R + j]);
            Bv(j) = bj;
            X(j) = zero;
            scale = fmaxf(scale, fabsf(bj.h));
        }
        // dual feasibility: w_j > tol, tol a few double-word roundings of the data
        const float tol = 64.f * (float)R * 1.4210855e-14f * scale;   // 2^-46
        uint32_t P = (uint32_t)(passive[r] & ((1ull << R) - 1ull));
        // warm start: shrink the previous passive set until its solution is positive
        for (int it = 0; it <= R && P; ++it) {
            const uint32_t bad = solve(P);
            if (!bad) {
                for (int j = 0; j < R; ++j) X(j) = Z(j);
                break;
            }
            P &= ~bad;
        }
        // Lawson-Hanson: add the most violated dual constraint, then step
        // towards the subproblem solution until it is positive on P
        for (int outer = 0; outer < 3 * R; ++outer) {
            int jb = -1;
            float wb = tol;
            for (int j = 0; j < R; ++j) {
                if (P >> j & 1u) continue;
                dwacc s = acc_from(Bv(j));
                for (int q = 0; q < R; ++q) acc_fma(s, dw_neg(As[j * R + q]), X(q));
                const float w = acc_val(s).h;
                if (w > wb) {
                    wb = w;
                    jb = j;
                }
            }
            if (jb < 0) break;
            P |= 1u << jb;
            for (int inner = 0; inner <= R; ++inner) {
                const uint32_t bad = solve(P);
                if (!bad) {
                    for (int j = 0; j < R; ++j) X(j) = Z(j);
                    break;
                }
                dw alpha = one;                          // min x_j / (x_j - z_j) over bad
                for (int j = 0; j < R; ++j) {
                    if (!(bad >> j & 1u)) continue;
                    const dw den = dw_sub(X(j), Z(j));
                    const dw a = den.h > 0.f ? dw_div(X(j), den) : zero;
                    if (a.h < alpha.h || (a.h == alpha.h && a.l < alpha.l)) alpha = a;
                }
                for (int j = 0; j < R; ++j) {
                    if (!(P >> j & 1u)) continue;
                    const dw xj = dw_fma(alpha, dw_sub(Z(j), X(j)), X(j));
                    if (xj.h > 0.f) {
                        X(j) = xj;
                    } else {
                        X(j) = zero;
                        P &= ~(1u << j);
                    }
                }
            }
        }
        for (int j = 0; j < R; ++j) store_out(out + (size_t)r * R + j, X(j));
        passive[r] = P;
    }
}

// ---------------------------------------------------------------------------
// 16 < R <= 64: one warp per row.  The same Lawson-Hanson iteration, warm
// start, tolerances and double-word arithmetic as k_nnls_rows, with the
// per-row storage (Cholesky factor of the passive block, packed lower, and
// the vectors) in shared memory once per warp instead of once per lane, and
// the vector work split over the lanes: the left-looking Cholesky factors
// column by column (the rows below the diagonal over the lanes, each lane
// forming its dot products), the triangular solves go column by column (one
// division, then an update of the remaining entries over the lanes), and the
// dual check, the step length and the passive-set updates take one entry per
// lane with warp reductions.  Every lane of a warp ends each step with the
// same passive set, so the warp stays converged.
// ---------------------------------------------------------------------------
__host__ __device__ inline size_t nnls_warp_dws(int R) {
    return (size_t)R * (R + 1) / 2 + 5 * (size_t)R + ((size_t)R + 7) / 8;   // + R index bytes
}
inline size_t nnls_warp_smem(int R, int warps) {
    return (size_t)R * R * sizeof(dw) + (size_t)warps * nnls_warp_dws(R) * sizeof(dw);
}

static __device__ __forceinline__ dw warp_sum_dw(dw v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
        v = dw_add(v, dw{__shfl_xor_sync(FULLMASK_NNLS, v.h, o), __shfl_xor_sync(FULLMASK_NNLS, v.l, o)});
    return v;
}
static __device__ __forceinline__ uint64_t warp_or64(uint64_t v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v |= __shfl_xor_sync(FULLMASK_NNLS, v, o);
    return v;
}

template <class B, class O>
__global__ void __launch_bounds__(256) k_nnls_warp(const double *__restrict__ Xa,
                                                   const double *__restrict__ Xb,
                                                   const B *__restrict__ rows, int64_t n, int R,
                                                   uint64_t *passive, O *out) {
    const int LP = R * (R + 1) / 2;
    extern __shared__ __align__(16) dw snw[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    dw *As = snw;                                  // R x R, A = Xa * Xb
    for (int e = threadIdx.x; e < R * R; e += blockDim.x) As[e] = to_dw(Xa[e] * Xb[e]);
    __syncthreads();
    float scale_a = 0.f;
    for (int e = lane; e < R * R; e += 32) scale_a = fmaxf(scale_a, fabsf(As[e].h));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) scale_a = fmaxf(scale_a, __shfl_xor_sync(FULLMASK_NNLS, scale_a, o));
    dw *ws = snw + (size_t)R * R + (size_t)warp * nnls_warp_dws(R);
    dw *Lp = ws;                                   // packed lower factor
    dw *RDv = Lp + LP;                             // reciprocal diagonal
    dw *Yv = RDv + R;
    dw *Xv = Yv + R;
    dw *Zv = Xv + R;
    dw *Bvv = Zv + R;
    unsigned char *IX = reinterpret_cast<unsigned char *>(Bvv + R);
    auto L = [Lp](int a, int c) -> dw & { return Lp[a * (a + 1) / 2 + c]; };
    const dw zero = dw_f(0.f), one = dw_f(1.f);
    const uint64_t rmask = R >= 64 ? ~0ull : ((1ull << R) - 1ull);

    // z_P = A_PP^{-1} b_P, z = 0 off P; returns the passive variables whose
    // solution is not positive (the same on every lane)
    auto solve = [&](uint64_t Pm) -> uint64_t {
        int p = 0;                                 // IX: the passive indices in order
        for (int j0 = 0; j0 < R; j0 += 32) {
            const int j = j0 + lane;
            const bool in = j < R && ((Pm >> j) & 1ull);
            const unsigned bal = __ballot_sync(FULLMASK_NNLS, in);
            if (in) IX[p + __popc(bal & ((1u << lane) - 1u))] = (unsigned char)j;
            p += __popc(bal);
        }
        __syncwarp();
        for (int c = 0; c < p; ++c) {              // left-looking Cholesky, column c
            const int ic = IX[c];
            acc_t<dw> sd = acc0<dw>();
            for (int q = lane; q < c; q += 32) acc_sqr(sd, L(c, q));
            const dw sq = warp_sum_dw(acc_val(sd));
            const dw sv = dw_sub(As[ic * R + ic], sq);
            const bool ok = sv.h > 0.f;            // A_PP positive definite
            const dw rt = ok ? dw_rsqrt(sv) : zero;
            if (lane == 0) {
                RDv[c] = rt;
                L(c, c) = ok ? dw_mul(sv, rt) : zero;
            }
            for (int a = c + 1 + lane; a < p; a += 32) {
                acc_t<dw> s = acc_from(As[IX[a] * R + ic]);
                for (int q = 0; q < c; ++q) acc_fma(s, dw_neg(L(a, q)), L(c, q));
                L(a, c) = dw_mul(acc_val(s), rt);
            }
            __syncwarp();
        }
        for (int a = lane; a < p; a += 32) Yv[a] = Bvv[IX[a]];
        __syncwarp();
        for (int a = 0; a < p; ++a) {              // L y = b_P, column by column
            const dw ya = dw_mul(Yv[a], RDv[a]);
            __syncwarp();
            if (lane == 0) Yv[a] = ya;
            for (int i = a + 1 + lane; i < p; i += 32) Yv[i] = dw_fma(dw_neg(L(i, a)), ya, Yv[i]);
            __syncwarp();
        }
        for (int a = p - 1; a >= 0; --a) {         // L^T z = y, in place
            const dw za = dw_mul(Yv[a], RDv[a]);
            __syncwarp();
            if (lane == 0) Yv[a] = za;
            for (int q = lane; q < a; q += 32) Yv[q] = dw_fma(dw_neg(L(a, q)), za, Yv[q]);
            __syncwarp();
        }
        for (int j = lane; j < R; j += 32) Zv[j] = zero;
        __syncwarp();
        uint64_t bad = 0;
        for (int a = lane; a < p; a += 32) {
            const int j = IX[a];
            Zv[j] = Yv[a];
            if (!(Yv[a].h > 0.f)) bad |= 1ull << j;
        }
        __syncwarp();
        return warp_or64(bad);
    };

    const int64_t nwarps = (int64_t)gridDim.x * nw;
    for (int64_t r = (int64_t)blockIdx.x * nw + warp; r < n; r += nwarps) {
        float scale = scale_a;
        for (int j = lane; j < R; j += 32) {
            const dw bj = to_dw(rows[(size_t)r * R + j]);
            Bvv[j] = bj;
            Xv[j] = zero;
            scale = fmaxf(scale, fabsf(bj.h));
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) scale = fmaxf(scale, __shfl_xor_sync(FULLMASK_NNLS, scale, o));
        __syncwarp();
        const float tol = 64.f * (float)R * 1.4210855e-14f * scale;   // 2^-46, as k_nnls_rows
        uint64_t P = passive[r] & rmask;
        for (int it = 0; it <= R && P; ++it) {     // warm start
            const uint64_t bad = solve(P);
            if (!bad) {
                for (int j = lane; j < R; j += 32) Xv[j] = Zv[j];
                __syncwarp();
                break;
            }
            P &= ~bad;
        }
        for (int outer = 0; outer < 3 * R; ++outer) {
            // most violated dual constraint (lowest index on ties)
            int jb = -1;
            float wb = tol;
            for (int j = lane; j < R; j += 32) {
                if ((P >> j) & 1ull) continue;
                acc_t<dw> s = acc_from(Bvv[j]);
                for (int q = 0; q < R; ++q) acc_fma(s, dw_neg(As[j * R + q]), Xv[q]);
                const float w = acc_val(s).h;
                if (w > wb) {
                    wb = w;
                    jb = j;
                }
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                const float w2 = __shfl_xor_sync(FULLMASK_NNLS, wb, o);
                const int j2 = __shfl_xor_sync(FULLMASK_NNLS, jb, o);
                if (j2 >= 0 && (jb < 0 || w2 > wb || (w2 == wb && j2 < jb))) {
                    wb = w2;
                    jb = j2;
                }
            }
            if (jb < 0) break;
            P |= 1ull << jb;
            for (int inner = 0; inner <= R; ++inner) {
                const uint64_t bad = solve(P);
                if (!bad) {
                    for (int j = lane; j < R; j += 32) Xv[j] = Zv[j];
                    __syncwarp();
                    break;
                }
                dw alpha = one;                    // min x_j / (x_j - z_j) over bad
                for (int j = lane; j < R; j += 32) {
                    if (!((bad >> j) & 1ull)) continue;
                    const dw den = dw_sub(Xv[j], Zv[j]);
                    const dw a = den.h > 0.f ? dw_div(Xv[j], den) : zero;
                    if (a.h < alpha.h || (a.h == alpha.h && a.l < alpha.l)) alpha = a;
                }
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) {
                    const dw a2{__shfl_xor_sync(FULLMASK_NNLS, alpha.h, o),
                                __shfl_xor_sync(FULLMASK_NNLS, alpha.l, o)};
                    if (a2.h < alpha.h || (a2.h == alpha.h && a2.l < alpha.l)) alpha = a2;
                }
                uint64_t drop = 0;
                for (int j = lane; j < R; j += 32) {
                    if (!((P >> j) & 1ull)) continue;
                    const dw xj = dw_fma(alpha, dw_sub(Zv[j], Xv[j]), Xv[j]);
                    if (xj.h > 0.f) {
                        Xv[j] = xj;
                    } else {
                        Xv[j] = zero;
                        drop |= 1ull << j;
                    }
                }
                __syncwarp();
                P &= ~warp_or64(drop);
            }
        }
        for (int j = lane; j < R; j += 32) store_out(out + (size_t)r * R + j, Xv[j]);
        if (lane == 0) passive[r] = P;
        __syncwarp();
    }
}

// Column sums of squares of V's unnormalised rows into fixed per-block
// partials (the layout k_solve_v_norm reads).
__global__ void __launch_bounds__(256) k_colsumsq(const double *__restrict__ Vun, int64_t J,
                                                  int R, double *part) {
    __shared__ double red[256];
    const int64_t per = (J + gridDim.x - 1) / gridDim.x;
    const int64_t j0 = (int64_t)blockIdx.x * per;
    const int64_t j1 = (j0 + per < J) ? (j0 + per) : J;
    for (int s = 0; s < R; ++s) {
        double acc = 0.0;
        for (int64_t j = j0 + threadIdx.x; j < j1; j += blockDim.x) {
            const double v = Vun[(size_t)j * R + s];
            acc = fma(v, v, acc);
        }
        red[threadIdx.x] = acc;
        __syncthreads();
        for (int o = blockDim.x / 2; o > 0; o >>= 1) {
            if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
            __syncthreads();
        }
        if (threadIdx.x == 0) part[(size_t)blockIdx.x * R + s] = red[0];
        __syncthreads();
    }
}

template <int R, class B, class O>
static cudaError_t launch_nnls_t(const p2_ctx *c, const double *Xa, const double *Xb,
                                 const B *rows, int64_t n, uint64_t *passive, O *out,
                                 cudaStream_t s) {
    const int nt = NNLS_THREADS;
    const size_t smem = nnls_smem<R>(nt);
    const int64_t want = (n + nt - 1) / nt;
    const int64_t cap = (int64_t)c->geo.nsm * 8;
    const int grid = (int)(want < cap ? (want > 0 ? want : 1) : cap);
    k_nnls_rows<R, B, O><<<grid, nt, smem, s>>>(Xa, Xb, rows, n, passive, out);
    return cudaGetLastError();
}

template <class B, class O>
static cudaError_t launch_nnls(const p2_ctx *c, const double *Xa, const double *Xb,
                               const B *rows, int64_t n, uint64_t *passive, O *out,
                               cudaStream_t s) {
    switch (c->R) {
#define P2_NNLS_CASE(r) \
        case r: return launch_nnls_t<r, B, O>(c, Xa, Xb, rows, n, passive, out, s);
        P2_NNLS_CASE(1) P2_NNLS_CASE(2) P2_NNLS_CASE(3) P2_NNLS_CASE(4) P2_NNLS_CASE(5)
        P2_NNLS_CASE(6) P2_NNLS_CASE(7) P2_NNLS_CASE(8) P2_NNLS_CASE(9) P2_NNLS_CASE(10)
        P2_NNLS_CASE(11) P2_NNLS_CASE(12) P2_NNLS_CASE(13) P2_NNLS_CASE(14) P2_NNLS_CASE(15)
        P2_NNLS_CASE(16)
#undef P2_NNLS_CASE
        default: break;
    }
    if (c->R > P2_RMAX) return cudaErrorInvalidValue;
    const int warps = 8;
    const size_t smem = nnls_warp_smem(c->R, warps);
    const int64_t want = (n + warps - 1) / warps;
    const int64_t cap = (int64_t)c->geo.nsm * 4;
    const int grid = (int)(want < cap ? (want > 0 ? want : 1) : cap);
    k_nnls_warp<B, O><<<grid, warps * 32, smem, s>>>(Xa, Xb, rows, n, c->R, passive, out);
    return cudaGetLastError();
}

// device address of an R x R member of the small state
static const double *state_member(const p2_ctx *c, size_t off) {
    return reinterpret_cast<const double *>(reinterpret_cast<const char *>(c->d_s) + off);
}

template <class B, class O>
static cudaError_t allow_nnls(int cap) {
    cudaError_t e = cudaSuccess;
#define P2_NNLS_ALLOW(r)                                                                       \
    if (e == cudaSuccess && nnls_smem<r>(128) <= (size_t)cap)                                  \
        e = cudaFuncSetAttribute(k_nnls_rows<r, B, O>, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                                 (int)nnls_smem<r>(128));
    P2_NNLS_ALLOW(1) P2_NNLS_ALLOW(2) P2_NNLS_ALLOW(3) P2_NNLS_ALLOW(4) P2_NNLS_ALLOW(5)
    P2_NNLS_ALLOW(6) P2_NNLS_ALLOW(7) P2_NNLS_ALLOW(8) P2_NNLS_ALLOW(9) P2_NNLS_ALLOW(10)
    P2_NNLS_ALLOW(11) P2_NNLS_ALLOW(12) P2_NNLS_ALLOW(13) P2_NNLS_ALLOW(14) P2_NNLS_ALLOW(15)
    P2_NNLS_ALLOW(16)
#undef P2_NNLS_ALLOW
    return e;
}

cudaError_t nnls_configure(int cap) {
    cudaError_t e = allow_nnls<float, float>(cap);
    if (e == cudaSuccess) e = allow_nnls<double, double>(cap);
    const int need = (int)nnls_warp_smem(P2_RMAX, 8);
    if (e == cudaSuccess && need <= cap)
        e = cudaFuncSetAttribute(k_nnls_warp<float, float>, cudaFuncAttributeMaxDynamicSharedMemorySize, need);
    if (e == cudaSuccess && need <= cap)
        e = cudaFuncSetAttribute(k_nnls_warp<double, double>, cudaFuncAttributeMaxDynamicSharedMemorySize, need);
    return e;
}

// Rows of any FP32 right-hand sides against A = Xa * Xb (device R x R FP64).
cudaError_t launch_nnls_rows(const p2_ctx *c, const double *Xa, const double *Xb,
                             const float *rows, int64_t n, uint64_t *passive, float *out,
                             cudaStream_t s) {
    return launch_nnls<float, float>(c, Xa, Xb, rows, n, passive, out, s);
}

// The model's V^TV and H^TH (the Gram-Hadamard product of the W update).
const double *state_vtv(const p2_ctx *c) { return state_member(c, offsetof(SmallState, VtV)); }
const double *state_hth(const p2_ctx *c) { return state_member(c, offsetof(SmallState, HtH)); }

// W rows: x = NNLS(V^TV * H^TH, M3(k,:)), written over the unconstrained W.
cudaError_t launch_nnls_w(p2_ctx *c) {
    return launch_nnls<float, float>(c, state_member(c, offsetof(SmallState, VtV)),
                                     state_member(c, offsetof(SmallState, HtH)), c->d_M3,
                                     c->X.K, c->d_passW, c->d_W, c->stream);
}

// V rows: Vun = NNLS(W^TW * H^TH, M2(j,:)) and the per-block column sums of
// squares of Vun in part (nparts blocks).
cudaError_t launch_nnls_v(p2_ctx *c, double *part, int nparts) {
    cudaError_t e = launch_nnls<double, double>(c, state_member(c, offsetof(SmallState, WtW)),
                                                state_member(c, offsetof(SmallState, HtH)),
                                                c->d_M2, c->X.J, c->d_passV, c->d_Vun,
                                                c->stream);
    if (e != cudaSuccess) return e;
    k_colsumsq<<<nparts, 256, 0, c->stream>>>(c->d_Vun, c->X.J, c->R, part);
    return cudaGetLastError();
}

}  // namespace p2
