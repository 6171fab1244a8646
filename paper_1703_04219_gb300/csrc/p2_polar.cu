// Procrustes step of the Q-step (Section 3.2, Algorithm 2's SVD loop), FP64,
// one GPU lane per subject.
//
// For subject k with Gram G_k = Z_k^T Z_k (Z_k = X_k V) and S_k = diag(W(k,:)):
//   M   = H S G S H^T                  (= A_k^T A_k, A_k = X_k V S_k H^T)
//   M   = Z diag(d) Z^T                (Householder tridiagonalisation + implicit QR)
//   f_i = d_i^{-1/2} if d_i > rtol^2 max(d) else 0    (rank cut of the SVD)
//   C   = Z diag(f) Z^T                (pseudo-inverse square root of M)
//   T_k = C H S                        (stored FP32; Q_k = X_k V T_k^T)
// The FP64 pipe of this GPU issues one warp instruction per ~66 cycles per
// SM sub-partition whatever the number of active lanes, so every lane owns a
// whole subject and the kernel is written to minimise FP64 instructions.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "p2_internal.cuh"
#include "p2_eig.cuh"
#include "p2_polar.cuh"

namespace p2 {

template <int R>
static __device__ __forceinline__ int pk(int i, int j) {   // packed lower index
    return (j <= i) ? (i * (i + 1) / 2 + j) : (j * (j + 1) / 2 + i);
}

// Small R: Gram and C held in registers, only Z (R x R) and the tridiagonal
// (d, e) in interleaved shared memory: R^2 + 2R doubles per lane.
template <int R>
__global__ void __launch_bounds__(256) k_polar_reg(const double *__restrict__ G,
                                                   const float *__restrict__ W, SmallState *st,
                                                   float *T, int64_t K, double rtol2) {
    constexpr int P = R * (R + 1) / 2;
    extern __shared__ __align__(16) double sm[];
    const int NT = blockDim.x;
    const int t = threadIdx.x;
    double *Hs = sm;
    double *th = sm + R * R;
    for (int i = t; i < R * R; i += NT) Hs[i] = st->H64[i];
    __syncthreads();
    const int64_t k = (int64_t)blockIdx.x * NT + t;
    unsigned long long flops = 0;
    if (k < K) {
        MatView A{th + t, NT, R};
        VecView d{th + (size_t)R * R * NT + t, NT};
        VecView e{th + (size_t)(R * R + R) * NT + t, NT};
        double w[R];
#pragma unroll
        for (int i = 0; i < R; ++i) w[i] = (double)W[(size_t)k * R + i];
        {
            double g[P];
            const double *Gk = G + (size_t)k * P;
#pragma unroll
            for (int i = 0, p = 0; i < R; ++i)
#pragma unroll
                for (int j = 0; j <= i; ++j, ++p) g[p] = Gk[p] * w[i] * w[j];
#pragma unroll 1
            for (int c = 0; c < R; ++c) {
                double tv[R];
#pragma unroll
                for (int i = 0; i < R; ++i) {
                    double s = 0.0;
#pragma unroll
                    for (int j = 0; j < R; ++j) s = fma(g[pk<R>(i, j)], Hs[c * R + j], s);
                    tv[i] = s;
                }
#pragma unroll
                for (int r = c; r < R; ++r) {
                    double s = 0.0;
#pragma unroll
                    for (int i = 0; i < R; ++i) s = fma(Hs[r * R + i], tv[i], s);
                    A(r, c) = s;
                }
            }
        }
        tridiagonalize<R>(R, A, d, e);
        int rot = 0;
        const int steps = tridiagonal_qr<R>(R, A, d, e, 30 * R, &rot);
        if (steps < 0) atomicOr(&st->flags, FLAG_EIG_NOCONV);
        double lmax = 0.0;
#pragma unroll
        for (int i = 0; i < R; ++i) lmax = fmax(lmax, d[i]);
        const double cut = rtol2 * lmax;
#pragma unroll
        for (int i = 0; i < R; ++i) {
            const double di = d[i];
            const double sf = (lmax > 0.0 && di > cut) ? sqrt(p2_rsqrt(di)) : 0.0;   // d^-1/4
#pragma unroll
            for (int r = 0; r < R; ++r) A(r, i) *= sf;
        }
        double Cl[P];
#pragma unroll
        for (int r = 0; r < R; ++r)
#pragma unroll
            for (int c = 0; c <= r; ++c) {
                double s = 0.0;
#pragma unroll
                for (int i = 0; i < R; ++i) s = fma(A(r, i), A(c, i), s);
                Cl[pk<R>(r, c)] = s;
            }
        const size_t tb = (size_t)k * R * R;
#pragma unroll 1
        for (int c = 0; c < R; ++c)
#pragma unroll
            for (int r = 0; r < R; ++r) {
                double s = 0.0;
#pragma unroll
                for (int u = 0; u < R; ++u) s = fma(Cl[pk<R>(r, u)], Hs[u * R + c], s);
                T[tb + r * R + c] = (float)(s * w[c]);
            }
        flops = polar_fixed_flops(R) + qr_flops(R, steps, rot);
    }
    add_flops(st, flops);
}

// Any R: scaled Gram and C in shared memory as well: R^2 + P + 3R doubles per lane.
__global__ void __launch_bounds__(128) k_polar_smem(const double *__restrict__ G,
                                                    const float *__restrict__ W, SmallState *st,
                                                    float *T, int64_t K, int R, double rtol2) {
    extern __shared__ __align__(16) double sm[];
    const int NT = blockDim.x;
    const int t = threadIdx.x;
    const int P = R * (R + 1) / 2;
    double *Hs = sm;
    double *th = sm + R * R;
    for (int i = t; i < R * R; i += NT) Hs[i] = st->H64[i];
    __syncthreads();
    const int64_t k = (int64_t)blockIdx.x * NT + t;
    unsigned long long flops = 0;
    if (k < K) {
        MatView A{th + t, NT, R};
        double *gp = th + (size_t)R * R * NT + t;
        VecView d{gp + (size_t)P * NT, NT};
        VecView e{gp + (size_t)(P + R) * NT, NT};
        VecView w{gp + (size_t)(P + 2 * R) * NT, NT};
        VecView tv = e;
        const float *Wk = W + (size_t)k * R;
        for (int i = 0; i < R; ++i) w[i] = (double)Wk[i];
        const double *Gk = G + (size_t)k * P;
        for (int i = 0, p = 0; i < R; ++i)
            for (int j = 0; j <= i; ++j, ++p) gp[(size_t)p * NT] = Gk[p] * w[i] * w[j];
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
        tridiagonalize<0>(R, A, d, e);
        int rot = 0;
        const int steps = tridiagonal_qr<0>(R, A, d, e, 30 * R, &rot);
        if (steps < 0) atomicOr(&st->flags, FLAG_EIG_NOCONV);
        double lmax = 0.0;
        for (int i = 0; i < R; ++i) lmax = fmax(lmax, d[i]);
        const double cut = rtol2 * lmax;
        for (int i = 0; i < R; ++i) {
            const double di = d[i];
            const double sf = (lmax > 0.0 && di > cut) ? sqrt(p2_rsqrt(di)) : 0.0;
            for (int r = 0; r < R; ++r) A(r, i) *= sf;
        }
        for (int r = 0, p = 0; r < R; ++r)          // C lower into the Gram's slot
            for (int c = 0; c <= r; ++c, ++p) {
                double s = 0.0;
                for (int i = 0; i < R; ++i) s = fma(A(r, i), A(c, i), s);
                gp[(size_t)p * NT] = s;
            }
        const size_t tb = (size_t)k * R * R;
        for (int r = 0; r < R; ++r)
            for (int c = 0; c < R; ++c) {
                double s = 0.0;
                for (int u = 0; u < R; ++u) {
                    const int p = (u <= r) ? (r * (r + 1) / 2 + u) : (u * (u + 1) / 2 + r);
                    s = fma(gp[(size_t)p * NT], Hs[u * R + c], s);
                }
                T[tb + r * R + c] = (float)(s * w[c]);
            }
        flops = polar_fixed_flops(R) + qr_flops(R, steps, rot);
    }
    add_flops(st, flops);
}

template <int R>
static int launch_reg(const p2_ctx *c, const double *G, const float *W, SmallState *st, float *T,
                      int64_t K, cudaStream_t s, double rtol2) {
    const int cap = c->geo.smem_optin;
    const size_t per = (size_t)(R * R + 2 * R) * 8;
    int nt = (int)((cap - (size_t)R * R * 8) / per);
    if (nt > 256) nt = 256;
    nt = (nt / 32) * 32;
    if (nt < 32) return -1;
    const size_t smem = (size_t)R * R * 8 + (size_t)nt * per;
    const int nblk = (int)((K + nt - 1) / nt);
    k_polar_reg<R><<<nblk, nt, smem, s>>>(G, W, st, T, K, rtol2);
    return 0;
}

int polar_configure(p2_ctx *c) {
    const int cap = c->geo.smem_optin;
    cudaError_t e = cudaSuccess;
#define P2_ALLOW(fn) \
    if (e == cudaSuccess) e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, cap)
    P2_ALLOW(k_polar_smem);
    P2_ALLOW(k_polar_reg<2>);
    P2_ALLOW(k_polar_reg<3>);
    P2_ALLOW(k_polar_reg<4>);
    P2_ALLOW(k_polar_reg<5>);
    P2_ALLOW(k_polar_reg<6>);
    P2_ALLOW(k_polar_reg<8>);
    P2_ALLOW(k_polar_reg<10>);
    P2_ALLOW(k_polar_reg<12>);
#undef P2_ALLOW
    if (e == cudaSuccess) e = polar_grp_configure(cap);
    if (e != cudaSuccess) {
        set_error("configuring the Procrustes kernels: %s", cudaGetErrorString(e));
        return P2_ECUDA;
    }
    return P2_OK;
}

// Enqueue the Procrustes kernel for K subjects (Gram G, weights W, state st
// holding H64) writing T; returns a cudaError_t.
cudaError_t launch_polar_on(const p2_ctx *c, const double *G, const float *W, SmallState *st,
                            float *T, int64_t K, cudaStream_t s) {
    const int R = c->R;
    const double rtol2 = c->opt.rank_rtol * c->opt.rank_rtol;
    if (K <= 0) return cudaSuccess;
    int rc = -1;
    switch (R) {
        case 2: rc = launch_reg<2>(c, G, W, st, T, K, s, rtol2); break;
        case 3: rc = launch_reg<3>(c, G, W, st, T, K, s, rtol2); break;
        case 4: rc = launch_reg<4>(c, G, W, st, T, K, s, rtol2); break;
        case 5: rc = launch_reg<5>(c, G, W, st, T, K, s, rtol2); break;
        case 6: rc = launch_reg<6>(c, G, W, st, T, K, s, rtol2); break;
        case 8: rc = launch_reg<8>(c, G, W, st, T, K, s, rtol2); break;
        case 10: rc = launch_reg<10>(c, G, W, st, T, K, s, rtol2); break;
        case 12: rc = launch_reg<12>(c, G, W, st, T, K, s, rtol2); break;
        default: break;
    }
    if (rc != 0 && R > 12) return launch_polar_grp(c, G, W, st, T, K, s, rtol2);
    if (rc != 0) {
        const int P = R * (R + 1) / 2;
        const size_t per = ((size_t)R * R + P + 3 * (size_t)R) * 8;
        int nt = (int)(((size_t)c->geo.smem_optin - (size_t)R * R * 8) / per);
        if (nt > 128) nt = 128;
        if (nt >= 32) nt = (nt / 32) * 32;
        if (nt < 1) nt = 1;
        const size_t smem = (size_t)R * R * 8 + (size_t)nt * per;
        const int nblk = (int)((K + nt - 1) / nt);
        k_polar_smem<<<nblk, nt, smem, s>>>(G, W, st, T, K, R, rtol2);
    }
    return cudaGetLastError();
}

cudaError_t launch_polar(p2_ctx *c) {
    return launch_polar_on(c, c->d_G, c->d_W, c->d_s, c->d_T, c->X.K, c->stream);
}

}  // namespace p2
