// Launch of the grouped Procrustes kernel (R > 12), one instantiation per
// register-array width RB = R rounded up to a multiple of eight, for a number
// type D (double-word or FP64).  Included by p2_polar_grp.cu (double-word)
// and p2_polar_grp_f64.cu (FP64), so the two sets of instances compile in
// parallel.
#pragma once

#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "p2_internal.cuh"
#include "p2_polar.cuh"
#include "p2_polar_grp.cuh"

namespace p2 {


template <class D, int RB, int PG, int RT = 0>
static void launch_grp(const p2_ctx *c, const dw *G, const float *W, SmallState *st, float *T,
                       int64_t K, cudaStream_t s, double rtol2, const int32_t *order,
                       int32_t *qrcnt) {
    const int R = c->R;
    const size_t per = grp_dws(R) * sizeof(dw);
    const size_t hbytes = grp_hdws(R) * sizeof(dw);
    // 16 bytes kept for the kernel's static shared memory
    int spb = (int)(((size_t)c->geo.smem_optin - hbytes - 16) / per);
    const int gpw = 32 / PG;                // subjects per warp
    if (spb > 8 * gpw) spb = 8 * gpw;      // at most 256 threads; a last partial warp idles its spare groups
    if (spb < 1) spb = 1;
    const int threads = ((spb + gpw - 1) / gpw) * 32;
    const size_t smem = hbytes + (size_t)spb * per;
    const int64_t nblk = (K + spb - 1) / spb;
    k_polar_grp<RB, PG, RT, D><<<(unsigned)nblk, threads, smem, s>>>(G, W, st, T, K, R, (float)rtol2, spb,
                                                               order, qrcnt);
}

// dynamic shared memory allowed: the opt-in maximum less the kernel's static
// shared memory
template <class D, int RB, int PG, int RT = 0>
static cudaError_t allow_grp(int cap) {
    cudaFuncAttributes a;
    cudaError_t e = cudaFuncGetAttributes(&a, k_polar_grp<RB, PG, RT, D>);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(k_polar_grp<RB, PG, RT, D>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                cap - (int)a.sharedSizeBytes);
}

// Group width: eight lanes per subject up to R = 32; above, sixteen, which
// doubles the warps that the shared memory (one working matrix per subject)
// allows per SM at the price of running the scalar recurrences on more lanes.
template <class D>
static cudaError_t grp_configure_t(int cap) {
    cudaError_t e = cudaSuccess;
    if (e == cudaSuccess) e = allow_grp<D, 16, 8>(cap);
    if (e == cudaSuccess) e = allow_grp<D, 24, 8>(cap);
    if (e == cudaSuccess) e = allow_grp<D, 32, 8>(cap);
    if (e == cudaSuccess) e = allow_grp<D, 48, 16>(cap);
    if (e == cudaSuccess) e = allow_grp<D, 64, 16>(cap);
    if (e == cudaSuccess) e = allow_grp<D, 16, 8, 13>(cap);
    if (e == cudaSuccess) e = allow_grp<D, 16, 8, 14>(cap);
    if (e == cudaSuccess) e = allow_grp<D, 16, 8, 15>(cap);
    if (e == cudaSuccess) e = allow_grp<D, 16, 8, 16>(cap);
    if (e == cudaSuccess) e = allow_grp<D, 24, 8, 24>(cap);
    if (e == cudaSuccess) e = allow_grp<D, 32, 8, 32>(cap);
    if (e == cudaSuccess) e = allow_grp<D, 48, 16, 40>(cap);
    if (e == cudaSuccess) e = allow_grp<D, 48, 16, 48>(cap);
    if (e == cudaSuccess) e = allow_grp<D, 64, 16, 56>(cap);
    if (e == cudaSuccess) e = allow_grp<D, 64, 16, 64>(cap);
    return e;
}

template <class D>
static cudaError_t launch_grp_t(const p2_ctx *c, const dw *G, const float *W, SmallState *st,
                             float *T, int64_t K, cudaStream_t s, double rtol2,
                             const int32_t *order, int32_t *qrcnt) {
    const int R = c->R;
    // ranks 13 .. 16 and the multiples of 8 run an instance compiled for the
    // rank (loop bounds and offsets constant), the others the generic one
    switch (R) {
        case 13: launch_grp<D, 16, 8, 13>(c, G, W, st, T, K, s, rtol2, order, qrcnt); return cudaGetLastError();
        case 14: launch_grp<D, 16, 8, 14>(c, G, W, st, T, K, s, rtol2, order, qrcnt); return cudaGetLastError();
        case 15: launch_grp<D, 16, 8, 15>(c, G, W, st, T, K, s, rtol2, order, qrcnt); return cudaGetLastError();
        case 16: launch_grp<D, 16, 8, 16>(c, G, W, st, T, K, s, rtol2, order, qrcnt); return cudaGetLastError();
        case 24: launch_grp<D, 24, 8, 24>(c, G, W, st, T, K, s, rtol2, order, qrcnt); return cudaGetLastError();
        case 32: launch_grp<D, 32, 8, 32>(c, G, W, st, T, K, s, rtol2, order, qrcnt); return cudaGetLastError();
        case 40: launch_grp<D, 48, 16, 40>(c, G, W, st, T, K, s, rtol2, order, qrcnt); return cudaGetLastError();
        case 48: launch_grp<D, 48, 16, 48>(c, G, W, st, T, K, s, rtol2, order, qrcnt); return cudaGetLastError();
        case 56: launch_grp<D, 64, 16, 56>(c, G, W, st, T, K, s, rtol2, order, qrcnt); return cudaGetLastError();
        case 64: launch_grp<D, 64, 16, 64>(c, G, W, st, T, K, s, rtol2, order, qrcnt); return cudaGetLastError();
        default: break;
    }
    if (R <= 16)
        launch_grp<D, 16, 8>(c, G, W, st, T, K, s, rtol2, order, qrcnt);
    else if (R <= 24)
        launch_grp<D, 24, 8>(c, G, W, st, T, K, s, rtol2, order, qrcnt);
    else if (R <= 32)
        launch_grp<D, 32, 8>(c, G, W, st, T, K, s, rtol2, order, qrcnt);
    else if (R <= 48)
        launch_grp<D, 48, 16>(c, G, W, st, T, K, s, rtol2, order, qrcnt);
    else
        launch_grp<D, 64, 16>(c, G, W, st, T, K, s, rtol2, order, qrcnt);
    return cudaGetLastError();
}

}  // namespace p2
