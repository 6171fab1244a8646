// Launch of the grouped Procrustes kernel (R > 12), one instantiation per
// register-array width RB = R rounded up to a multiple of eight.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "p2_internal.cuh"
#include "p2_polar.cuh"
#include "p2_polar_grp.cuh"

namespace p2 {

template <int RB>
static void launch_grp(const p2_ctx *c, const dw *G, const float *W, SmallState *st, float *T,
                       int64_t K, cudaStream_t s, double rtol2, const int32_t *order,
                       int32_t *qrcnt) {
    const int R = c->R;
    const size_t per = grp_dws(R) * sizeof(dw);
    const size_t hbytes = grp_hdws(R) * sizeof(dw);
    // 16 bytes kept for the kernel's static shared memory
    int spb = (int)(((size_t)c->geo.smem_optin - hbytes - 16) / per);
    if (spb > 32) spb = 32;                 // four subjects per warp; a last partial warp idles its spare groups
    if (spb < 1) spb = 1;
    const int threads = ((spb + 3) / 4) * 32;
    const size_t smem = hbytes + (size_t)spb * per;
    const int64_t nblk = (K + spb - 1) / spb;
    k_polar_grp<RB><<<(unsigned)nblk, threads, smem, s>>>(G, W, st, T, K, R, (float)rtol2, spb,
                                                           order, qrcnt);
}

// dynamic shared memory allowed: the opt-in maximum less the kernel's static
// shared memory
template <int RB>
static cudaError_t allow_grp(int cap) {
    cudaFuncAttributes a;
    cudaError_t e = cudaFuncGetAttributes(&a, k_polar_grp<RB>);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(k_polar_grp<RB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                cap - (int)a.sharedSizeBytes);
}

cudaError_t polar_grp_configure(int cap) {
    cudaError_t e = cudaSuccess;
    if (e == cudaSuccess) e = allow_grp<16>(cap);
    if (e == cudaSuccess) e = allow_grp<24>(cap);
    if (e == cudaSuccess) e = allow_grp<32>(cap);
    if (e == cudaSuccess) e = allow_grp<40>(cap);
    if (e == cudaSuccess) e = allow_grp<48>(cap);
    if (e == cudaSuccess) e = allow_grp<56>(cap);
    if (e == cudaSuccess) e = allow_grp<64>(cap);
    return e;
}

cudaError_t launch_polar_grp(const p2_ctx *c, const dw *G, const float *W, SmallState *st,
                             float *T, int64_t K, cudaStream_t s, double rtol2,
                             const int32_t *order, int32_t *qrcnt) {
    switch ((c->R + PG - 1) / PG) {
        case 1:
        case 2: launch_grp<16>(c, G, W, st, T, K, s, rtol2, order, qrcnt); break;
        case 3: launch_grp<24>(c, G, W, st, T, K, s, rtol2, order, qrcnt); break;
        case 4: launch_grp<32>(c, G, W, st, T, K, s, rtol2, order, qrcnt); break;
        case 5: launch_grp<40>(c, G, W, st, T, K, s, rtol2, order, qrcnt); break;
        case 6: launch_grp<48>(c, G, W, st, T, K, s, rtol2, order, qrcnt); break;
        case 7: launch_grp<56>(c, G, W, st, T, K, s, rtol2, order, qrcnt); break;
        default: launch_grp<64>(c, G, W, st, T, K, s, rtol2, order, qrcnt); break;
    }
    return cudaGetLastError();
}

}  // namespace p2
