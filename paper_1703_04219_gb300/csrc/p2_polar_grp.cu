// Launch of the grouped Procrustes kernel (R > 12), one instantiation per
// register-array width RB = R rounded up to a multiple of eight.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "p2_internal.cuh"
#include "p2_polar.cuh"
#include "p2_polar_grp.cuh"

namespace p2 {

template <int RB, int PG>
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
    k_polar_grp<RB, PG><<<(unsigned)nblk, threads, smem, s>>>(G, W, st, T, K, R, (float)rtol2, spb,
                                                               order, qrcnt);
}

// dynamic shared memory allowed: the opt-in maximum less the kernel's static
// shared memory
template <int RB, int PG>
static cudaError_t allow_grp(int cap) {
    cudaFuncAttributes a;
    cudaError_t e = cudaFuncGetAttributes(&a, k_polar_grp<RB, PG>);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(k_polar_grp<RB, PG>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                cap - (int)a.sharedSizeBytes);
}

// Group width: eight lanes per subject up to R = 32; above, sixteen, which
// doubles the warps that the shared memory (one working matrix per subject)
// allows per SM at the price of running the scalar recurrences on more lanes.
cudaError_t polar_grp_configure(int cap) {
    cudaError_t e = cudaSuccess;
    if (e == cudaSuccess) e = allow_grp<16, 8>(cap);
    if (e == cudaSuccess) e = allow_grp<24, 8>(cap);
    if (e == cudaSuccess) e = allow_grp<32, 8>(cap);
    if (e == cudaSuccess) e = allow_grp<48, 16>(cap);
    if (e == cudaSuccess) e = allow_grp<64, 16>(cap);
    return e;
}

cudaError_t launch_polar_grp(const p2_ctx *c, const dw *G, const float *W, SmallState *st,
                             float *T, int64_t K, cudaStream_t s, double rtol2,
                             const int32_t *order, int32_t *qrcnt) {
    const int R = c->R;
    if (R <= 16)
        launch_grp<16, 8>(c, G, W, st, T, K, s, rtol2, order, qrcnt);
    else if (R <= 24)
        launch_grp<24, 8>(c, G, W, st, T, K, s, rtol2, order, qrcnt);
    else if (R <= 32)
        launch_grp<32, 8>(c, G, W, st, T, K, s, rtol2, order, qrcnt);
    else if (R <= 48)
        launch_grp<48, 16>(c, G, W, st, T, K, s, rtol2, order, qrcnt);
    else
        launch_grp<64, 16>(c, G, W, st, T, K, s, rtol2, order, qrcnt);
    return cudaGetLastError();
}

}  // namespace p2
