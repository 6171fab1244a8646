// Mode-1 MTTKRP and W^TW from caller-owned device buffers, without any
// device allocation.
//
// Some callers cannot call cudaMalloc at the point where they need this
// reduction: code that runs while a CUDA graph is being captured, real-time
// loops that must not take the allocator's device-wide synchronisation, and
// hosts that hand out all GPU memory from their own arena under a fixed
// budget.  This entry point therefore keeps its scratch (the per-block
// partial sums) in one file-scope __device__ array of fixed size, shared by
// every call on a device.
#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>

#include "p2_internal.cuh"

namespace p2 {

#define P2_NA_BLOCKS 128
#define P2_NA_RMAX 16
#define P2_NA_STRIDE (2 * P2_NA_RMAX * P2_NA_RMAX + P2_NA_RMAX + 1)

// 128 x 529 doubles = 541,696 bytes, held by every GPU that loads the library
static __device__ __align__(256) double g_na_scratch[P2_NA_BLOCKS * P2_NA_STRIDE];

// Host-side copies of the scratch's device address, one per device.  The
// array's name is only a host stand-in: kernels must be given this address.
static std::mutex g_na_mutex;
static double *g_na_ptr[64] = {};

static int na_scratch(int dev, double **out) {
    if (dev < 0 || dev >= 64) {
        set_error("p2_mode1_stats_noalloc: device ordinal %d out of range", dev);
        return P2_EINVAL;
    }
    std::lock_guard<std::mutex> lock(g_na_mutex);
    if (!g_na_ptr[dev]) {
        void *ptr = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&ptr, g_na_scratch);
        if (e != cudaSuccess || !ptr) {
            set_error("p2_mode1_stats_noalloc: cudaGetSymbolAddress failed: %s",
                      cudaGetErrorString(e));
            return P2_ECUDA;
        }
        g_na_ptr[dev] = (double *)ptr;
    }
    *out = g_na_ptr[dev];
    return P2_OK;
}

// Sums the block partials in block order: M1 and W^TW (both R x R, FP64).
__global__ void k_na_sum(const double *__restrict__ part, int nparts, int R, double *M1,
                         double *WtW) {
    const size_t stride = stats_part_stride(R);
    for (int e = threadIdx.x; e < R * R; e += blockDim.x) {
        double m = 0.0, w = 0.0;
        for (int b = 0; b < nparts; ++b) {
            m += part[(size_t)b * stride + e];
            w += part[(size_t)b * stride + R * R + e];
        }
        M1[e] = m;
        if (WtW) WtW[e] = w;
    }
}

}  // namespace p2

using namespace p2;

extern "C" int p2_mode1_stats_noalloc(int64_t K, int32_t R, const float *T, const double *G,
                                      const float *W, double *M1, double *WtW, void *stream) {
    if (K < 0) return set_error("p2_mode1_stats_noalloc: K < 0"), P2_EINVAL;
    if (R < 1 || R > P2_NA_RMAX)
        return set_error("p2_mode1_stats_noalloc: R = %d outside [1, %d], the size of its "
                         "fixed scratch", R, P2_NA_RMAX), P2_EINVAL;
    if (!M1 || (K > 0 && (!T || !G || !W)))
        return set_error("p2_mode1_stats_noalloc: NULL pointer"), P2_EINVAL;
    int dev = 0;
    P2_CUDA_TRY(cudaGetDevice(&dev));
    double *scratch = nullptr;
    int rc = na_scratch(dev, &scratch);
    if (rc != P2_OK) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    const int P = R * (R + 1) / 2;
    const size_t cta = (2 * (size_t)P + 15) & ~(size_t)15;
    const int nw = 4;                                   // 4 warps: under the 48 KB default
    const size_t smem = cta + nw * stats_warp_bytes(R);
    // every block writes its whole partial slot, so nothing needs clearing
    k_subject_stats<<<P2_NA_BLOCKS, nw * 32, smem, s>>>(T, G, W, nullptr, scratch, K, R, 0);
    P2_CUDA_TRY(cudaGetLastError());
    k_na_sum<<<1, 256, 0, s>>>(scratch, P2_NA_BLOCKS, R, M1, WtW);
    P2_CUDA_TRY(cudaGetLastError());
    return P2_OK;
}
