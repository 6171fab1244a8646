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
#include <stdint.h>

#include "p2_internal.cuh"

namespace p2 {

#define P2_NA_BLOCKS 128
#define P2_NA_RMAX 16
#define P2_NA_STRIDE (2 * P2_NA_RMAX * P2_NA_RMAX + P2_NA_RMAX + 1)

// 128 x 529 doubles = 541,696 bytes, held by every GPU that loads the library
static __device__ __align__(256) double g_na_scratch[P2_NA_BLOCKS * P2_NA_STRIDE];

// The array's name is only a host stand-in: kernels must be given its device
// address, looked up on every call for the current device (the lookup
// allocates nothing, and a fresh lookup stays valid after a device reset).
static int na_scratch(double **out) {
    void *ptr = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&ptr, g_na_scratch);
    if (e != cudaSuccess || !ptr) {
        set_error("p2_mode1_stats_noalloc: cudaGetSymbolAddress failed: %s",
                  cudaGetErrorString(e));
        return P2_ECUDA;
    }
    *out = (double *)ptr;
    return P2_OK;
}

// cuMemGetAddressRange from the driver, looked up once (NULL if unavailable):
// the base and size of the allocation that holds a device address.
typedef int (*mem_range_fn)(unsigned long long *, size_t *, unsigned long long);
static mem_range_fn na_range_fn() {
    static std::once_flag once;
    static mem_range_fn fn = nullptr;
    std::call_once(once, [] {
        void *f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuMemGetAddressRange", &f, 12000, cudaEnableDefault,
                                             &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (mem_range_fn)f;
        else
            cudaGetLastError();
    });
    return fn;
}

// A caller buffer must be device (or managed) memory of the current device
// and, where the driver reports the allocation's extent, hold `bytes` bytes.
// Host pointers, pointers of another device and buffers that end past their
// allocation are rejected before anything is enqueued.
static int na_check_buffer(const void *p, size_t bytes, int dev, const char *name) {
    cudaPointerAttributes a;
    cudaError_t e = cudaPointerGetAttributes(&a, p);
    if (e != cudaSuccess) {
        cudaGetLastError();
        set_error("p2_mode1_stats_noalloc: %s is not a CUDA pointer (%s)", name,
                  cudaGetErrorString(e));
        return P2_EINVAL;
    }
    if (a.type != cudaMemoryTypeDevice && a.type != cudaMemoryTypeManaged) {
        set_error("p2_mode1_stats_noalloc: %s is not device memory", name);
        return P2_EINVAL;
    }
    if (a.device != dev) {
        set_error("p2_mode1_stats_noalloc: %s is on device %d, the current device is %d", name,
                  a.device, dev);
        return P2_EINVAL;
    }
    mem_range_fn range = na_range_fn();
    if (range && bytes > 0) {
        unsigned long long base = 0;
        size_t size = 0;
        if (range(&base, &size, (unsigned long long)(uintptr_t)p) == 0) {
            const unsigned long long a0 = (unsigned long long)(uintptr_t)p;
            if (a0 < base || a0 - base + bytes > size) {
                set_error("p2_mode1_stats_noalloc: %s needs %zu bytes, its allocation holds %llu "
                          "from that address", name, bytes, base + size - a0);
                return P2_EINVAL;
            }
        }
    }
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
    const size_t RR = (size_t)R * R, Pk = (size_t)R * (R + 1) / 2;
    int rc = P2_OK;
    if (K > 0) {
        if (rc == P2_OK) rc = na_check_buffer(T, (size_t)K * RR * sizeof(float), dev, "T");
        if (rc == P2_OK) rc = na_check_buffer(G, (size_t)K * Pk * sizeof(double), dev, "G");
        if (rc == P2_OK) rc = na_check_buffer(W, (size_t)K * R * sizeof(float), dev, "W");
    }
    if (rc == P2_OK) rc = na_check_buffer(M1, RR * sizeof(double), dev, "M1");
    if (rc == P2_OK && WtW) rc = na_check_buffer(WtW, RR * sizeof(double), dev, "WtW");
    if (rc != P2_OK) return rc;
    double *scratch = nullptr;
    rc = na_scratch(&scratch);
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
