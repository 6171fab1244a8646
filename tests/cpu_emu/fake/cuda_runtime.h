// Minimal CPU stand-in for the CUDA runtime + device intrinsics, used to run
// the library's kernels on the host (one std::thread per CUDA thread, blocks
// run one after another) under AddressSanitizer.
#pragma once
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <functional>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <vector>

#define __host__
#define __device__
#define __global__
#define __forceinline__ inline
#define __restrict__
#define __align__(x)
#define __launch_bounds__(...)
#define __shared__ static

struct dim3 {
    unsigned x, y, z;
    dim3(unsigned a = 1, unsigned b = 1, unsigned c = 1) : x(a), y(b), z(c) {}
};
struct emu_uint3 { unsigned x = 0, y = 0, z = 0; };
struct alignas(16) float4 { float x, y, z, w; };
struct alignas(16) uint4 { unsigned x, y, z, w; };
inline uint4 make_uint4(unsigned a, unsigned b, unsigned c, unsigned d) { return uint4{a, b, c, d}; }
extern thread_local emu_uint3 threadIdx, blockIdx;
extern thread_local dim3 blockDim, gridDim;

typedef int cudaError_t;
enum { cudaSuccess = 0, cudaErrorInvalidValue = 1, cudaErrorMemoryAllocation = 2,
       cudaErrorInvalidConfiguration = 9, cudaErrorNotSupported = 801 };
typedef void *cudaStream_t;
typedef void *cudaEvent_t;
typedef void *cudaGraph_t;
typedef void *cudaGraphExec_t;
enum cudaMemcpyKind { cudaMemcpyHostToHost, cudaMemcpyHostToDevice, cudaMemcpyDeviceToHost,
                      cudaMemcpyDeviceToDevice, cudaMemcpyDefault };
enum cudaStreamCaptureStatus { cudaStreamCaptureStatusNone, cudaStreamCaptureStatusActive };
enum cudaStreamCaptureMode { cudaStreamCaptureModeGlobal, cudaStreamCaptureModeThreadLocal };
enum cudaFuncAttribute { cudaFuncAttributeMaxDynamicSharedMemorySize };
enum { cudaStreamNonBlocking = 1, cudaEventRecordExternal = 1 };
struct cudaFuncAttributes { size_t sharedSizeBytes = 0; int numRegs = 0; };
struct cudaDeviceProp { int multiProcessorCount; size_t sharedMemPerBlockOptin; char name[256]; };

inline const char *cudaGetErrorString(cudaError_t e) { return e == 0 ? "no error" : "emulated error"; }
inline cudaError_t cudaGetLastError() { return cudaSuccess; }
inline cudaError_t cudaSetDevice(int) { return cudaSuccess; }
inline cudaError_t cudaGetDevice(int *d) { *d = 0; return cudaSuccess; }
inline cudaError_t cudaGetDeviceCount(int *n) { *n = 1; return cudaSuccess; }
int emu_nsm();
inline cudaError_t cudaGetDeviceProperties(cudaDeviceProp *p, int) {
    p->multiProcessorCount = emu_nsm();
    p->sharedMemPerBlockOptin = 232448;
    strcpy(p->name, "emulated");
    return cudaSuccess;
}
template <class T> inline cudaError_t cudaMalloc(T **p, size_t n) {
    *p = (T *)malloc(n ? n : 1);
    if (*p) memset((void *)*p, 0xA5, n);      // garbage like fresh device memory
    return *p ? cudaSuccess : cudaErrorMemoryAllocation;
}
template <class T> inline cudaError_t cudaMallocAsync(T **p, size_t n, cudaStream_t) { return cudaMalloc(p, n); }
inline cudaError_t cudaFree(void *p) { free(p); return cudaSuccess; }
// free memory: EMU_FREE_BYTES if set (to drive size-dependent paths), else 8 GiB
inline cudaError_t cudaMemGetInfo(size_t *f, size_t *t) {
    const char *e = getenv("EMU_FREE_BYTES");
    *f = e ? (size_t)strtoull(e, nullptr, 10) : ((size_t)8 << 30);
    *t = (size_t)16 << 30;
    return cudaSuccess;
}
inline cudaError_t cudaFreeAsync(void *p, cudaStream_t) { free(p); return cudaSuccess; }
// memory pools: creation refused, so callers take their cudaMalloc path
typedef void *cudaMemPool_t;
enum cudaMemAllocationType { cudaMemAllocationTypePinned = 1 };
enum cudaMemAllocationHandleType { cudaMemHandleTypeNone = 0 };
enum cudaMemLocationType { cudaMemLocationTypeDevice = 1 };
struct cudaMemLocation { cudaMemLocationType type; int id; };
struct cudaMemPoolProps {
    cudaMemAllocationType allocType;
    cudaMemAllocationHandleType handleTypes;
    cudaMemLocation location;
    void *win32SecurityAttributes;
    size_t maxSize;
    unsigned char reserved[56];
};
enum cudaMemPoolAttr { cudaMemPoolAttrReleaseThreshold = 4 };
inline cudaError_t cudaMemPoolCreate(cudaMemPool_t *, const cudaMemPoolProps *) { return cudaErrorNotSupported; }
inline cudaError_t cudaMemPoolSetAttribute(cudaMemPool_t, cudaMemPoolAttr, void *) { return cudaErrorNotSupported; }
inline cudaError_t cudaMemPoolDestroy(cudaMemPool_t) { return cudaSuccess; }
template <class T> inline cudaError_t cudaMallocFromPoolAsync(T **p, size_t n, cudaMemPool_t, cudaStream_t) { return cudaMalloc(p, n); }
inline cudaError_t cudaMemcpy(void *d, const void *s, size_t n, cudaMemcpyKind) { if (n) memmove(d, s, n); return cudaSuccess; }
inline cudaError_t cudaMemcpyAsync(void *d, const void *s, size_t n, cudaMemcpyKind k, cudaStream_t = nullptr) { return cudaMemcpy(d, s, n, k); }
inline cudaError_t cudaMemsetAsync(void *d, int v, size_t n, cudaStream_t = nullptr) { memset(d, v, n); return cudaSuccess; }
inline cudaError_t cudaStreamSynchronize(cudaStream_t) { return cudaSuccess; }
inline cudaError_t cudaStreamCreate(cudaStream_t *s) { *s = (void *)1; return cudaSuccess; }
inline cudaError_t cudaStreamCreateWithFlags(cudaStream_t *s, unsigned) { *s = (void *)1; return cudaSuccess; }
inline cudaError_t cudaStreamDestroy(cudaStream_t) { return cudaSuccess; }
inline cudaError_t cudaStreamIsCapturing(cudaStream_t, cudaStreamCaptureStatus *c) { *c = cudaStreamCaptureStatusNone; return cudaSuccess; }
inline cudaError_t cudaStreamBeginCapture(cudaStream_t, cudaStreamCaptureMode) { return cudaErrorNotSupported; }
inline cudaError_t cudaStreamEndCapture(cudaStream_t, cudaGraph_t *) { return cudaErrorNotSupported; }
inline cudaError_t cudaGraphInstantiate(cudaGraphExec_t *, cudaGraph_t, unsigned long long) { return cudaErrorNotSupported; }
inline cudaError_t cudaGraphLaunch(cudaGraphExec_t, cudaStream_t) { return cudaErrorNotSupported; }
inline cudaError_t cudaGraphDestroy(cudaGraph_t) { return cudaSuccess; }
inline cudaError_t cudaGraphExecDestroy(cudaGraphExec_t) { return cudaSuccess; }
inline cudaError_t cudaEventCreate(cudaEvent_t *e) { *e = new double(0); return cudaSuccess; }
inline cudaError_t cudaEventDestroy(cudaEvent_t e) { delete (double *)e; return cudaSuccess; }
inline cudaError_t cudaEventRecord(cudaEvent_t e, cudaStream_t = nullptr) {
    *(double *)e = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now().time_since_epoch()).count();
    return cudaSuccess;
}
inline cudaError_t cudaEventRecordWithFlags(cudaEvent_t e, cudaStream_t s, unsigned) { return cudaEventRecord(e, s); }
inline cudaError_t cudaEventSynchronize(cudaEvent_t) { return cudaSuccess; }
inline cudaError_t cudaEventElapsedTime(float *ms, cudaEvent_t a, cudaEvent_t b) { *ms = (float)(*(double *)b - *(double *)a); return cudaSuccess; }
template <class F> inline cudaError_t cudaOccupancyMaxActiveBlocksPerMultiprocessor(int *n, F, int, size_t) { *n = 1; return cudaSuccess; }
template <class F> inline cudaError_t cudaFuncGetAttributes(cudaFuncAttributes *a, F) { *a = cudaFuncAttributes{}; return cudaSuccess; }
template <class F> inline cudaError_t cudaFuncSetAttribute(F, cudaFuncAttribute, int) { return cudaSuccess; }
template <class T> inline cudaError_t cudaGetSymbolAddress(void **p, T &sym) { *p = (void *)&sym; return cudaSuccess; }
// every pointer counts as device memory of device 0; no driver entry points
enum cudaMemoryType { cudaMemoryTypeUnregistered = 0, cudaMemoryTypeHost = 1,
                      cudaMemoryTypeDevice = 2, cudaMemoryTypeManaged = 3 };
struct cudaPointerAttributes { cudaMemoryType type; int device; void *devicePointer; void *hostPointer; };
inline cudaError_t cudaPointerGetAttributes(cudaPointerAttributes *a, const void *p) {
    *a = cudaPointerAttributes{cudaMemoryTypeDevice, 0, (void *)p, nullptr};
    return cudaSuccess;
}
enum cudaDriverEntryPointQueryResult { cudaDriverEntryPointSuccess = 0, cudaDriverEntryPointSymbolNotFound = 1 };
enum { cudaEnableDefault = 0 };
inline cudaError_t cudaGetDriverEntryPointByVersion(const char *, void **f, unsigned, unsigned long long,
                                                    cudaDriverEntryPointQueryResult *q) {
    *f = nullptr;
    if (q) *q = cudaDriverEntryPointSymbolNotFound;
    return cudaErrorNotSupported;
}

// ---- device side ---------------------------------------------------------
void emu_syncthreads();
void emu_warp_sync(unsigned mask);
uint64_t emu_warp_xchg(unsigned mask, uint64_t v, int src);   // value of lane src (in warp)
extern thread_local unsigned char *emu_dyn_smem_ptr;
inline void __syncthreads() { emu_syncthreads(); }
inline void __syncwarp(unsigned mask = 0xffffffffu) { emu_warp_sync(mask); }
template <class T> inline uint64_t emu_bits(T v) { uint64_t b = 0; memcpy(&b, &v, sizeof(T)); return b; }
template <class T> inline T emu_from(uint64_t b) { T v; memcpy(&v, &b, sizeof(T)); return v; }
inline int emu_lane() { return (int)(threadIdx.x & 31); }
template <class T> inline T __shfl_sync(unsigned m, T v, int src) { return emu_from<T>(emu_warp_xchg(m, emu_bits(v), src & 31)); }
template <class T> inline T __shfl_xor_sync(unsigned m, T v, int o) { return emu_from<T>(emu_warp_xchg(m, emu_bits(v), emu_lane() ^ o)); }
template <class T> inline T __shfl_up_sync(unsigned m, T v, int d) {
    const int l = emu_lane();
    T r = emu_from<T>(emu_warp_xchg(m, emu_bits(v), l >= d ? l - d : l));
    return r;
}
template <class T> inline T __shfl_down_sync(unsigned m, T v, int d) {
    const int l = emu_lane();
    return emu_from<T>(emu_warp_xchg(m, emu_bits(v), l + d < 32 ? l + d : l));
}
// bit l set when lane l's predicate is true (every lane of mask m takes part)
inline unsigned __ballot_sync(unsigned m, int pred) {
    unsigned r = 0;
    for (int l = 0; l < 32; ++l)
        if (emu_warp_xchg(m, (uint64_t)(pred != 0), l)) r |= 1u << l;
    return r & m;
}
unsigned emu_match_any(unsigned m, uint64_t key);
template <class T> inline unsigned __match_any_sync(unsigned m, T key) { return emu_match_any(m, emu_bits(key)); }
inline int __popc(unsigned x) { return __builtin_popcount(x); }
template <class T> inline T __ldg(const T *p) { return *p; }
inline int __float_as_int(float f) { int i; memcpy(&i, &f, 4); return i; }
inline float __int_as_float(int i) { float f; memcpy(&f, &i, 4); return f; }
inline int __double2hiint(double d) { int64_t b; memcpy(&b, &d, 8); return (int)(b >> 32); }
std::mutex &emu_atomic_mutex();
template <class T, class U> inline T atomicAdd(T *p, U v) { std::lock_guard<std::mutex> g(emu_atomic_mutex()); T o = *p; *p = o + (T)v; return o; }
template <class T, class U> inline T atomicOr(T *p, U v) { std::lock_guard<std::mutex> g(emu_atomic_mutex()); T o = *p; *p = o | (T)v; return o; }
template <class T, class U> inline T atomicMax(T *p, U v) { std::lock_guard<std::mutex> g(emu_atomic_mutex()); T o = *p; *p = std::max(o, (T)v); return o; }
using std::max;
using std::min;

// ---- launches ---------------------------------------------------------------
struct EmuCfg { dim3 g, b; size_t smem; };
inline EmuCfg emu_cfg(dim3 g, dim3 b, size_t smem = 0, cudaStream_t = nullptr) { return EmuCfg{g, b, smem}; }
void emu_run_grid(const EmuCfg &c, const std::function<void()> &f);
