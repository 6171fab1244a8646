// Launch of the grouped Procrustes kernel (R > 12), one instantiation per
// register-array width RB = R rounded up to a multiple of eight, for a number
// type D (double-word or FP64).  Included by p2_polar_grp.cu (double-word)
// and p2_polar_grp_f64.cu (FP64), so the two sets of instances compile in
// parallel.
#pragma once

#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <type_traits>

#include "p2_internal.cuh"
#include "p2_polar.cuh"
#include "p2_polar_grp.cuh"

namespace p2 {


template <class D, int RB, int PG, int RT = 0, int MODE = 0>
static void launch_grp(const p2_ctx *c, const dw *G, const float *W, SmallState *st, float *T,
                       int64_t K, cudaStream_t s, double rtol2, const int32_t *order,
                       int32_t *qrcnt, GrpSplit<D> sc = GrpSplit<D>{}) {
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
    k_polar_grp<RB, PG, RT, D, MODE><<<(unsigned)nblk, threads, smem, s>>>(
        G, W, st, T, K, R, (float)rtol2, spb, order, qrcnt, sc);
}

// Pointers into the context's scratch for one chunk of the split step.
static GrpSplit<dw> split_scratch(const p2_ctx *c, const dw *mpre) {
    const int64_t CH = c->split_chunk, R = c->R, cap = c->split_cap;
    unsigned char *b = c->d_split;
    auto take = [&b](size_t bytes) {
        unsigned char *p = b;
        b += (bytes + 255) & ~(size_t)255;
        return p;
    };
    GrpSplit<dw> sc;
    sc.mpre = mpre;
    sc.qh = reinterpret_cast<dw *>(take(sizeof(dw) * CH * R * R));
    sc.de = reinterpret_cast<dw *>(take(sizeof(dw) * CH * 2 * R));
    sc.dout = reinterpret_cast<dw *>(take(sizeof(dw) * CH * R));
    sc.wv = reinterpret_cast<float *>(take(sizeof(float) * CH * R));
    sc.meta = reinterpret_cast<int *>(take(sizeof(int) * CH));
    sc.nrec = reinterpret_cast<int32_t *>(take(sizeof(int32_t) * CH));
    sc.rec = reinterpret_cast<RotRec<dw> *>(take(sizeof(RotRec<dw>) * CH * cap));
    sc.rkr = reinterpret_cast<uint8_t *>(take((size_t)CH * cap));
    sc.cap = cap;
    const int64_t want = c->tune.split_record_cap;
    sc.lim = (want > 0 && want < cap) ? want : cap;
    return sc;
}

// The split step runs for the double-word arithmetic when the scratch exists,
// the subjects come in a Q-step order and the tuning selects it.
static bool use_split(const p2_ctx *c, int64_t K, const int32_t *order) {
    return c->d_split && order && K > 0 && c->tune.procrustes_split;
}

// The split Procrustes step over chunks of subjects: MODE 1 (tridiagonal
// form, Q_h to the scratch), k_qr_record (QR on the tridiagonal, rotations
// recorded), MODE 2 (rotations applied to Q_h, T_k), then the fused kernel
// for the subjects whose rotations did not fit.  Same results as the fused
// kernel, bit for bit.
template <int RB, int PG, int RT = 0>
static void launch_grp_split(const p2_ctx *c, const dw *G, const float *W, SmallState *st,
                             float *T, int64_t K, cudaStream_t s, double rtol2,
                             const int32_t *order, int32_t *qrcnt, const dw *mpre) {
    const int R = c->R;
    GrpSplit<dw> sc = split_scratch(c, mpre);
    const int64_t CH = c->split_chunk;
    const int nt = QR_THREADS;
    const size_t smb = (size_t)2 * R * nt * sizeof(dw);
    for (int64_t c0 = 0; c0 < K; c0 += CH) {
        const int64_t n = (K - c0) < CH ? (K - c0) : CH;
        const int32_t *ord = order + c0;
        launch_grp<dw, RB, PG, RT, 1>(c, G, W, st, T, n, s, rtol2, ord, qrcnt, sc);
        k_qr_record<RT, dw><<<(unsigned)((n + nt - 1) / nt), nt, smb, s>>>(sc, n, R, ord, qrcnt, st);
        launch_grp<dw, RB, PG, RT, 2>(c, G, W, st, T, n, s, rtol2, ord, qrcnt, sc);
        cudaMemsetAsync(c->d_split_cnt, 0, sizeof(int32_t), s);
        k_split_collect<<<(unsigned)((n + 255) / 256 < 1024 ? (n + 255) / 256 : 1024), 256, 0, s>>>(
            sc.nrec, n, ord, c->d_split_list, c->d_split_cnt);
        GrpSplit<dw> fb{};
        fb.kdev = c->d_split_cnt;
        fb.mpre = mpre;
        launch_grp<dw, RB, PG, RT, 0>(c, G, W, st, T, n, s, rtol2, c->d_split_list, qrcnt, fb);
    }
}

// dynamic shared memory allowed: the opt-in maximum less the kernel's static
// shared memory
template <class D, int RB, int PG, int RT = 0, int MODE = 0>
static cudaError_t allow_grp1(int cap) {
    cudaFuncAttributes a;
    cudaError_t e = cudaFuncGetAttributes(&a, k_polar_grp<RB, PG, RT, D, MODE>);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(k_polar_grp<RB, PG, RT, D, MODE>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize,
                                cap - (int)a.sharedSizeBytes);
}
// the fused instance, and for the double-word type the two split ones and
// the QR recorder
template <class D, int RB, int PG, int RT = 0>
static cudaError_t allow_grp(int cap) {
    cudaError_t e = allow_grp1<D, RB, PG, RT, 0>(cap);
    if constexpr (std::is_same<D, dw>::value) {
        if (e == cudaSuccess) e = allow_grp1<D, RB, PG, RT, 1>(cap);
        if (e == cudaSuccess) e = allow_grp1<D, RB, PG, RT, 2>(cap);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(k_qr_record<RT, D>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)(2 * P2_RMAX * 128 * sizeof(D)));
    }
    return e;
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
                             const int32_t *order, int32_t *qrcnt, const dw *mpre = nullptr) {
    const int R = c->R;
    GrpSplit<D> fz{};
    if constexpr (std::is_same<D, dw>::value) fz.mpre = mpre;
    if constexpr (std::is_same<D, dw>::value) {
        if (use_split(c, K, order)) {
            switch (R) {
#define P2_SPLIT(r, rb, pg) \
                case r: launch_grp_split<rb, pg, r>(c, G, W, st, T, K, s, rtol2, order, qrcnt, mpre); \
                        return cudaGetLastError();
                P2_SPLIT(13, 16, 8) P2_SPLIT(14, 16, 8) P2_SPLIT(15, 16, 8) P2_SPLIT(16, 16, 8)
                P2_SPLIT(24, 24, 8) P2_SPLIT(32, 32, 8) P2_SPLIT(40, 48, 16) P2_SPLIT(48, 48, 16)
                P2_SPLIT(56, 64, 16) P2_SPLIT(64, 64, 16)
#undef P2_SPLIT
                default: break;
            }
            if (R <= 16) launch_grp_split<16, 8>(c, G, W, st, T, K, s, rtol2, order, qrcnt, mpre);
            else if (R <= 24) launch_grp_split<24, 8>(c, G, W, st, T, K, s, rtol2, order, qrcnt, mpre);
            else if (R <= 32) launch_grp_split<32, 8>(c, G, W, st, T, K, s, rtol2, order, qrcnt, mpre);
            else if (R <= 48) launch_grp_split<48, 16>(c, G, W, st, T, K, s, rtol2, order, qrcnt, mpre);
            else launch_grp_split<64, 16>(c, G, W, st, T, K, s, rtol2, order, qrcnt, mpre);
            return cudaGetLastError();
        }
    }
    // ranks 13 .. 16 and the multiples of 8 run an instance compiled for the
    // rank (loop bounds and offsets constant), the others the generic one
    switch (R) {
        case 13: launch_grp<D, 16, 8, 13>(c, G, W, st, T, K, s, rtol2, order, qrcnt, fz); return cudaGetLastError();
        case 14: launch_grp<D, 16, 8, 14>(c, G, W, st, T, K, s, rtol2, order, qrcnt, fz); return cudaGetLastError();
        case 15: launch_grp<D, 16, 8, 15>(c, G, W, st, T, K, s, rtol2, order, qrcnt, fz); return cudaGetLastError();
        case 16: launch_grp<D, 16, 8, 16>(c, G, W, st, T, K, s, rtol2, order, qrcnt, fz); return cudaGetLastError();
        case 24: launch_grp<D, 24, 8, 24>(c, G, W, st, T, K, s, rtol2, order, qrcnt, fz); return cudaGetLastError();
        case 32: launch_grp<D, 32, 8, 32>(c, G, W, st, T, K, s, rtol2, order, qrcnt, fz); return cudaGetLastError();
        case 40: launch_grp<D, 48, 16, 40>(c, G, W, st, T, K, s, rtol2, order, qrcnt, fz); return cudaGetLastError();
        case 48: launch_grp<D, 48, 16, 48>(c, G, W, st, T, K, s, rtol2, order, qrcnt, fz); return cudaGetLastError();
        case 56: launch_grp<D, 64, 16, 56>(c, G, W, st, T, K, s, rtol2, order, qrcnt, fz); return cudaGetLastError();
        case 64: launch_grp<D, 64, 16, 64>(c, G, W, st, T, K, s, rtol2, order, qrcnt, fz); return cudaGetLastError();
        default: break;
    }
    if (R <= 16)
        launch_grp<D, 16, 8>(c, G, W, st, T, K, s, rtol2, order, qrcnt, fz);
    else if (R <= 24)
        launch_grp<D, 24, 8>(c, G, W, st, T, K, s, rtol2, order, qrcnt, fz);
    else if (R <= 32)
        launch_grp<D, 32, 8>(c, G, W, st, T, K, s, rtol2, order, qrcnt, fz);
    else if (R <= 48)
        launch_grp<D, 48, 16>(c, G, W, st, T, K, s, rtol2, order, qrcnt, fz);
    else
        launch_grp<D, 64, 16>(c, G, W, st, T, K, s, rtol2, order, qrcnt, fz);
    return cudaGetLastError();
}

}  // namespace p2
