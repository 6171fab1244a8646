// C ABI of libp2.so: context, memory, call order, CUDA graph replay.
// Every numerical step runs in the kernels of p2_kernels.cu / p2_load.cu.
#include <cuda_runtime.h>
#include <stdarg.h>
#include <stdint.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <utility>
#include <vector>
#include <math.h>

#include "p2_internal.cuh"

namespace p2 {

static thread_local char g_err[1024] = "";

void set_error(const char *fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
}

static int fail(int code, const char *msg) {
    set_error("%s", msg);
    return code;
}

// Device memory of a context comes, stream-ordered, from the context's own
// pool, which keeps what is freed for the next allocation (a reload of
// slices reuses it without cudaMalloc/cudaFree and their device-wide
// synchronisation); the pool's memory goes back at p2_destroy.  Without a
// pool (creation refused) plain cudaMalloc/cudaFree.
cudaError_t ctx_malloc(const p2_ctx *c, void **p, size_t bytes) {
    if (c->pool) return cudaMallocFromPoolAsync(p, bytes, c->pool, c->stream);
    return cudaMalloc(p, bytes);
}
void ctx_free(const p2_ctx *c, void *p) {
    if (!p) return;
    if (c->pool)
        cudaFreeAsync(p, c->stream);
    else
        cudaFree(p);
}

template <class T>
static int dalloc(p2_ctx *c, T **p, size_t count) {
    *p = nullptr;
    if (count == 0) count = 1;
    cudaError_t e = ctx_malloc(c, (void **)p, sizeof(T) * count);
    if (e != cudaSuccess) {
        cudaGetLastError();
        set_error("cudaMalloc of %zu bytes failed: %s", sizeof(T) * count, cudaGetErrorString(e));
        return e == cudaErrorMemoryAllocation ? P2_ENOMEM : P2_ECUDA;
    }
    c->dev_bytes += sizeof(T) * count;
    return P2_OK;
}

template <class T>
static void dfree(p2_ctx *c, T **p, size_t count) {
    if (*p) {
        ctx_free(c, *p);
        if (count == 0) count = 1;
        c->dev_bytes -= sizeof(T) * count;
    }
    *p = nullptr;
}

#define P2_TRY(x)                   \
    do {                            \
        int _rc = (x);              \
        if (_rc != P2_OK) return _rc; \
    } while (0)

static void free_data(p2_ctx *c) {
    const size_t K = (size_t)c->X.K, J = (size_t)c->X.J, N = (size_t)c->X.N,
                 nnz = (size_t)c->X.nnz, R = (size_t)c->R, P = (size_t)c->P;
    dfree(c, &c->X.subj_row, K + 1);
    dfree(c, &c->X.subj_nnz, K + 1);
    dfree(c, &c->X.row_len, N);
    dfree(c, &c->X.col, nnz);
    dfree(c, &c->X.val, nnz);
    dfree(c, &c->d_perm_old2new, J);
    dfree(c, &c->d_colcount, J);
    dfree(c, &c->d_V, J * v_stride<float>((int)R));
    dfree(c, &c->d_Vprev, J * v_stride<float>((int)R));
    dfree(c, &c->d_Vh, J * v_stride<bf16_t>((int)R));
    dfree(c, &c->d_Vprevh, J * v_stride<bf16_t>((int)R));
    dfree(c, &c->d_Ph, (size_t)c->X.p_rows * v_stride<bf16_t>((int)R));
    dfree(c, &c->d_Vun, J * R);
    dfree(c, &c->d_M2, J * R);
    dfree(c, &c->d_P, (size_t)c->X.p_rows * v_stride<float>((int)R));
    dfree(c, &c->X.csc_row, nnz);
    dfree(c, &c->X.csc_val, nnz);
    dfree(c, &c->X.seg_start, (size_t)c->X.nseg);
    dfree(c, &c->X.seg_end, (size_t)c->X.nseg);
    dfree(c, &c->X.col_seg, (size_t)c->X.nblk * J + 1);
    dfree(c, &c->d_segpart, (size_t)c->X.nseg * R);
    dfree(c, &c->d_W, K * R);
    dfree(c, &c->d_M3, K * R);
    dfree(c, &c->d_qrcnt, K);
    dfree(c, &c->d_passW, K);
    dfree(c, &c->d_sorder, K);
    dfree(c, &c->d_passV, J);
    dfree(c, &c->d_order, K);
    dfree(c, &c->d_rank, K);
    dfree(c, &c->d_binoff, (size_t)((K + P2_ORDER_CHUNK - 1) / P2_ORDER_CHUNK) * P2_ORDER_BINS);
    dfree(c, &c->d_T, K * R * R);
    dfree(c, &c->d_G, K * P);
    dfree(c, &c->d_Gf, K * P);
    dfree(c, &c->d_split, c->split_bytes);
    dfree(c, &c->d_split_list, (size_t)c->split_chunk);
    dfree(c, &c->d_split_cnt, 1);
    dfree(c, &c->d_Mtc, K * P);
    c->split_chunk = c->split_cap = 0;
    c->split_bytes = 0;
    delete[] c->h_perm_new2old;
    delete[] c->h_perm_old2new;
    c->h_perm_new2old = c->h_perm_old2new = nullptr;
    if (c->graph) {
        cudaGraphExecDestroy(c->graph);
        c->graph = nullptr;
    }
    c->X = DevX{};
    c->loaded = false;
    c->inited = false;
    c->iters_done = 0;
}

static int alloc_data(p2_ctx *c, int64_t K, int32_t J, int64_t N, int64_t nnz) {
    const size_t R = (size_t)c->R, P = (size_t)c->P;
    c->X.K = K;
    c->X.J = J;
    c->X.N = N;
    c->X.nnz = nnz;
    P2_TRY(dalloc(c, &c->X.subj_row, (size_t)K + 1));
    P2_TRY(dalloc(c, &c->X.subj_nnz, (size_t)K + 1));
    P2_TRY(dalloc(c, &c->X.row_len, (size_t)N));
    P2_TRY(dalloc(c, &c->X.col, (size_t)nnz));
    P2_TRY(dalloc(c, &c->X.val, (size_t)nnz));
    P2_TRY(dalloc(c, &c->d_perm_old2new, (size_t)J));
    P2_TRY(dalloc(c, &c->d_colcount, (size_t)J));
    if (c->bf16) {
        const size_t nv = (size_t)J * v_stride<bf16_t>(R);    // padded rows, zero padding
        P2_TRY(dalloc(c, &c->d_Vh, nv));
        P2_TRY(dalloc(c, &c->d_Vprevh, nv));
        P2_CUDA_TRY(cudaMemsetAsync(c->d_Vh, 0, sizeof(bf16_t) * nv, c->stream));
        P2_CUDA_TRY(cudaMemsetAsync(c->d_Vprevh, 0, sizeof(bf16_t) * nv, c->stream));
        P2_TRY(dalloc(c, &c->d_Ph, (size_t)N * v_stride<bf16_t>(R)));   // rows padded as V
        c->X.p_rows = N;
    } else {
        const size_t nv = (size_t)J * v_stride<float>(R);     // padded rows, zero padding
        P2_TRY(dalloc(c, &c->d_V, nv));
        P2_TRY(dalloc(c, &c->d_Vprev, nv));
        P2_CUDA_TRY(cudaMemsetAsync(c->d_V, 0, sizeof(float) * nv, c->stream));
        P2_CUDA_TRY(cudaMemsetAsync(c->d_Vprev, 0, sizeof(float) * nv, c->stream));
        P2_TRY(dalloc(c, &c->d_P, (size_t)N * v_stride<float>(R)));     // rows padded as V
        c->X.p_rows = N;
    }
    P2_TRY(dalloc(c, &c->d_T, (size_t)K * R * R));
    P2_TRY(dalloc(c, &c->d_Vun, (size_t)J * R));
    P2_TRY(dalloc(c, &c->d_M2, (size_t)J * R));
    P2_TRY(dalloc(c, &c->d_W, (size_t)K * R));
    P2_TRY(dalloc(c, &c->d_M3, (size_t)K * R));
    P2_TRY(dalloc(c, &c->d_qrcnt, (size_t)K));
    P2_TRY(dalloc(c, &c->d_order, (size_t)K));
    P2_TRY(dalloc(c, &c->d_rank, (size_t)K));
    P2_TRY(dalloc(c, &c->d_binoff,
                  (size_t)((K + P2_ORDER_CHUNK - 1) / P2_ORDER_CHUNK) * P2_ORDER_BINS));
    P2_CUDA_TRY(cudaMemsetAsync(c->d_qrcnt, 0, sizeof(int32_t) * (size_t)K, c->stream));
    P2_TRY(dalloc(c, &c->d_sorder, (size_t)K));
    if (c->opt.nonneg) {
        P2_TRY(dalloc(c, &c->d_passW, (size_t)K));
        P2_TRY(dalloc(c, &c->d_passV, (size_t)J));
        P2_CUDA_TRY(cudaMemsetAsync(c->d_passW, 0, sizeof(uint64_t) * (size_t)K, c->stream));
        P2_CUDA_TRY(cudaMemsetAsync(c->d_passV, 0, sizeof(uint64_t) * (size_t)J, c->stream));
    }
    P2_TRY(dalloc(c, &c->d_G, (size_t)K * P));
    P2_TRY(dalloc(c, &c->d_Gf, (size_t)K * P));
    P2_CUDA_TRY(cudaMemsetAsync(c->d_M3, 0, sizeof(float) * (size_t)K * R, c->stream));
    c->h_perm_new2old = new int32_t[J];
    c->h_perm_old2new = new int32_t[J];
    if (R >= 2 && K > 0 && !c->opt.fp64_procrustes) {
        // scratch of the split Procrustes step for one chunk of subjects: at
        // most 8 GiB and an eighth of the free memory, a chunk of at least 4,096
        // subjects (otherwise the fused kernel runs)
        const size_t cap = 2 * R * R + 2 * R;       // rotations recorded per subject
        const size_t per = 8 * R * R + 28 * R + 8 + 17 * cap;
        size_t fr = 0, tot = 0;
        if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) {
            cudaGetLastError();
            fr = 0;
        }
        size_t budget = (size_t)8 << 30;
        if (fr / 8 < budget) budget = fr / 8;
        int64_t ch = (int64_t)(budget / per);
        if (ch > K) ch = K;
        if (ch >= 4096 || ch == K) {
            c->split_chunk = ch;
            c->split_cap = (int64_t)cap;
            c->split_bytes = (size_t)ch * per + 16 * 256;
            if (dalloc(c, &c->d_split, c->split_bytes) != P2_OK ||
                dalloc(c, &c->d_split_list, (size_t)ch) != P2_OK ||
                dalloc(c, &c->d_split_cnt, 1) != P2_OK) {
                // the fused kernel needs none of it
                dfree(c, &c->d_split, c->split_bytes);
                dfree(c, &c->d_split_list, (size_t)ch);
                dfree(c, &c->d_split_cnt, 1);
                c->split_chunk = c->split_cap = 0;
                c->split_bytes = 0;
                set_error("");
            }
        }
    }
    if (K > 0 && tc_m_wanted(c)) {
        // every subject's M' for the grouped Procrustes kernels; without the
        // memory they form M' themselves
        if (dalloc(c, &c->d_Mtc, (size_t)K * P) != P2_OK) {
            c->d_Mtc = nullptr;
            set_error("");
        }
    }
    return P2_OK;
}

static int check_ready(p2_ctx *c, bool need_init) {
    if (!c) return fail(P2_EINVAL, "NULL context");
    if (!c->loaded) return fail(P2_ESTATE, "no slices loaded (call p2_load_slices first)");
    if (need_init && !c->inited) return fail(P2_ESTATE, "factors not initialised (call p2_init first)");
    return P2_OK;
}

static int read_flags(p2_ctx *c, int *flags) {
    P2_CUDA_TRY(cudaMemcpyAsync(flags, &c->d_s->flags, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    P2_CUDA_TRY(cudaStreamSynchronize(c->stream));
    return P2_OK;
}

static int flags_status(int flags) {
    if (flags & FLAG_TC_TIMEOUT) {
        set_error("a tensor-core MMA did not complete within its wait limit (flags 0x%x)", flags);
        return P2_ECUDA;
    }
    if (flags & FLAG_NONFINITE) {
        set_error("numeric problem detected on the device (flags 0x%x: non-finite loss)", flags);
        return P2_ENUMERIC;
    }
    return P2_OK;
}

// float -> bfloat16 bits, round to nearest even (NaN kept quiet)
static uint16_t to_bf16_bits(float f) {
    uint32_t u;
    memcpy(&u, &f, 4);
    if ((u & 0x7fffffffu) > 0x7f800000u) return (uint16_t)((u >> 16) | 0x40u);
    u += 0x7fffu + ((u >> 16) & 1u);
    return (uint16_t)(u >> 16);
}
static float from_bf16_bits(uint16_t h) {
    const uint32_t u = (uint32_t)h << 16;
    float f;
    memcpy(&f, &u, 4);
    return f;
}

// Statistics of the factors now on the device and the first Q-step.
static int finish_init(p2_ctx *c) {
    P2_TRY(enqueue_factor_stats(c));
    P2_TRY(enqueue_prologue(c));
    int flags = 0;
    P2_TRY(read_flags(c, &flags));
    c->inited = true;
    c->iters_done = 0;
    return P2_OK;
}

static int set_factors_impl(p2_ctx *c, const float *H, const float *V, const float *W) {
    // the factors are replaced from here on: until finish_init succeeds the
    // context holds no consistent state, so p2_iterate must refuse
    c->inited = false;
    const int R = c->R;
    const int32_t J = c->X.J;
    const int64_t K = c->X.K;
    // relabelled row order, rows padded to the device stride with zeros
    const int VS = c->bf16 ? v_stride<bf16_t>(R) : v_stride<float>(R);
    std::vector<float> Vp((size_t)J * VS, 0.f);
    std::vector<uint16_t> Vb;
    for (int32_t j = 0; j < J; ++j)
        memcpy(&Vp[(size_t)c->h_perm_old2new[j] * VS], V + (size_t)j * R, sizeof(float) * R);
    if (c->bf16) {                          // V stored bfloat16
        Vb.resize(Vp.size());
        for (size_t i = 0; i < Vp.size(); ++i) Vb[i] = to_bf16_bits(Vp[i]);
        P2_CUDA_TRY(cudaMemcpyAsync(c->d_Vh, Vb.data(), sizeof(uint16_t) * Vb.size(),
                                    cudaMemcpyHostToDevice, c->stream));
    } else {
        P2_CUDA_TRY(cudaMemcpyAsync(c->d_V, Vp.data(), sizeof(float) * Vp.size(),
                                    cudaMemcpyHostToDevice, c->stream));
    }
    P2_CUDA_TRY(cudaMemcpyAsync(c->d_H, H, sizeof(float) * R * R, cudaMemcpyHostToDevice, c->stream));
    P2_CUDA_TRY(cudaMemcpyAsync(c->d_W, W, sizeof(float) * (size_t)K * R, cudaMemcpyHostToDevice,
                                c->stream));
    int zero = 0;
    P2_CUDA_TRY(cudaMemcpyAsync(&c->d_s->flags, &zero, sizeof(int), cudaMemcpyHostToDevice, c->stream));
    return finish_init(c);   // its flag read-back also keeps Vp and Vb alive until the copies finished
}

}  // namespace p2

using namespace p2;

extern "C" {

void p2_default_options(p2_options *opt, int32_t R) {
    if (!opt) return;
    memset(opt, 0, sizeof(*opt));
    opt->R = R;
    opt->precision = P2_FP32;
    opt->device = 0;
    opt->use_graph = 1;
    opt->rank_rtol = 1e-5;
    opt->stream = nullptr;
    opt->timing = 0;
    opt->seed = 20170314ULL;
    opt->nonneg = 0;
    opt->fp64_procrustes = 0;
    opt->autotune = 0;
    opt->tune_cache = nullptr;
    opt->tensor_core_m = -1;
}

int p2_create(p2_ctx **out, const p2_options *opt) {
    if (!out || !opt) return fail(P2_EINVAL, "p2_create: NULL argument");
    *out = nullptr;
    if (opt->R < 1 || opt->R > P2_RMAX) return fail(P2_EINVAL, "p2_create: R must be in [1, 64]");
    if (opt->precision != P2_FP32 && opt->precision != P2_BF16)
        return fail(P2_EINVAL, "p2_create: precision must be P2_FP32 or P2_BF16");
    int ndev = 0;
    P2_CUDA_TRY(cudaGetDeviceCount(&ndev));
    if (opt->device < 0 || opt->device >= ndev) return fail(P2_EINVAL, "p2_create: bad device");
    P2_CUDA_TRY(cudaSetDevice(opt->device));
    p2_ctx *c = new p2_ctx();
    c->opt = *opt;
    if (opt->tune_cache) c->tune_cache = opt->tune_cache;
    c->opt.tune_cache = nullptr;                 // the copy above is the one used
    if (!(c->opt.rank_rtol > 0.0)) c->opt.rank_rtol = 1e-5;
    c->R = opt->R;
    c->P = opt->R * (opt->R + 1) / 2;
    c->bf16 = opt->precision == P2_BF16;
    cudaDeviceProp prop;
    cudaError_t e = cudaGetDeviceProperties(&prop, opt->device);
    if (e != cudaSuccess) {
        delete c;
        set_error("cudaGetDeviceProperties: %s", cudaGetErrorString(e));
        return P2_ECUDA;
    }
    c->geo.nsm = prop.multiProcessorCount;
    c->geo.smem_optin = (int)prop.sharedMemPerBlockOptin;
    c->geo.red_blocks = 2 * prop.multiProcessorCount;
    if (opt->stream) {
        c->stream = (cudaStream_t)opt->stream;
        c->own_stream = false;
    } else {
        e = cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) {
            delete c;
            set_error("cudaStreamCreate: %s", cudaGetErrorString(e));
            return P2_ECUDA;
        }
        c->own_stream = true;
    }
    {
        cudaMemPoolProps props;
        memset(&props, 0, sizeof(props));
        props.allocType = cudaMemAllocationTypePinned;
        props.handleTypes = cudaMemHandleTypeNone;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = opt->device;
        if (cudaMemPoolCreate(&c->pool, &props) == cudaSuccess) {
            uint64_t keep = ~0ull;               // keep freed memory for reuse
            if (cudaMemPoolSetAttribute(c->pool, cudaMemPoolAttrReleaseThreshold, &keep) !=
                cudaSuccess) {
                cudaGetLastError();
                cudaMemPoolDestroy(c->pool);
                c->pool = nullptr;
            }
        } else {
            cudaGetLastError();
            c->pool = nullptr;
        }
    }
    if (c->opt.timing) {
        for (int i = 0; i < 8; ++i) {
            if (cudaEventCreate(&c->ev[i]) != cudaSuccess) {
                set_error("cudaEventCreate failed");
                p2_destroy(c);
                return P2_ECUDA;
            }
        }
    }
    int rc = dalloc(c, &c->d_s, 1);
    if (rc == P2_OK) rc = dalloc(c, &c->d_H, (size_t)c->R * c->R);
    const size_t part_stride = stats_part_stride(c->R);
    if (rc == P2_OK) rc = dalloc(c, &c->d_part, (size_t)c->geo.red_blocks * part_stride);
    if (rc == P2_OK) rc = dalloc(c, &c->d_part2, (size_t)c->geo.red_blocks * part_stride);
    if (rc == P2_OK) rc = dalloc(c, &c->d_red, part_stride);
    if (rc == P2_OK) rc = configure_kernels(c);
    if (rc == P2_OK) {
        if (cudaMemsetAsync(c->d_s, 0, sizeof(SmallState), c->stream) != cudaSuccess) rc = P2_ECUDA;
    }
    if (rc != P2_OK) {
        p2_destroy(c);
        return rc;
    }
    *out = c;
    return P2_OK;
}

int p2_get_tuning(p2_ctx *c, p2_tuning *t) {
    if (!c || !t) return fail(P2_EINVAL, "p2_get_tuning: NULL argument");
    *t = c->tune;
    return P2_OK;
}

const char *p2_tuning_note(p2_ctx *c) {
    return c ? c->tune_note.c_str() : "";
}

int p2_set_tuning(p2_ctx *c, const p2_tuning *t) {
    if (!c || !t) return fail(P2_EINVAL, "p2_set_tuning: NULL argument");
    if ((t->procrustes_split != 0 && t->procrustes_split != 1) || t->subject_bins < -1 ||
        t->subject_bins > 1 || t->split_record_cap < 0 || t->m2_block_kib < 0)
        return fail(P2_EINVAL, "p2_set_tuning: bad value");
    c->tune = *t;
    if (c->graph) {                 // the captured iteration holds the old launches
        cudaGraphExecDestroy(c->graph);
        c->graph = nullptr;
    }
    return P2_OK;
}

int p2_set_exchange(p2_ctx *c, p2_exchange_fn fn, void *user) {
    if (!c) return fail(P2_EINVAL, "p2_set_exchange: NULL context");
    if (c->loaded)
        return fail(P2_ESTATE, "p2_set_exchange: call it before p2_load_slices");
    c->xfn = fn;
    c->xuser = fn ? user : nullptr;
    return P2_OK;
}

int p2_destroy(p2_ctx *c) {
    if (!c) return P2_OK;
    cudaSetDevice(c->opt.device);
    if (c->stream) cudaStreamSynchronize(c->stream);
    free_data(c);
    dfree(c, &c->d_s, 1);
    dfree(c, &c->d_H, (size_t)c->R * c->R);
    const size_t part_stride = stats_part_stride(c->R);
    dfree(c, &c->d_part, (size_t)c->geo.red_blocks * part_stride);
    dfree(c, &c->d_part2, (size_t)c->geo.red_blocks * part_stride);
    dfree(c, &c->d_red, part_stride);
    for (int i = 0; i < 8; ++i)
        if (c->ev[i]) cudaEventDestroy(c->ev[i]);
    if (c->stream) cudaStreamSynchronize(c->stream);   // the frees above are stream-ordered
    if (c->pool) cudaMemPoolDestroy(c->pool);
    if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
    delete c;
    return P2_OK;
}

int p2_load_slices(p2_ctx *c, int64_t K, int32_t J, const int64_t *subj_ptr,
                   const int64_t *row_ptr, const int32_t *col, const float *val,
                   int32_t location) {
    if (!c) return fail(P2_EINVAL, "NULL context");
    if (K < 1) return fail(P2_EINVAL, "p2_load_slices: K must be >= 1");
    if (J < 1 || J > 65535) return fail(P2_EINVAL, "p2_load_slices: J must be in [1, 65535]");
    if (!subj_ptr || !row_ptr) return fail(P2_EINVAL, "p2_load_slices: NULL pointer array");
    if (location != 0 && location != 1) return fail(P2_EINVAL, "p2_load_slices: location must be 0 or 1");
    P2_CUDA_TRY(cudaSetDevice(c->opt.device));
    cudaStream_t s = c->stream;
    const cudaMemcpyKind kind = location == 0 ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
    // endpoints: subj_ptr[0] = 0, N = subj_ptr[K]; row_ptr[0] = 0, nnz = row_ptr[N]
    int64_t s0 = 0, N = 0, r0 = 0, nnz = 0;
    if (location == 0) {
        s0 = subj_ptr[0];
        N = subj_ptr[K];
    } else {
        P2_CUDA_TRY(cudaMemcpy(&s0, subj_ptr, 8, cudaMemcpyDeviceToHost));
        P2_CUDA_TRY(cudaMemcpy(&N, subj_ptr + K, 8, cudaMemcpyDeviceToHost));
    }
    if (s0 != 0 || N < 0 || N >= (1LL << 31))
        return fail(P2_EINVAL, "p2_load_slices: subj_ptr[0] must be 0 and 0 <= subj_ptr[K] < 2^31");
    if (location == 0) {
        r0 = row_ptr[0];
        nnz = row_ptr[N];
    } else {
        P2_CUDA_TRY(cudaMemcpy(&r0, row_ptr, 8, cudaMemcpyDeviceToHost));
        P2_CUDA_TRY(cudaMemcpy(&nnz, row_ptr + N, 8, cudaMemcpyDeviceToHost));
    }
    if (r0 != 0 || nnz < 0 || nnz >= (1LL << 31))
        return fail(P2_EINVAL, "p2_load_slices: row_ptr[0] must be 0 and 0 <= row_ptr[N] < 2^31");
    if (nnz > 0 && (!col || !val)) return fail(P2_EINVAL, "p2_load_slices: NULL col/val");
    free_data(c);
    P2_TRY(alloc_data(c, K, J, N, nnz));
    // raw copies of the caller's arrays (subject pointers land in place)
    int64_t *d_row_ptr = nullptr;
    int32_t *d_col = nullptr;
    P2_TRY(dalloc(c, &d_row_ptr, (size_t)N + 1));
    int rc = dalloc(c, &d_col, (size_t)nnz);
    if (rc != P2_OK) {
        dfree(c, &d_row_ptr, (size_t)N + 1);
        free_data(c);
        return rc;
    }
    int64_t *d_subj = nullptr;
    rc = dalloc(c, &d_subj, (size_t)K + 1);
    cudaError_t e = cudaSuccess;
    if (rc == P2_OK) {
        e = cudaMemcpyAsync(d_subj, subj_ptr, 8 * ((size_t)K + 1), kind, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(d_row_ptr, row_ptr, 8 * ((size_t)N + 1), kind, s);
        if (e == cudaSuccess && nnz > 0) e = cudaMemcpyAsync(d_col, col, 4 * (size_t)nnz, kind, s);
        if (e == cudaSuccess && nnz > 0) e = cudaMemcpyAsync(c->X.val, val, 4 * (size_t)nnz, kind, s);
        if (e != cudaSuccess) {
            set_error("p2_load_slices: copy failed: %s", cudaGetErrorString(e));
            rc = P2_ECUDA;
        }
    }
    if (rc == P2_OK) rc = launch_load(c, d_subj, d_row_ptr, d_col, c->X.val, K, J, N, nnz);
    if (rc == P2_OK) {
        const cudaError_t e = launch_subject_bins(c);
        if (e != cudaSuccess) {
            set_error("p2_load_slices: subject bins failed: %s", cudaGetErrorString(e));
            rc = P2_ECUDA;
        }
    }
    cudaStreamSynchronize(s);
    dfree(c, &d_subj, (size_t)K + 1);
    dfree(c, &d_row_ptr, (size_t)N + 1);
    dfree(c, &d_col, (size_t)nnz);
    if (rc != P2_OK) {
        free_data(c);
        return rc;
    }
    c->loaded = true;
    return P2_OK;
}

// SplitMix64 (Steele, Lea & Flood, OOPSLA 2014): the finaliser and one step.
static inline uint64_t sm64_mix(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}
// n initial values of array a: uniform in [0, 1), multiples of 2^-24 (the
// counter-based layout documented with p2_init)
static void init_uniform(uint64_t seed, uint64_t a, size_t n, float *out) {
    const uint64_t g = 0x9E3779B97F4A7C15ULL, t = 5 + 16 * a;
    for (size_t i = 0; i < n; ++i) {
        const uint64_t s = sm64_mix(seed + g * (t + 1)) ^ sm64_mix((uint64_t)i * g + t);
        const uint64_t x = sm64_mix(s + g);
        out[i] = (float)((double)(x >> 40) * 0x1.0p-24);
    }
}

int p2_init(p2_ctx *c, const float *H0, const float *V0, const float *W0) {
    P2_TRY(check_ready(c, false));
    P2_CUDA_TRY(cudaSetDevice(c->opt.device));
    if (!H0 && !V0 && !W0) {
        const size_t R = (size_t)c->R;
        std::vector<float> H(R * R), V((size_t)c->X.J * R), W((size_t)c->X.K * R);
        init_uniform(c->opt.seed, 1, H.size(), H.data());
        init_uniform(c->opt.seed, 2, V.size(), V.data());
        init_uniform(c->opt.seed, 3, W.size(), W.data());
        return set_factors_impl(c, H.data(), V.data(), W.data());
    }
    if (!H0 || !V0 || !W0) return fail(P2_EINVAL, "p2_init: some but not all factors NULL");
    return set_factors_impl(c, H0, V0, W0);
}

// Device scratch of p2_init_eig, freed on every return path.
struct EigScratch {
    double *v = nullptr, *vn = nullptr, *y = nullptr, *w = nullptr, *z = nullptr, *seg = nullptr,
           *dist = nullptr;
    ~EigScratch() {
        cudaFree(seg);
        cudaFree(v);
        cudaFree(vn);
        cudaFree(y);
        cudaFree(w);
        cudaFree(z);
        cudaFree(dist);
    }
};

int p2_init_eig(p2_ctx *c, int32_t max_iter, double tol, int32_t *n_done) {
    P2_TRY(check_ready(c, false));
    if (c && c->xfn) return fail(P2_EINVAL, "p2_init_eig: not available on a sharded context");
    if (max_iter < 1) return fail(P2_EINVAL, "p2_init_eig: max_iter < 1");
    if (!(tol >= 0.0)) return fail(P2_EINVAL, "p2_init_eig: tol must be >= 0");
    const int R = c->R;
    const int32_t J = c->X.J;
    if (J < R) return fail(P2_EINVAL, "p2_init_eig: J < R (fewer columns than components)");
    P2_CUDA_TRY(cudaSetDevice(c->opt.device));
    c->inited = false;                     // as in set_factors_impl
    // block width: oversampled so that the leading R Ritz vectors converge at
    // lambda_{b+1} / lambda_R; at most the CTA eigen-solver's size and J
    const int b = std::min(std::min(std::max(2 * R, R + 8), (int)P2_RMAX), (int)J);
    // product columns per pass: the N x CW FP64 scratch held to a quarter of
    // the free device memory, at most 16 GiB (every pass re-reads X)
    size_t free_b = 0, total_b = 0;
    P2_CUDA_TRY(cudaMemGetInfo(&free_b, &total_b));
    const size_t budget = std::min(free_b / 4, (size_t)16 << 30);
    const size_t N = c->X.N > 0 ? (size_t)c->X.N : 1;
    const int CW = (int)std::min<size_t>((size_t)b, std::max<size_t>(1, budget / (8 * N)));
    const size_t Jb = (size_t)J * b;
    EigScratch s;
    P2_CUDA_TRY(cudaMalloc(&s.v, Jb * sizeof(double)));
    P2_CUDA_TRY(cudaMalloc(&s.vn, Jb * sizeof(double)));
    P2_CUDA_TRY(cudaMalloc(&s.y, Jb * sizeof(double)));
    P2_CUDA_TRY(cudaMalloc(&s.w, Jb * sizeof(double)));
    P2_CUDA_TRY(cudaMalloc(&s.z, N * CW * sizeof(double)));
    P2_CUDA_TRY(cudaMalloc(&s.seg, ((size_t)c->X.nseg > 0 ? (size_t)c->X.nseg : 1) * CW * sizeof(double)));
    P2_CUDA_TRY(cudaMalloc(&s.dist, sizeof(double)));
    // seeded start block: uniform [0, 1) from the seed's V stream, rows relabelled
    std::vector<float> V0(Jb);
    init_uniform(c->opt.seed, 2, Jb, V0.data());
    std::vector<double> Y0(Jb);
    for (int32_t j = 0; j < J; ++j)
        for (int r = 0; r < b; ++r)
            Y0[(size_t)c->h_perm_old2new[j] * b + r] = (double)V0[(size_t)j * b + r];
    P2_CUDA_TRY(cudaMemcpyAsync(s.y, Y0.data(), Jb * sizeof(double), cudaMemcpyHostToDevice, c->stream));
    int zero = 0;
    P2_CUDA_TRY(cudaMemcpyAsync(&c->d_s->flags, &zero, sizeof(int), cudaMemcpyHostToDevice, c->stream));
    P2_TRY(enqueue_eig_fill(c));
    P2_TRY(enqueue_eig_orth(c, s.y, nullptr, s.v, b, nullptr));
    int32_t it = 0;
    while (it < max_iter) {
        P2_TRY(enqueue_eig_product(c, s.v, b, CW, s.z, s.seg, s.y));   // Y = A V
        P2_TRY(enqueue_eig_ritz(c, s.y, s.v, s.w, b, 0));      // W = Y U
        P2_TRY(enqueue_eig_orth(c, s.w, s.v, s.vn, b, s.dist));
        std::swap(s.v, s.vn);
        ++it;
        double dist = 0.0;
        P2_CUDA_TRY(cudaMemcpyAsync(&dist, s.dist, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
        P2_CUDA_TRY(cudaStreamSynchronize(c->stream));       // also keeps Y0 alive for its copy
        if (!(dist == dist)) break;                           // non-finite: reported below
        if (dist <= tol * tol) break;
    }
    P2_TRY(enqueue_eig_product(c, s.v, b, CW, s.z, s.seg, s.y));
    P2_TRY(enqueue_eig_ritz(c, s.y, s.v, s.w, b, 1));
    int flags = 0;
    P2_TRY(read_flags(c, &flags));
    if (flags & FLAG_EIG_NOCONV) {
        set_error("p2_init_eig: an eigen step did not converge (flags 0x%x)", flags);
        return P2_ENUMERIC;
    }
    if (n_done) *n_done = it;
    return finish_init(c);
}

int p2_set_factors(p2_ctx *c, const float *H, const float *V, const float *W) {
    P2_TRY(check_ready(c, false));
    if (!H || !V || !W) return fail(P2_EINVAL, "p2_set_factors: NULL factor");
    P2_CUDA_TRY(cudaSetDevice(c->opt.device));
    return set_factors_impl(c, H, V, W);
}

// The autotuner (p2_options.autotune): the launch choices of p2_tuning timed
// on this context's data, before the first iteration is captured.  Every
// choice computes the same values, so the trials change no result.
static std::string tune_key(const p2_ctx *c) {
    char b[256];
    snprintf(b, sizeof b, "R=%d precision=%d nonneg=%d fp64=%d tc=%d K=%lld J=%d nnz=%lld", c->R,
             c->opt.precision, c->opt.nonneg ? 1 : 0, c->opt.fp64_procrustes ? 1 : 0,
             c->d_Mtc ? 1 : 0, (long long)c->X.K, (int)c->X.J, (long long)c->X.nnz);
    return b;
}

static bool tune_from_cache(p2_ctx *c, const std::string &key) {
    FILE *f = fopen(c->tune_cache.c_str(), "r");
    if (!f) return false;
    char line[1024];
    bool found = false;
    const std::string want = "\"key\": \"" + key + "\"";
    while (fgets(line, sizeof line, f)) {
        if (!strstr(line, want.c_str())) continue;
        const char *a = strstr(line, "\"procrustes_split\":");
        const char *b = strstr(line, "\"subject_bins\":");
        int ps = 0, sb = 0;
        if (a && b && sscanf(a, "\"procrustes_split\": %d", &ps) == 1 &&
            sscanf(b, "\"subject_bins\": %d", &sb) == 1 && (ps == 0 || ps == 1) &&
            (sb == 0 || sb == 1)) {
            c->tune.procrustes_split = ps;
            c->tune.subject_bins = sb;
            found = true;                 // the last matching line wins
        }
    }
    fclose(f);
    return found;
}

static int autotune(p2_ctx *c) {
    c->tuned = true;
    const std::string key = tune_key(c);
    if (!c->tune_cache.empty() && tune_from_cache(c, key)) {
        c->tune_note = "cache";
        return P2_OK;
    }
    char note[256];
    float q_split = -1.f, q_fused = -1.f;
    if (c->R >= 2 && c->d_split && !c->opt.fp64_procrustes) {
        for (int split = 1; split >= 0; --split) {
            c->tune.procrustes_split = split;
            float ms = 0.f;
            P2_TRY(tune_time_qstep(c, 2, &ms));
            (split ? q_split : q_fused) = ms;
        }
        c->tune.procrustes_split = q_split <= q_fused ? 1 : 0;
    }
    float b_off = 0.f, b_on = 0.f;
    c->tune.subject_bins = 0;
    P2_TRY(tune_time_mode2(c, 2, &b_off));
    c->tune.subject_bins = 1;
    P2_TRY(tune_time_mode2(c, 2, &b_on));
    c->tune.subject_bins = b_on < b_off ? 1 : 0;
    snprintf(note, sizeof note,
             "timed: Q-step split %.3f ms, fused %.3f ms; mode-2 pass bins %.3f ms, no bins %.3f ms",
             q_split, q_fused, b_on, b_off);
    c->tune_note = note;
    if (!c->tune_cache.empty()) {
        FILE *f = fopen(c->tune_cache.c_str(), "a");
        if (f) {
            fprintf(f, "{\"key\": \"%s\", \"procrustes_split\": %d, \"subject_bins\": %d}\n",
                    key.c_str(), c->tune.procrustes_split, c->tune.subject_bins);
            fclose(f);
        }
    }
    return P2_OK;
}

int p2_iterate(p2_ctx *c, int32_t n_iter, double *fit_out) {
    P2_TRY(check_ready(c, true));
    if (n_iter < 0) return fail(P2_EINVAL, "p2_iterate: n_iter < 0");
    P2_CUDA_TRY(cudaSetDevice(c->opt.device));
    if (n_iter > 0 && c->opt.autotune && !c->tuned) {
        P2_TRY(autotune(c));
        if (c->graph) {
            cudaGraphExecDestroy(c->graph);
            c->graph = nullptr;
        }
    }
    const bool use_graph = c->opt.use_graph && !c->xfn;   // a sharded iteration calls the hook
    if (n_iter > 0 && use_graph && !c->graph) {
        cudaGraph_t g = nullptr;
        P2_CUDA_TRY(cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal));
        const int64_t before = c->enqueued;
        int rc = enqueue_iteration(c);
        c->graph_kernels = c->enqueued - before;
        c->enqueued = before;                  // captured, not yet run
        cudaError_t e = cudaStreamEndCapture(c->stream, &g);
        if (rc != P2_OK) {
            if (g) cudaGraphDestroy(g);
            return rc;
        }
        if (e != cudaSuccess) {
            set_error("graph capture failed: %s", cudaGetErrorString(e));
            return P2_ECUDA;
        }
        e = cudaGraphInstantiate(&c->graph, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) {
            c->graph = nullptr;
            set_error("graph instantiate failed: %s", cudaGetErrorString(e));
            return P2_ECUDA;
        }
    }
    for (int32_t i = 0; i < n_iter; ++i) {
        if (use_graph) {
            P2_CUDA_TRY(cudaGraphLaunch(c->graph, c->stream));
            c->enqueued += c->graph_kernels;
        } else {
            P2_TRY(enqueue_iteration(c));
        }
    }
    c->iters_done += n_iter;
    if (fit_out) {
        int flags = 0;
        P2_TRY(read_flags(c, &flags));
        P2_TRY(flags_status(flags));
        P2_CUDA_TRY(cudaMemcpy(fit_out, &c->d_s->fit, sizeof(double), cudaMemcpyDeviceToHost));
    }
    return P2_OK;
}

int p2_fit(p2_ctx *c, double *fit, double *loss) {
    P2_TRY(check_ready(c, true));
    if (c->iters_done == 0) return fail(P2_ESTATE, "p2_fit: no iteration completed yet");
    P2_CUDA_TRY(cudaSetDevice(c->opt.device));
    int flags = 0;
    P2_TRY(read_flags(c, &flags));
    P2_TRY(flags_status(flags));
    if (fit) P2_CUDA_TRY(cudaMemcpy(fit, &c->d_s->fit, sizeof(double), cudaMemcpyDeviceToHost));
    if (loss) P2_CUDA_TRY(cudaMemcpy(loss, &c->d_s->loss, sizeof(double), cudaMemcpyDeviceToHost));
    return P2_OK;
}

int p2_get_factors(p2_ctx *c, float *H, float *V, float *W) {
    P2_TRY(check_ready(c, true));
    P2_CUDA_TRY(cudaSetDevice(c->opt.device));
    const int R = c->R;
    P2_CUDA_TRY(cudaStreamSynchronize(c->stream));
    if (H) P2_CUDA_TRY(cudaMemcpy(H, c->d_H, sizeof(float) * R * R, cudaMemcpyDeviceToHost));
    if (V) {
        const int VS = c->bf16 ? v_stride<bf16_t>(R) : v_stride<float>(R);
        std::vector<float> Vp((size_t)c->X.J * VS);
        if (c->bf16) {
            std::vector<uint16_t> Vb(Vp.size());
            P2_CUDA_TRY(cudaMemcpy(Vb.data(), c->d_Vh, sizeof(uint16_t) * Vb.size(),
                                   cudaMemcpyDeviceToHost));
            for (size_t i = 0; i < Vb.size(); ++i) Vp[i] = from_bf16_bits(Vb[i]);
        } else {
            P2_CUDA_TRY(cudaMemcpy(Vp.data(), c->d_V, sizeof(float) * Vp.size(), cudaMemcpyDeviceToHost));
        }
        for (int32_t j = 0; j < c->X.J; ++j)
            memcpy(V + (size_t)j * R, &Vp[(size_t)c->h_perm_old2new[j] * VS], sizeof(float) * R);
    }
    if (W) P2_CUDA_TRY(cudaMemcpy(W, c->d_W, sizeof(float) * (size_t)c->X.K * R, cudaMemcpyDeviceToHost));
    return P2_OK;
}

int p2_get_mttkrp(p2_ctx *c, int32_t mode, double *out) {
    P2_TRY(check_ready(c, true));
    if (!out) return fail(P2_EINVAL, "p2_get_mttkrp: NULL out");
    if (c->iters_done == 0) return fail(P2_ESTATE, "p2_get_mttkrp: no iteration completed yet");
    P2_CUDA_TRY(cudaSetDevice(c->opt.device));
    P2_CUDA_TRY(cudaStreamSynchronize(c->stream));
    const int R = c->R;
    if (mode == 1) {
        P2_CUDA_TRY(cudaMemcpy(out, c->d_s->M1, sizeof(double) * R * R, cudaMemcpyDeviceToHost));
    } else if (mode == 2) {
        std::vector<double> M((size_t)c->X.J * R);
        P2_CUDA_TRY(cudaMemcpy(M.data(), c->d_M2, sizeof(double) * M.size(), cudaMemcpyDeviceToHost));
        for (int32_t j = 0; j < c->X.J; ++j)
            memcpy(out + (size_t)j * R, &M[(size_t)c->h_perm_old2new[j] * R], sizeof(double) * R);
    } else if (mode == 3) {
        std::vector<float> M((size_t)c->X.K * R);
        P2_CUDA_TRY(cudaMemcpy(M.data(), c->d_M3, sizeof(float) * M.size(), cudaMemcpyDeviceToHost));
        for (size_t i = 0; i < M.size(); ++i) out[i] = (double)M[i];
    } else {
        return fail(P2_EINVAL, "p2_get_mttkrp: mode must be 1, 2 or 3");
    }
    return P2_OK;
}

int p2_get_procrustes(p2_ctx *c, int64_t k0, int64_t k1, float *T) {
    P2_TRY(check_ready(c, true));
    if (k0 < 0 || k1 < k0 || k1 > c->X.K) return fail(P2_EINVAL, "p2_get_procrustes: bad range");
    if (k1 > k0 && !T) return fail(P2_EINVAL, "p2_get_procrustes: NULL out");
    P2_CUDA_TRY(cudaSetDevice(c->opt.device));
    P2_CUDA_TRY(cudaStreamSynchronize(c->stream));
    const size_t RR = (size_t)c->R * c->R;
    if (k1 > k0)
        P2_CUDA_TRY(cudaMemcpy(T, c->d_T + (size_t)k0 * RR, sizeof(float) * RR * (size_t)(k1 - k0),
                               cudaMemcpyDeviceToHost));
    return P2_OK;
}

int p2_get_U(p2_ctx *c, int64_t k0, int64_t k1, float *U) {
    P2_TRY(check_ready(c, true));
    if (k0 < 0 || k1 < k0 || k1 > c->X.K) return fail(P2_EINVAL, "p2_get_U: bad range");
    P2_CUDA_TRY(cudaSetDevice(c->opt.device));
    P2_CUDA_TRY(cudaStreamSynchronize(c->stream));
    int64_t rr[2] = {0, 0};
    P2_CUDA_TRY(cudaMemcpy(&rr[0], c->X.subj_row + k0, sizeof(int64_t), cudaMemcpyDeviceToHost));
    P2_CUDA_TRY(cudaMemcpy(&rr[1], c->X.subj_row + k1, sizeof(int64_t), cudaMemcpyDeviceToHost));
    const int64_t n = rr[1] - rr[0];
    if (n == 0) return P2_OK;
    if (!U) return fail(P2_EINVAL, "p2_get_U: NULL out");
    float *d = nullptr;
    const size_t bytes = sizeof(float) * (size_t)n * c->R;
    P2_CUDA_TRY(cudaMalloc(&d, bytes));
    cudaError_t e = cudaMemsetAsync(d, 0, bytes, c->stream);     // rows of empty subjects stay 0
    if (e == cudaSuccess) e = launch_get_u(c, k0, k1, rr[0], d);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e == cudaSuccess) e = cudaMemcpy(U, d, bytes, cudaMemcpyDeviceToHost);
    cudaFree(d);
    if (e != cudaSuccess) {
        set_error("p2_get_U: %s", cudaGetErrorString(e));
        return P2_ECUDA;
    }
    return P2_OK;
}

int p2_iterate_until(p2_ctx *c, int32_t max_iter, double tol, int32_t *n_done,
                     double *fit_out) {
    if (n_done) *n_done = 0;
    if (max_iter < 0 || !(tol >= 0.0)) return fail(P2_EINVAL, "p2_iterate_until: bad max_iter or tol");
    double prev = 0.0, fit = 0.0;
    int32_t it = 0;
    while (it < max_iter) {
        P2_TRY(p2_iterate(c, 1, &fit));
        ++it;
        if (n_done) *n_done = it;
        if (fit_out) *fit_out = fit;
        if (it > 1 && fabs(fit - prev) <= tol) break;
        prev = fit;
    }
    return P2_OK;
}

int p2_stats(p2_ctx *c, p2_stats_t *out) {
    if (!c || !out) return fail(P2_EINVAL, "NULL argument");
    memset(out, 0, sizeof(*out));
    P2_CUDA_TRY(cudaSetDevice(c->opt.device));
    P2_CUDA_TRY(cudaStreamSynchronize(c->stream));
    out->kernel_launches = c->enqueued;
    out->iterations = c->iters_done;
    if (c->d_s) {
        unsigned long long fl = 0;
        P2_CUDA_TRY(cudaMemcpy(&fl, &c->d_s->polar_flops, sizeof(fl), cudaMemcpyDeviceToHost));
        out->polar_fp64_flops = (double)fl;
    }
    if (c->opt.timing && c->iters_done > 0) {
        out->n_phases = 7;
        for (int i = 0; i < 7; ++i) {
            float ms = -1.f;
            if (cudaEventElapsedTime(&ms, c->ev[i], c->ev[i + 1]) != cudaSuccess) {
                cudaGetLastError();
                ms = -1.f;
            }
            out->phase_ms[i] = ms;
        }
    }
    return P2_OK;
}

int p2_device_bytes(p2_ctx *c, int64_t *bytes) {
    if (!c || !bytes) return fail(P2_EINVAL, "NULL argument");
    *bytes = (int64_t)c->dev_bytes;
    return P2_OK;
}

const char *p2_last_error(void) { return g_err; }

}  // extern "C"
