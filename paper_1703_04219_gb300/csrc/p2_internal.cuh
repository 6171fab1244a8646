// Internal declarations shared by the translation units of libp2.so.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>
#include <string>
#include <vector>

#include "../../include/p2.h"
#include "p2_dw.cuh"

#define P2_RMAX 64

namespace p2 {

// error flags raised by kernels (bit mask in ctx device memory)
enum : int {
    FLAG_BAD_PTR = 1,        // non-monotone subject/row pointers or row longer than 65535
    FLAG_BAD_COL = 2,        // column out of range or not strictly increasing in a row
    FLAG_BAD_VAL = 4,        // non-finite value
    FLAG_EIG_NOCONV = 8,     // an eigen iteration hit its step limit
    FLAG_NONFINITE = 32,     // non-finite loss / factor
    FLAG_TC_TIMEOUT = 64,    // a tensor-core MMA did not complete within its wait limit
};

void set_error(const char *fmt, ...);

#define P2_CUDA_TRY(call)                                                                  \
    do {                                                                                   \
        cudaError_t _e = (call);                                                           \
        if (_e != cudaSuccess) {                                                           \
            ::p2::set_error("%s failed: %s (%s:%d)", #call, cudaGetErrorString(_e),      \
                            __FILE__, __LINE__);                                           \
            return P2_ECUDA;                                                               \
        }                                                                                  \
    } while (0)

// Small FP64 state that lives in device memory (one copy per context).
struct SmallState {
    double M1[P2_RMAX * P2_RMAX];       // mode-1 MTTKRP used by the last H solve
    double WtW[P2_RMAX * P2_RMAX];
    double VtV[P2_RMAX * P2_RMAX];
    double HtH[P2_RMAX * P2_RMAX];
    double H64[P2_RMAX * P2_RMAX];      // FP32 H widened to FP64
    double P2inv[P2_RMAX * P2_RMAX];    // (W^TW * H^TH)^+ for the V solve
    double G3inv[P2_RMAX * P2_RMAX];    // (V^TV * H^TH)^+ for the W solve
    double colnorm[P2_RMAX];            // column norms of the unnormalised V
    double wm3;                          // <W, M3>
    double loss;
    double fit;
    double normx2;                       // ||X||_F^2
    unsigned long long polar_flops;     // FP64 flops executed by k_polar (running total)
    int flags;
    int iter;
};

// Storage type of V and of the mode-2 rows P: float (P2_FP32) or bfloat16
// (P2_BF16, round to nearest even); arithmetic is FP32 in both cases.
typedef __nv_bfloat16 bf16_t;
template <class S> struct Stor;
template <> struct Stor<float> {
    static __device__ __forceinline__ float ld(const float *p) { return __ldg(p); }
    static __device__ __forceinline__ float ldp(const float *p) { return *p; }
    static __device__ __forceinline__ void st(float *p, float v) { *p = v; }
};
template <> struct Stor<bf16_t> {
    static __device__ __forceinline__ float ld(const bf16_t *p) { return __bfloat162float(__ldg(p)); }
    static __device__ __forceinline__ float ldp(const bf16_t *p) { return __bfloat162float(*p); }
    static __device__ __forceinline__ void st(bf16_t *p, float v) { *p = __float2bfloat16_rn(v); }
};

// Row stride of V (and Vprev) in device memory: R rounded up so that a row
// is a whole number of 16-byte vectors; the padding is zero.
template <class S> __host__ __device__ inline int v_stride(int R);
template <> __host__ __device__ inline int v_stride<float>(int R) { return (R + 3) & ~3; }
template <> __host__ __device__ inline int v_stride<bf16_t>(int R) { return (R + 7) & ~7; }

// Device-resident sparse slices in the internal format.
struct DevX {
    int64_t K = 0, N = 0, nnz = 0;
    int32_t J = 0;
    int64_t *subj_row = nullptr;   // [K+1] row offsets
    int64_t *subj_nnz = nullptr;   // [K+1] non-zero offsets
    uint16_t *row_len = nullptr;   // [N]
    uint16_t *col = nullptr;       // [nnz] relabelled column ids
    float *val = nullptr;          // [nnz]
    // column-major copy for the mode-2 reduction (built once at load)
    uint32_t *csc_row = nullptr;   // [nnz] stacked row id of each non-zero, column-major
    float *csc_val = nullptr;      // [nnz]
    int64_t nseg = 0;              // column segments of at most P2_SEG non-zeros
    int64_t *seg_start = nullptr;  // [nseg] first non-zero of each segment (offsets into csc_*)
    int64_t *seg_end = nullptr;    // [nseg] one past its last
    // The mode-2 pass runs over row blocks (whole subjects, P rows of one block
    // sized to stay in L2): a column's non-zeros, sorted by row, fall into one
    // run per block, cut into segments; segments are numbered block by block.
    int64_t *col_seg = nullptr;    // [nblk J + 1] first segment of (block b, column j) at b J + j
    int32_t nblk = 1;
    int64_t p_rows = 0;            // rows of the P buffer: the largest block
    std::vector<int64_t> blk_subj; // host [nblk+1]: first subject of each block
    std::vector<int64_t> blk_row;  // host [nblk+1]: first stacked row of each block
    std::vector<int64_t> blk_seg;  // host [nblk+1]: first segment of each block
};

#define P2_SEG 1024

// Read-only view of slices in the internal format, passed to kernels by value.
struct XView {
    const int64_t *__restrict__ subj_row;
    const int64_t *__restrict__ subj_nnz;
    const uint16_t *__restrict__ row_len;
    const uint16_t *__restrict__ col;
    const float *__restrict__ val;
    int64_t K;
    // processing order of the subjects (position i handles subject order[i]);
    // NULL: natural order
    const int32_t *__restrict__ order = nullptr;
};

// Launch geometry decided once per context.
struct Geometry {
    int nsm = 0;
    int smem_optin = 0;
    int red_blocks = 0;     // blocks of the grid reductions (fixed => deterministic)
};

// device memory of a context (its stream-ordered pool, p2_api.cu)
cudaError_t ctx_malloc(const struct ::p2_ctx *c, void **p, size_t bytes);
void ctx_free(const struct ::p2_ctx *c, void *p);

// kernel launchers (defined in the .cu files)
int launch_load(struct ::p2_ctx *ctx, const int64_t *d_subj_ptr, const int64_t *d_row_ptr,
                const int32_t *d_col, const float *d_val, int64_t K, int32_t J, int64_t N,
                int64_t nnz);

}  // namespace p2

struct p2_ctx {
    p2_options opt;
    int R = 0;
    int P = 0;                      // R(R+1)/2
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    cudaMemPool_t pool = nullptr;   // the context's device memory (ctx_malloc)
    p2::Geometry geo;

    p2::DevX X;
    bool loaded = false;
    int32_t *d_perm_old2new = nullptr;   // [J]
    int32_t *h_perm_new2old = nullptr;   // host [J]
    int32_t *h_perm_old2new = nullptr;   // host [J]

    // factors and per-subject state
    // Storage of V, Vprev and P follows opt.precision: the float pointers are
    // used with P2_FP32, the *h (bfloat16) ones with P2_BF16; the others stay
    // null.  H (R x R) and T_k are float in both modes: H is too small for its
    // storage to matter, and Q_k = Z_k T_k^T is formed from T_k with a
    // cancellation that amplifies its rounding by cond(A_k).
    bool bf16 = false;
    float *d_H = nullptr;       // R x R
    float *d_V = nullptr;       // J x R (relabelled rows)
    float *d_Vprev = nullptr;   // J x R
    p2::bf16_t *d_Vh = nullptr, *d_Vprevh = nullptr, *d_Ph = nullptr;
    float *d_W = nullptr;       // K x R
    float *d_T = nullptr;       // K x R x R
    p2::dw *d_G = nullptr;      // K x P packed lower Gram of Z_k, double-word (hi + lo)
    float *d_Gf = nullptr;      // K x P the same rounded to float (mode-1 statistics)
    float *d_M3 = nullptr;      // K x R
    // Q-step order: subjects sorted by the QR rotation count of their previous
    // Q-step, so the lanes of a warp converge after similar numbers of trips
    int32_t *d_qrcnt = nullptr;  // [K] rotations of the last Q-step (0 before the first)
    int32_t *d_order = nullptr;  // [K] subject processed by each Procrustes slot
    int32_t *d_rank = nullptr;   // [K] rank within the subject's bin and chunk
    int32_t *d_binoff = nullptr; // [nchunk x 256] bin counts, then offsets
    // subject bins: the sparse passes take the subjects in decreasing order of
    // their non-zero count (built at load), so every warp of the persistent
    // grid receives an even mix of large and small subjects
    int32_t *d_sorder = nullptr; // [K]
    // non-negative variant: each row's passive set (bit j: x_j > 0) of the last solve
    uint64_t *d_passW = nullptr; // [K]
    uint64_t *d_passV = nullptr; // [J]
    double *d_M2 = nullptr;     // J x R (relabelled rows)
    float *d_P = nullptr;       // N x R rows of P_k = Z_k F_k (mode-2 pass)
    double *d_segpart = nullptr; // nseg x R partial sums of the mode-2 reduction
    double *d_Vun = nullptr;    // J x R unnormalised V
    p2::SmallState *d_s = nullptr;
    double *d_part = nullptr;   // reduction partials (red_blocks x stats_part_stride(R))
    double *d_part2 = nullptr;  // second partial buffer
    int *d_colcount = nullptr;  // [J] (load time)

    // split Procrustes step (R > 12): one chunk's scratch (GrpSplit in
    // p2_polar_grp.cuh, carved by split_scratch), the fallback list
    unsigned char *d_split = nullptr;
    size_t split_bytes = 0;
    int64_t split_chunk = 0, split_cap = 0;
    int32_t *d_split_list = nullptr;
    int32_t *d_split_cnt = nullptr;
    // tensor-core formation of M' (p2_options.tensor_core_m): every subject's
    // packed lower M' (K x P double-words), read by the grouped kernels
    p2::dw *d_Mtc = nullptr;
    p2_tuning tune{1, -1, 0, 0};   // launch choices (p2_set_tuning, the autotuner)
    bool tuned = false;         // the autotuner has run (or read the cache)
    std::string tune_cache;     // opt.tune_cache, copied
    std::string tune_note;      // how the choices were made (p2_tuning_note)

    // subject-sharded form: the caller's exchange hook (NULL: unsharded) and
    // the one-row sum of the statistics partials that it exchanges
    p2_exchange_fn xfn = nullptr;
    void *xuser = nullptr;
    double *d_red = nullptr;    // stats_part_stride(R) doubles

    bool inited = false;
    int iters_done = 0;
    cudaGraphExec_t graph = nullptr;
    int64_t graph_kernels = 0;      // kernels in one captured iteration
    int64_t enqueued = 0;           // kernels enqueued (eager launches and graph replays)
    cudaEvent_t ev[8] = {};         // phase boundaries when opt.timing
    size_t dev_bytes = 0;
};

namespace p2 {
// shared-memory bytes per warp of k_subject_stats (multiple of 16: FP64 first)
static inline __host__ __device__ size_t stats_warp_bytes(int R) {
    return ((size_t)R * R * 16 + ((size_t)2 * R * R + R) * 4 + 15) & ~(size_t)15;
}
// per-subject statistics after the Q-step (p2_kernels.cu): block partials
// [R*R M1][R*R WtW][1 <W,M3>] over fixed contiguous subject ranges;
// stats_part_stride(R) doubles per block (also the per-block size of the
// other partial buffers, which need at most R*R)
static inline __host__ __device__ size_t stats_part_stride(int R) {
    return 2 * (size_t)R * R + 1;
}
__global__ void __launch_bounds__(256) k_subject_stats(const float *__restrict__ T,
                                                       const double *__restrict__ G,
                                                       const float *__restrict__ W,
                                                       const float *__restrict__ M3, double *part,
                                                       int64_t K, int R, int with_m3);
// per-iteration pieces (p2_kernels.cu)
// autotuner trials (p2_kernels.cu): the Q-step, or the mode-2 pass (its
// kernels only), enqueued `reps` times; the fastest time in ms.  Both leave
// the state they feed forward as one run would (the Q-step's T and rotation
// counts; the mode-2 pass's outputs are recomputed by every iteration).
int tune_time_qstep(p2_ctx *c, int reps, float *ms);
int tune_time_mode2(p2_ctx *c, int reps, float *ms);
// exchange hook call of a sharded context (P2_OK if unsharded)
int exchange(p2_ctx *c, double *buf, int64_t count);
int enqueue_prologue(p2_ctx *c);     // Q-step + mode-1 MTTKRP for the current (H, V, W)
int enqueue_iteration(p2_ctx *c);    // one ALS iteration
int enqueue_factor_stats(p2_ctx *c); // HtH, VtV, WtW for freshly set factors
int configure_kernels(p2_ctx *c);    // smem attributes etc.
// rational start (p2_kernels.cu), on FP64 blocks of b columns (J x b,
// row-major, relabelled rows): H = I and W = 1; Y = X^T (X Vd) with the
// product's columns taken CW at a time through Z (N x CW FP64 scratch) and
// seg (nseg x CW FP64 segment partials);
// orthonormal basis of Y's columns into Q, with the subspace distance of the
// leading R columns to Vold when given; Rayleigh-Ritz step (Out = Y U, or,
// final, the sign-fixed Ritz vectors Vd U with the leading R columns stored
// to the device V)
int enqueue_eig_fill(p2_ctx *c);
int enqueue_eig_product(p2_ctx *c, const double *Vd, int b, int CW, double *Z, double *seg,
                        double *Y);
int enqueue_eig_orth(p2_ctx *c, const double *Y, const double *Vold, double *Q, int b,
                     double *dist);
int enqueue_eig_ritz(p2_ctx *c, const double *Y, const double *Vd, double *Out, int b,
                     int final_step);
// Procrustes step (p2_polar.cu)
int polar_configure(p2_ctx *c);
cudaError_t launch_polar(p2_ctx *c);
// subjects in decreasing order of key (chunked counting sort into 256 bins,
// keys clamped to [0, 255]); rank and binoff are scratch of the Q-step order's sizes
cudaError_t launch_order_desc(const int32_t *key, int64_t K, int32_t *rank, int32_t *binoff,
                              int32_t *order, cudaStream_t s);
// subject bins by non-zero count into c->d_sorder (load time)
cudaError_t launch_subject_bins(p2_ctx *c);
cudaError_t launch_polar_on(const p2_ctx *c, const dw *G, const float *W, SmallState *st,
                            float *T, int64_t K, cudaStream_t s, const int32_t *order = nullptr,
                            int32_t *qrcnt = nullptr, const dw *mpre = nullptr);
// subjects per chunk of the ordering kernels (p2_polar.cu)
#define P2_ORDER_CHUNK 4096
#define P2_ORDER_BINS 256
// kernels launch_polar enqueues for this context (the ordering, the optional
// tensor-core formation of M, the Procrustes kernel or the split step's
// kernels per chunk)
int polar_launches(const p2_ctx *c);
// M' = H' S' G' S' H'^T of every subject on the tensor cores (p2_form_tc.cu),
// packed lower double-words, for 13 <= R <= P2_TC_RMAX
#define P2_TC_RMAX 48
bool form_m_tc_supported(int R);
// whether the context's options select the tensor-core formation of M'
bool tc_m_wanted(const p2_ctx *c);
cudaError_t form_m_tc_configure(int R);
cudaError_t launch_form_m_tc(const p2_ctx *c, const dw *G, const float *W, SmallState *st,
                             dw *Mout, int64_t K, cudaStream_t s);
// non-negative variant (p2_nnls.cu): row-wise NNLS for the W and V updates
cudaError_t nnls_configure(int cap);
cudaError_t launch_nnls_w(p2_ctx *c);
cudaError_t launch_nnls_v(p2_ctx *c, double *part, int nparts);
cudaError_t launch_nnls_rows(const p2_ctx *c, const double *Xa, const double *Xb,
                             const float *rows, int64_t n, uint64_t *passive, float *out,
                             cudaStream_t s);
const double *state_vtv(const p2_ctx *c);
const double *state_hth(const p2_ctx *c);
// U_k = Q_k H rows of subjects k0 .. k1-1 into a device FP32 buffer (p2_kernels.cu)
cudaError_t launch_get_u(p2_ctx *c, int64_t k0, int64_t k1, int64_t r0, float *U);
// Gram of Z_k = X_k V for a batch of new subjects (p2_kernels.cu)
cudaError_t launch_gram(const p2_ctx *c, const XView &X, const SmallState *st, dw *G,
                        cudaStream_t s);
// R > 12: grouped Procrustes kernel (p2_polar_grp.cu)
// fp64: the FP64 instances (opt-in FP64 arm) instead of the double-word ones
cudaError_t polar_grp_configure(int cap, bool fp64);
cudaError_t polar_grp_configure_f64(int cap);
cudaError_t launch_polar_grp_f64(const p2_ctx *c, const dw *G, const float *W, SmallState *st,
                                 float *T, int64_t K, cudaStream_t s, double rtol2,
                                 const int32_t *order, int32_t *qrcnt);
// mpre (nullable, double-word instances only): each subject's M' from
// launch_form_m_tc instead of forming it in the kernel
cudaError_t launch_polar_grp(const p2_ctx *c, const dw *G, const float *W, SmallState *st,
                             float *T, int64_t K, cudaStream_t s, double rtol2,
                             const int32_t *order, int32_t *qrcnt, const dw *mpre = nullptr);
}  // namespace p2
