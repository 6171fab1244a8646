// Projection of new subjects onto a fixed model (serving).
//
// For each new subject X (I x J) with the model's H and V fixed, alternate
// Algorithm 2's Q-step (Procrustes on X V S H^T, Section 3.2) and Algorithm
// 1's W update for that one subject (mode-3 MTTKRP, Eq. mttkrp3_row_wise,
// times (V^TV * H^TH)^+), starting from s = 1.  With V fixed, Z = X V and its
// Gram G are computed once; every later step is R x R work per subject:
//   T = C H S (Procrustes, FP64),  Y V = T G,  m3 = coldot(H, T G),
//   s = m3 (V^TV * H^TH)^+ (FP64).
// Subjects are independent, so a subject's result does not depend on the
// batch it is in.  A projector owns its stream and scratch, so several
// projectors overlap their batches on the device.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <string.h>

#include "p2_internal.cuh"

struct p2_projector {
    p2_ctx *model = nullptr;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    int64_t cap_k = 0, cap_rows = 0, cap_nnz = 0;
    // raw batch copies
    int64_t *d_sp = nullptr, *d_rp = nullptr;
    int32_t *d_col32 = nullptr;
    // internal format
    p2::DevX X;
    // per subject
    p2::dw *d_G = nullptr;
    float *d_S = nullptr, *d_T = nullptr;
    float *d_M3 = nullptr;              // non-negative models: the subjects' mode-3 rows
    uint64_t *d_pass = nullptr;         // non-negative models: NNLS passive sets
    p2::SmallState *d_st = nullptr;     // private copy of H64, G3inv; flags
    int pending_flags_check = 0;
};

namespace p2 {

#define FULLMASK 0xffffffffu

// batch CSR -> internal format, relabelled by the model's column permutation
__global__ void k_proj_rows(const int64_t *__restrict__ rp, const int32_t *__restrict__ col,
                            const int32_t *__restrict__ perm, int64_t N, int64_t nnz, int32_t J,
                            uint16_t *row_len, uint16_t *col16, SmallState *st) {
    int fl = 0;
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < N;
         r += (int64_t)gridDim.x * blockDim.x) {
        const int64_t b = rp[r], e = rp[r + 1];
        if (b < 0 || e > nnz || e < b || e - b > 65535) {
            fl |= FLAG_BAD_PTR;
            row_len[r] = 0;
            continue;
        }
        row_len[r] = (uint16_t)(e - b);
        int prev = -1;
        for (int64_t i = b; i < e; ++i) {
            const int j = col[i];
            if (j < 0 || j >= J || j <= prev) {
                fl |= FLAG_BAD_COL;
                col16[i] = 0;
            } else {
                col16[i] = (uint16_t)perm[j];
            }
            prev = j;
        }
    }
    if (fl) atomicOr(&st->flags, fl);
}

__global__ void k_proj_subjects(const int64_t *__restrict__ sp, const int64_t *__restrict__ rp,
                                int64_t K, int64_t N, int64_t *subj_row, int64_t *subj_nnz,
                                float *S, int R, SmallState *st) {
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k <= K;
         k += (int64_t)gridDim.x * blockDim.x) {
        int64_t a = sp[k];
        if (a < 0 || a > N || (k < K && sp[k + 1] < a)) {
            atomicOr(&st->flags, FLAG_BAD_PTR);
            a = a < 0 ? 0 : (a > N ? N : a);
        }
        subj_row[k] = a;
        subj_nnz[k] = rp[a];
        if (k < K)
            for (int r = 0; r < R; ++r) S[(size_t)k * R + r] = 1.0f;
    }
}

// s <- coldot(H, T G) (V^TV * H^TH)^+ for every subject; one warp per subject.
// M3 (nullable) receives the rows coldot(H, T G) (the non-negative variant
// solves s from them afterwards).
__global__ void __launch_bounds__(256) k_proj_update(const float *__restrict__ T,
                                                     const dw *__restrict__ G,
                                                     const float *__restrict__ H,
                                                     const SmallState *__restrict__ st, float *S,
                                                     float *M3, int64_t K, int R) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int P = R * (R + 1) / 2;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    double *G3s = reinterpret_cast<double *>(smem_raw);           // R R
    float *Hs = reinterpret_cast<float *>(G3s + R * R);           // R R
    float *wb = Hs + R * R + warp * (3 * R * R + R);
    float *Ts = wb, *Gs = wb + R * R, *Pr = wb + 2 * R * R, *m3 = wb + 3 * R * R;
    for (int i = threadIdx.x; i < R * R; i += blockDim.x) {
        G3s[i] = st->G3inv[i];
        Hs[i] = H[i];
    }
    __syncthreads();
    const int64_t nwarps = (int64_t)gridDim.x * nw;
    for (int64_t k = (int64_t)blockIdx.x * nw + warp; k < K; k += nwarps) {
        const float *Tg = T + (size_t)k * R * R;
        const dw *Gg = G + (size_t)k * P;
        for (int e = lane; e < R * R; e += 32) Ts[e] = Tg[e];
        for (int p = lane; p < P; p += 32) {
            int r = (int)((sqrt(8.0 * p + 1.0) - 1.0) * 0.5);
            while ((r + 1) * (r + 2) / 2 <= p) ++r;
            while (r * (r + 1) / 2 > p) --r;
            const int c = p - r * (r + 1) / 2;
            const float g = Gg[p].h;
            Gs[r * R + c] = g;
            Gs[c * R + r] = g;
        }
        __syncwarp();
        for (int e = lane; e < R * R; e += 32) {
            const int r = e / R, c = e - r * R;
            float b = 0.f;
            for (int u = 0; u < R; ++u) b = fmaf(Ts[r * R + u], Gs[u * R + c], b);
            Pr[e] = Hs[e] * b;
        }
        __syncwarp();
        for (int c = lane; c < R; c += 32) {
            float m = 0.f;
            for (int r = 0; r < R; ++r) m += Pr[r * R + c];
            m3[c] = m;
            if (M3) M3[(size_t)k * R + c] = m;
        }
        __syncwarp();
        for (int c = lane; c < R; c += 32) {
            double w = 0.0;
            for (int u = 0; u < R; ++u) w = fma((double)m3[u], G3s[u * R + c], w);
            S[(size_t)k * R + c] = (float)w;
        }
        __syncwarp();
    }
}

}  // namespace p2

using namespace p2;

namespace {

int proj_fail(int code, const char *msg) {
    set_error("%s", msg);
    return code;
}

// Host-side validation of a batch given in host memory (so that no kernel
// ever reads outside the batch's arrays).
int validate_host(int64_t K, int32_t J, const int64_t *sp, const int64_t *rp, const int32_t *col,
                  const float *val, int64_t N, int64_t nnz) {
    for (int64_t k = 0; k < K; ++k)
        if (sp[k + 1] < sp[k]) return proj_fail(P2_EINVAL, "p2_project: subj_ptr not non-decreasing");
    for (int64_t r = 0; r < N; ++r) {
        const int64_t b = rp[r], e = rp[r + 1];
        if (e < b || b < 0 || e > nnz || e - b > 65535)
            return proj_fail(P2_EINVAL, "p2_project: bad row_ptr or a row longer than 65535");
        int prev = -1;
        for (int64_t i = b; i < e; ++i) {
            if (col[i] < 0 || col[i] >= J || col[i] <= prev)
                return proj_fail(P2_EINVAL, "p2_project: column out of range or not increasing");
            if (!(val[i] - val[i] == 0.0f)) return proj_fail(P2_EINVAL, "p2_project: non-finite value");
            prev = col[i];
        }
    }
    return P2_OK;
}

template <class T>
cudaError_t palloc(T **p, size_t n) {
    return cudaMalloc((void **)p, sizeof(T) * (n > 0 ? n : 1));
}

void proj_free(p2_projector *pj) {
    cudaFree(pj->d_sp);
    cudaFree(pj->d_rp);
    cudaFree(pj->d_col32);
    cudaFree(pj->X.subj_row);
    cudaFree(pj->X.subj_nnz);
    cudaFree(pj->X.row_len);
    cudaFree(pj->X.col);
    cudaFree(pj->X.val);
    cudaFree(pj->d_G);
    cudaFree(pj->d_S);
    cudaFree(pj->d_M3);
    cudaFree(pj->d_pass);
    cudaFree(pj->d_T);
    cudaFree(pj->d_st);
}

}  // namespace

extern "C" {

int p2_projector_bytes(p2_ctx *model, int64_t max_subjects, int64_t max_rows, int64_t max_nnz,
                       int64_t *bytes) {
    if (!model || !bytes) return proj_fail(P2_EINVAL, "p2_projector_bytes: NULL argument");
    if (max_subjects < 1 || max_rows < 0 || max_nnz < 0)
        return proj_fail(P2_EINVAL, "p2_projector_bytes: bad capacity");
    const int64_t R = model->R, P = model->P;
    // the allocations of p2_projector_create, element by element
    int64_t per_subject = 8 + 8 + 8 + (int64_t)sizeof(dw) * P + 4 * R + 4 * R * R;
    if (model->opt.nonneg) per_subject += 4 * R + 8;
    *bytes = per_subject * max_subjects + 3 * 8 + (8 + 2) * max_rows + 8 +
             (4 + 2 + 4) * max_nnz + (int64_t)sizeof(SmallState);
    return P2_OK;
}

int p2_projector_create(p2_ctx *model, int64_t max_subjects, int64_t max_rows, int64_t max_nnz,
                        void *stream, p2_projector **out) {
    if (!out) return proj_fail(P2_EINVAL, "p2_projector_create: NULL out");
    *out = nullptr;
    if (!model) return proj_fail(P2_EINVAL, "p2_projector_create: NULL model");
    if (!model->loaded || !model->inited)
        return proj_fail(P2_ESTATE, "p2_projector_create: the model has no factors yet");
    if (max_subjects < 1 || max_rows < 0 || max_nnz < 0 || max_rows >= (1LL << 31) ||
        max_nnz >= (1LL << 31))
        return proj_fail(P2_EINVAL, "p2_projector_create: bad capacity");
    P2_CUDA_TRY(cudaSetDevice(model->opt.device));
    p2_projector *pj = new p2_projector();
    pj->model = model;
    pj->cap_k = max_subjects;
    pj->cap_rows = max_rows;
    pj->cap_nnz = max_nnz;
    const int R = model->R, P = model->P;
    cudaError_t e = cudaSuccess;
    if (stream) {
        pj->stream = (cudaStream_t)stream;
    } else {
        e = cudaStreamCreateWithFlags(&pj->stream, cudaStreamNonBlocking);
        pj->own_stream = true;
    }
    if (e == cudaSuccess) e = palloc(&pj->d_sp, max_subjects + 1);
    if (e == cudaSuccess) e = palloc(&pj->d_rp, max_rows + 1);
    if (e == cudaSuccess) e = palloc(&pj->d_col32, max_nnz);
    if (e == cudaSuccess) e = palloc(&pj->X.subj_row, max_subjects + 1);
    if (e == cudaSuccess) e = palloc(&pj->X.subj_nnz, max_subjects + 1);
    if (e == cudaSuccess) e = palloc(&pj->X.row_len, max_rows);
    if (e == cudaSuccess) e = palloc(&pj->X.col, max_nnz);
    if (e == cudaSuccess) e = palloc(&pj->X.val, max_nnz);
    if (e == cudaSuccess) e = palloc(&pj->d_G, (size_t)max_subjects * P);
    if (e == cudaSuccess) e = palloc(&pj->d_S, (size_t)max_subjects * R);
    if (e == cudaSuccess && model->opt.nonneg) e = palloc(&pj->d_M3, (size_t)max_subjects * R);
    if (e == cudaSuccess && model->opt.nonneg) e = palloc(&pj->d_pass, (size_t)max_subjects);
    if (e == cudaSuccess) e = palloc(&pj->d_T, (size_t)max_subjects * R * R);
    if (e == cudaSuccess) e = palloc(&pj->d_st, 1);
    if (e == cudaSuccess) e = cudaMemsetAsync(pj->d_st, 0, sizeof(SmallState), pj->stream);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_proj_update, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                   model->geo.smem_optin);
    if (e != cudaSuccess) {
        cudaGetLastError();
        proj_free(pj);
        if (pj->own_stream && pj->stream) cudaStreamDestroy(pj->stream);
        delete pj;
        set_error("p2_projector_create: %s", cudaGetErrorString(e));
        return e == cudaErrorMemoryAllocation ? P2_ENOMEM : P2_ECUDA;
    }
    *out = pj;
    return P2_OK;
}

int p2_projector_destroy(p2_projector *pj) {
    if (!pj) return P2_OK;
    cudaSetDevice(pj->model->opt.device);
    if (pj->stream) cudaStreamSynchronize(pj->stream);
    proj_free(pj);
    if (pj->own_stream && pj->stream) cudaStreamDestroy(pj->stream);
    delete pj;
    return P2_OK;
}

int p2_project(p2_projector *pj, int64_t n_req, const int64_t *subj_ptr, const int64_t *row_ptr,
               const int32_t *col, const float *val, int32_t location, int32_t n_iter,
               float *S_out, float *T_out, int32_t out_location) {
    if (!pj) return proj_fail(P2_EINVAL, "p2_project: NULL projector");
    p2_ctx *m = pj->model;
    if (n_req < 1 || n_req > pj->cap_k) return proj_fail(P2_EINVAL, "p2_project: n_req outside [1, capacity]");
    if (n_iter < 1) return proj_fail(P2_EINVAL, "p2_project: n_iter < 1");
    if (!subj_ptr || !row_ptr || !S_out) return proj_fail(P2_EINVAL, "p2_project: NULL pointer");
    if (location != 0 && location != 1) return proj_fail(P2_EINVAL, "p2_project: bad location");
    if (out_location != 0 && out_location != 1) return proj_fail(P2_EINVAL, "p2_project: bad out_location");
    P2_CUDA_TRY(cudaSetDevice(m->opt.device));
    cudaStream_t s = pj->stream;
    int64_t s0 = 0, N = 0, r0 = 0, nnz = 0;
    if (location == 0) {
        s0 = subj_ptr[0];
        N = subj_ptr[n_req];
    } else {
        P2_CUDA_TRY(cudaMemcpy(&s0, subj_ptr, 8, cudaMemcpyDeviceToHost));
        P2_CUDA_TRY(cudaMemcpy(&N, subj_ptr + n_req, 8, cudaMemcpyDeviceToHost));
    }
    if (s0 != 0 || N < 0 || N > pj->cap_rows)
        return proj_fail(P2_EINVAL, "p2_project: subj_ptr[0] must be 0 and the rows fit the capacity");
    if (location == 0) {
        r0 = row_ptr[0];
        nnz = row_ptr[N];
    } else {
        P2_CUDA_TRY(cudaMemcpy(&r0, row_ptr, 8, cudaMemcpyDeviceToHost));
        P2_CUDA_TRY(cudaMemcpy(&nnz, row_ptr + N, 8, cudaMemcpyDeviceToHost));
    }
    if (r0 != 0 || nnz < 0 || nnz > pj->cap_nnz)
        return proj_fail(P2_EINVAL, "p2_project: row_ptr[0] must be 0 and the non-zeros fit the capacity");
    if (nnz > 0 && (!col || !val)) return proj_fail(P2_EINVAL, "p2_project: NULL col/val");
    if (location == 0) {
        const int rc = validate_host(n_req, m->X.J, subj_ptr, row_ptr, col, val, N, nnz);
        if (rc != P2_OK) return rc;
    }
    const cudaMemcpyKind kin = location == 0 ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
    const cudaMemcpyKind kout = out_location == 0 ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
    const int R = m->R;
    const int nsm = m->geo.nsm;
    // inputs, and a private copy of the model's H64 / G3inv for this batch
    P2_CUDA_TRY(cudaMemcpyAsync(pj->d_sp, subj_ptr, 8 * (size_t)(n_req + 1), kin, s));
    P2_CUDA_TRY(cudaMemcpyAsync(pj->d_rp, row_ptr, 8 * (size_t)(N + 1), kin, s));
    if (nnz > 0) {
        P2_CUDA_TRY(cudaMemcpyAsync(pj->d_col32, col, 4 * (size_t)nnz, kin, s));
        P2_CUDA_TRY(cudaMemcpyAsync(pj->X.val, val, 4 * (size_t)nnz, kin, s));
    }
    P2_CUDA_TRY(cudaMemcpyAsync(pj->d_st->H64, m->d_s->H64, sizeof(double) * P2_RMAX * P2_RMAX,
                                cudaMemcpyDeviceToDevice, s));
    P2_CUDA_TRY(cudaMemcpyAsync(pj->d_st->G3inv, m->d_s->G3inv, sizeof(double) * P2_RMAX * P2_RMAX,
                                cudaMemcpyDeviceToDevice, s));
    // convert
    if (N > 0)
        k_proj_rows<<<4 * nsm, 256, 0, s>>>(pj->d_rp, pj->d_col32, m->d_perm_old2new, N, nnz,
                                            m->X.J, pj->X.row_len, pj->X.col, pj->d_st);
    k_proj_subjects<<<(int)((n_req + 256) / 256), 256, 0, s>>>(pj->d_sp, pj->d_rp, n_req, N,
                                                               pj->X.subj_row, pj->X.subj_nnz,
                                                               pj->d_S, R, pj->d_st);
    P2_CUDA_TRY(cudaGetLastError());
    if (location == 1) {
        // device input: check the validation flags before any kernel reads the batch
        int flags = 0;
        P2_CUDA_TRY(cudaMemcpyAsync(&flags, &pj->d_st->flags, sizeof(int), cudaMemcpyDeviceToHost, s));
        P2_CUDA_TRY(cudaStreamSynchronize(s));
        if (flags & (FLAG_BAD_PTR | FLAG_BAD_COL)) {
            int zero = 0;
            cudaMemcpy(&pj->d_st->flags, &zero, sizeof(int), cudaMemcpyHostToDevice);
            return proj_fail(P2_EINVAL, "p2_project: malformed request slices");
        }
    }
    pj->X.K = n_req;
    pj->X.N = N;
    pj->X.nnz = nnz;
    XView xv{pj->X.subj_row, pj->X.subj_nnz, pj->X.row_len, pj->X.col, pj->X.val, n_req};
    P2_CUDA_TRY(launch_gram(m, xv, pj->d_st, pj->d_G, s));
    if (m->opt.nonneg)
        P2_CUDA_TRY(cudaMemsetAsync(pj->d_pass, 0, sizeof(uint64_t) * (size_t)n_req, s));
    int uw = 8;
    while (uw > 1 && (size_t)R * R * 12 + uw * (size_t)(3 * R * R + R) * 4 > (size_t)m->geo.smem_optin) --uw;
    const size_t upd_smem = (size_t)R * R * 12 + uw * (size_t)(3 * R * R + R) * 4;
    const int ub = (int)((n_req + uw - 1) / uw < 16 * (int64_t)nsm ? (n_req + uw - 1) / uw : 16 * (int64_t)nsm);
    for (int it = 0; it < n_iter; ++it) {
        P2_CUDA_TRY(launch_polar_on(m, pj->d_G, pj->d_S, pj->d_st, pj->d_T, n_req, s));
        k_proj_update<<<ub, uw * 32, upd_smem, s>>>(pj->d_T, pj->d_G, m->d_H, pj->d_st, pj->d_S,
                                                    pj->d_M3, n_req, R);
        P2_CUDA_TRY(cudaGetLastError());
        if (m->opt.nonneg)          // the model's S_k are non-negative: s by NNLS (Section 5.1)
            P2_CUDA_TRY(launch_nnls_rows(m, state_vtv(m), state_hth(m), pj->d_M3, n_req,
                                         pj->d_pass, pj->d_S, s));
    }
    if (T_out) P2_CUDA_TRY(launch_polar_on(m, pj->d_G, pj->d_S, pj->d_st, pj->d_T, n_req, s));
    P2_CUDA_TRY(cudaMemcpyAsync(S_out, pj->d_S, sizeof(float) * (size_t)n_req * R, kout, s));
    if (T_out)
        P2_CUDA_TRY(cudaMemcpyAsync(T_out, pj->d_T, sizeof(float) * (size_t)n_req * R * R, kout, s));
    pj->pending_flags_check = 1;
    return P2_OK;
}

int p2_projector_sync(p2_projector *pj) {
    if (!pj) return proj_fail(P2_EINVAL, "p2_projector_sync: NULL projector");
    P2_CUDA_TRY(cudaSetDevice(pj->model->opt.device));
    int flags = 0;
    P2_CUDA_TRY(cudaMemcpyAsync(&flags, &pj->d_st->flags, sizeof(int), cudaMemcpyDeviceToHost,
                                pj->stream));
    P2_CUDA_TRY(cudaStreamSynchronize(pj->stream));
    if (flags & (FLAG_BAD_PTR | FLAG_BAD_COL)) {
        int zero = 0;
        cudaMemcpy(&pj->d_st->flags, &zero, sizeof(int), cudaMemcpyHostToDevice);
        set_error("p2_project: malformed request slices (flags 0x%x); results are not valid", flags);
        return P2_EINVAL;
    }
    return P2_OK;
}

}  // extern "C"
