// Loading {X_k}: validation and conversion to the internal streaming format,
// on the device.
//
// Internal format (what the passes stream): per subject int64 row and
// non-zero offsets, per row a uint16 length, per non-zero a uint16 column id
// (relabelled by decreasing column frequency so that the hottest columns are
// the smallest ids) and an FP32 value: 6 bytes per non-zero + 2 per row.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "p2_internal.cuh"

namespace p2 {

struct LoadScratch {
    int flags;
};

__global__ void k_check_subjects(const int64_t *__restrict__ subj_ptr,
                                 const int64_t *__restrict__ row_ptr, int64_t K, int64_t N,
                                 int64_t *subj_row, int64_t *subj_nnz, LoadScratch *ls) {
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k <= K;
         k += (int64_t)gridDim.x * blockDim.x) {
        const int64_t a = subj_ptr[k];
        subj_row[k] = a;
        if (a < 0 || a > N) {
            atomicOr(&ls->flags, FLAG_BAD_PTR);
            subj_nnz[k] = 0;
            continue;
        }
        subj_nnz[k] = row_ptr[a];
        if (k < K && subj_ptr[k + 1] < a) atomicOr(&ls->flags, FLAG_BAD_PTR);
    }
}

// Per row: bounds, strictly increasing columns, finite values; column
// frequencies (a shared-memory histogram per block when J is small, merged
// with one global atomic per touched column; global atomics otherwise).
__global__ void k_check_rows(const int64_t *__restrict__ row_ptr, const int32_t *__restrict__ col,
                             const float *__restrict__ val, int64_t N, int64_t nnz, int32_t J,
                             uint16_t *row_len, int *colcount, LoadScratch *ls, int smem_hist) {
    extern __shared__ int hist[];
    if (smem_hist) {
        for (int j = threadIdx.x; j < J; j += blockDim.x) hist[j] = 0;
        __syncthreads();
    }
    int fl = 0;
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < N;
         r += (int64_t)gridDim.x * blockDim.x) {
        const int64_t b = row_ptr[r], e = row_ptr[r + 1];
        const int64_t len = e - b;
        if (b < 0 || e > nnz || len < 0 || len > 65535) {
            fl |= FLAG_BAD_PTR;
            row_len[r] = 0;
            continue;
        }
        row_len[r] = (uint16_t)len;
        int prev = -1;
        for (int64_t i = b; i < e; ++i) {
            const int j = col[i];
            const float x = val[i];
            if (j < 0 || j >= J || j <= prev) {
                fl |= FLAG_BAD_COL;
            } else if (smem_hist) {
                atomicAdd(&hist[j], 1);
            } else {
                atomicAdd(&colcount[j], 1);
            }
            prev = j;
            if (!isfinite(x)) fl |= FLAG_BAD_VAL;
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) fl |= __shfl_xor_sync(0xffffffffu, fl, o);
    if ((threadIdx.x & 31) == 0 && fl) atomicOr(&ls->flags, fl);
    if (smem_hist) {
        __syncthreads();
        for (int j = threadIdx.x; j < J; j += blockDim.x)
            if (hist[j]) atomicAdd(&colcount[j], hist[j]);
    }
}

// deterministic partial sums of x^2 over fixed non-zero ranges
__global__ void k_sumsq(const float *__restrict__ val, int64_t nnz, double *part) {
    __shared__ double red[256];
    const int64_t per = (nnz + gridDim.x - 1) / gridDim.x;
    const int64_t a = (int64_t)blockIdx.x * per;
    const int64_t b = (a + per < nnz) ? (a + per) : nnz;
    double s = 0.0;
    for (int64_t i = a + threadIdx.x; i < b; i += blockDim.x) {
        const double x = (double)val[i];
        s = fma(x, x, s);
    }
    red[threadIdx.x] = s;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = red[0];
}

__global__ void k_relabel(const int32_t *__restrict__ col, const int32_t *__restrict__ perm,
                          int64_t nnz, uint16_t *col16) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nnz;
         i += (int64_t)gridDim.x * blockDim.x)
        col16[i] = (uint16_t)perm[col[i]];
}

// ---- column-major copy: deterministic counting sort of the non-zeros by column
__global__ void k_rowid(const int64_t *__restrict__ row_ptr, int64_t N, uint32_t *rowid) {
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < N;
         r += (int64_t)gridDim.x * blockDim.x)
        for (int64_t e = row_ptr[r]; e < row_ptr[r + 1]; ++e) rowid[e] = (uint32_t)r;
}

// per-chunk column histogram (integer atomics: order independent)
__global__ void k_chunk_hist(const uint16_t *__restrict__ col, int64_t nnz, int64_t chunk,
                             int32_t J, int *cnt) {
    const int64_t a = (int64_t)blockIdx.x * chunk;
    const int64_t b = (a + chunk < nnz) ? (a + chunk) : nnz;
    int *row = cnt + (size_t)blockIdx.x * J;
    for (int64_t e = a + threadIdx.x; e < b; e += blockDim.x) atomicAdd(&row[col[e]], 1);
}

// counts -> start offsets, column by column, chunks in order
__global__ void k_col_scan(const int64_t *__restrict__ colptr, int nch, int32_t J, int *cnt) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= J) return;
    int run = (int)colptr[j];
    for (int b = 0; b < nch; ++b) {
        const int c = cnt[(size_t)b * J + j];
        cnt[(size_t)b * J + j] = run;
        run += c;
    }
}

// one warp per chunk, non-zeros in order: equal columns inside a group of 32
// get ranks in lane order, so each column keeps increasing non-zero order
__global__ void k_chunk_place(const uint16_t *__restrict__ col, const float *__restrict__ val,
                              const uint32_t *__restrict__ rowid, int64_t nnz, int64_t chunk,
                              int32_t J, int *cnt, uint32_t *csc_row, float *csc_val) {
    const int lane = threadIdx.x & 31;
    const int64_t a = (int64_t)blockIdx.x * chunk;
    const int64_t b = (a + chunk < nnz) ? (a + chunk) : nnz;
    int *off = cnt + (size_t)blockIdx.x * J;
    for (int64_t base = a; base < b; base += 32) {
        const int64_t e = base + lane;
        const bool valid = e < b;
        const int j = valid ? (int)col[e] : 0;
        const unsigned key = valid ? (unsigned)j : (0x10000u + lane);
        const unsigned mask = __match_any_sync(0xffffffffu, key);
        const int rank = __popc(mask & ((1u << lane) - 1u));
        int b0 = 0;
        if (valid) {
            b0 = off[j];
            const int dest = b0 + rank;
            csc_row[dest] = rowid[e];
            csc_val[dest] = val[e];
        }
        __syncwarp();
        if (valid && rank == 0) off[j] = b0 + __popc(mask);
        __syncwarp();
    }
}

// First position of each block's run in each column (the column's non-zeros
// are sorted by stacked row): vstart[j (nblk + 1) + b], b = 0 .. nblk.
__global__ void k_block_runs(const uint32_t *__restrict__ csc_row,
                             const int64_t *__restrict__ colptr,
                             const int64_t *__restrict__ blk_row, int nblk, int32_t J,
                             int64_t *vstart) {
    const int64_t n = (int64_t)J * (nblk + 1);
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t j = t / (nblk + 1);
        const int b = (int)(t - j * (nblk + 1));
        int64_t lo = colptr[j], hi = colptr[j + 1];
        if (b == 0) {
            vstart[t] = lo;
        } else if (b == nblk) {
            vstart[t] = hi;
        } else {
            const uint64_t key = (uint64_t)blk_row[b];
            while (lo < hi) {                      // first row >= the block's first row
                const int64_t mid = lo + (hi - lo) / 2;
                if ((uint64_t)csc_row[mid] < key) lo = mid + 1;
                else hi = mid;
            }
            vstart[t] = lo;
        }
    }
}

// Row blocks of the mode-2 pass: whole subjects, at most `budget` stacked
// rows each (a subject longer than the budget is a block of its own).
static void plan_blocks(const std::vector<int64_t> &subj_row, int64_t budget,
                        std::vector<int64_t> &blk_subj, std::vector<int64_t> &blk_row) {
    const int64_t K = (int64_t)subj_row.size() - 1;
    blk_subj.assign(1, 0);
    blk_row.assign(1, 0);
    int64_t k = 0;
    while (k < K) {
        int64_t e = k + 1;
        while (e < K && subj_row[e + 1] - subj_row[k] <= budget) ++e;
        blk_subj.push_back(e);
        blk_row.push_back(subj_row[e]);
        k = e;
    }
    if (K == 0) {
        blk_subj.push_back(0);
        blk_row.push_back(subj_row.empty() ? 0 : subj_row[0]);
    }
}

static int build_csc(p2_ctx *c, const int64_t *d_row_ptr, const int32_t *h_count_new,
                     int64_t N, int64_t nnz, int32_t J) {
    cudaStream_t s = c->stream;
    const int nsm = c->geo.nsm;
    const int64_t K = c->X.K;
    // column pointers (host; J <= 65535)
    std::vector<int64_t> colptr((size_t)J + 1, 0);
    for (int32_t j = 0; j < J; ++j) colptr[j + 1] = colptr[j] + h_count_new[j];
    // row blocks from the subjects' row offsets
    {
        std::vector<int64_t> sr((size_t)K + 1);
        P2_CUDA_TRY(cudaMemcpyAsync(sr.data(), c->X.subj_row, sizeof(int64_t) * ((size_t)K + 1),
                                    cudaMemcpyDeviceToHost, s));
        P2_CUDA_TRY(cudaStreamSynchronize(s));
        const int64_t elem = c->bf16 ? 2 : 4;
        // m2_block_kib = 0: one block, the whole collection (measured fastest:
        // every extra block adds a pair of launches and their tails, which
        // cost more than the L2 hits on the P rows save)
        int64_t budget = c->tune.m2_block_kib > 0
                             ? ((int64_t)c->tune.m2_block_kib << 10) / (elem * c->R)
                             : (int64_t)N;
        if (budget < 1) budget = 1;
        plan_blocks(sr, budget, c->X.blk_subj, c->X.blk_row);
        c->X.nblk = (int32_t)c->X.blk_subj.size() - 1;
        int64_t rows = 0;
        for (int b = 0; b < c->X.nblk; ++b)
            rows = std::max<int64_t>(rows, c->X.blk_row[b + 1] - c->X.blk_row[b]);
        // the P buffer holds one block
        if (rows < c->X.p_rows) {
            void **pp = c->bf16 ? (void **)&c->d_Ph : (void **)&c->d_P;
            ctx_free(c, *pp);
            *pp = nullptr;
            const size_t ps = c->bf16 ? v_stride<bf16_t>(c->R) : v_stride<float>(c->R);
            c->dev_bytes -= (size_t)c->X.p_rows * ps * elem;
            const cudaError_t e = ctx_malloc(c, pp, (size_t)(rows > 0 ? rows : 1) * ps * elem);
            if (e != cudaSuccess) {
                cudaGetLastError();
                c->X.p_rows = 0;
                set_error("load: allocation of the mode-2 rows failed: %s", cudaGetErrorString(e));
                return e == cudaErrorMemoryAllocation ? P2_ENOMEM : P2_ECUDA;
            }
            c->X.p_rows = rows;
            c->dev_bytes += (size_t)rows * ps * elem;
        }
    }
    const int nblk = c->X.nblk;
    cudaError_t e = ctx_malloc(c, (void **)&c->X.csc_row, sizeof(uint32_t) * (nnz > 0 ? nnz : 1));
    if (e == cudaSuccess) e = ctx_malloc(c, (void **)&c->X.csc_val, sizeof(float) * (nnz > 0 ? nnz : 1));
    if (e != cudaSuccess) {
        cudaGetLastError();
        set_error("load: allocation of the column-major copy failed: %s", cudaGetErrorString(e));
        return e == cudaErrorMemoryAllocation ? P2_ENOMEM : P2_ECUDA;
    }
    c->dev_bytes += (sizeof(uint32_t) + sizeof(float)) * (size_t)nnz;
    std::vector<int64_t> vstart((size_t)J * (nblk + 1), 0);
    if (nnz > 0) {
        // chunking keeps the per-chunk count matrix near 256 MB at most
        int64_t nch = (nnz + 65535) / 65536;
        const int64_t maxch = (256ll << 20) / (4ll * J);
        if (nch > maxch) nch = maxch > 0 ? maxch : 1;
        const int64_t chunk = (nnz + nch - 1) / nch;
        nch = (nnz + chunk - 1) / chunk;
        int64_t *d_colptr = nullptr, *d_blkrow = nullptr, *d_vstart = nullptr;
        uint32_t *d_rowid = nullptr;
        int *d_cnt = nullptr;
        e = ctx_malloc(c, (void **)&d_colptr, sizeof(int64_t) * ((size_t)J + 1));
        if (e == cudaSuccess) e = ctx_malloc(c, (void **)&d_rowid, sizeof(uint32_t) * (size_t)nnz);
        if (e == cudaSuccess) e = ctx_malloc(c, (void **)&d_cnt, sizeof(int) * (size_t)nch * J);
        if (e == cudaSuccess) e = ctx_malloc(c, (void **)&d_blkrow, sizeof(int64_t) * ((size_t)nblk + 1));
        if (e == cudaSuccess) e = ctx_malloc(c, (void **)&d_vstart, sizeof(int64_t) * vstart.size());
        if (e == cudaSuccess) e = cudaMemcpyAsync(d_colptr, colptr.data(), sizeof(int64_t) * ((size_t)J + 1),
                                                  cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(d_blkrow, c->X.blk_row.data(),
                                                  sizeof(int64_t) * ((size_t)nblk + 1),
                                                  cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess) e = cudaMemsetAsync(d_cnt, 0, sizeof(int) * (size_t)nch * J, s);
        if (e == cudaSuccess) {
            k_rowid<<<8 * nsm, 256, 0, s>>>(d_row_ptr, N, d_rowid);
            k_chunk_hist<<<(int)nch, 256, 0, s>>>(c->X.col, nnz, chunk, J, d_cnt);
            k_col_scan<<<(J + 255) / 256, 256, 0, s>>>(d_colptr, (int)nch, J, d_cnt);
            k_chunk_place<<<(int)nch, 32, 0, s>>>(c->X.col, c->X.val, d_rowid, nnz, chunk, J, d_cnt,
                                                  c->X.csc_row, c->X.csc_val);
            const int64_t nv = (int64_t)vstart.size();
            k_block_runs<<<(int)std::min<int64_t>((nv + 255) / 256, 8 * nsm), 256, 0, s>>>(
                c->X.csc_row, d_colptr, d_blkrow, nblk, J, d_vstart);
            e = cudaGetLastError();
        }
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(vstart.data(), d_vstart, sizeof(int64_t) * vstart.size(),
                                cudaMemcpyDeviceToHost, s);
        cudaError_t e2 = cudaStreamSynchronize(s);
        ctx_free(c, d_colptr);
        ctx_free(c, d_rowid);
        ctx_free(c, d_cnt);
        ctx_free(c, d_blkrow);
        ctx_free(c, d_vstart);
        if (e == cudaSuccess) e = e2;
        if (e != cudaSuccess) {
            set_error("load: building the column-major copy failed: %s", cudaGetErrorString(e));
            return P2_ECUDA;
        }
    }
    // segments block by block, column by column within a block: each
    // (block, column) run cut into pieces of at most P2_SEG non-zeros
    std::vector<int64_t> s_lo, s_hi, vseg((size_t)nblk * J + 1, 0);
    c->X.blk_seg.assign((size_t)nblk + 1, 0);
    for (int b = 0; b < nblk; ++b) {
        c->X.blk_seg[b] = (int64_t)s_lo.size();
        for (int32_t j = 0; j < J; ++j) {
            vseg[(size_t)b * J + j] = (int64_t)s_lo.size();
            const int64_t lo = vstart[(size_t)j * (nblk + 1) + b];
            const int64_t hi = vstart[(size_t)j * (nblk + 1) + b + 1];
            for (int64_t a0 = lo; a0 < hi; a0 += P2_SEG) {
                s_lo.push_back(a0);
                s_hi.push_back(std::min<int64_t>(a0 + P2_SEG, hi));
            }
        }
    }
    c->X.blk_seg[nblk] = (int64_t)s_lo.size();
    vseg[(size_t)nblk * J] = (int64_t)s_lo.size();
    const int64_t nseg = (int64_t)s_lo.size();
    c->X.nseg = nseg;
    e = ctx_malloc(c, (void **)&c->X.seg_start, sizeof(int64_t) * (size_t)(nseg > 0 ? nseg : 1));
    if (e == cudaSuccess) e = ctx_malloc(c, (void **)&c->X.seg_end, sizeof(int64_t) * (size_t)(nseg > 0 ? nseg : 1));
    if (e == cudaSuccess) e = ctx_malloc(c, (void **)&c->X.col_seg, sizeof(int64_t) * vseg.size());
    if (e == cudaSuccess) e = ctx_malloc(c, (void **)&c->d_segpart, sizeof(double) * (size_t)(nseg > 0 ? nseg : 1) * c->R);
    if (e != cudaSuccess) {
        cudaGetLastError();
        set_error("load: allocation of the mode-2 segments failed: %s", cudaGetErrorString(e));
        return e == cudaErrorMemoryAllocation ? P2_ENOMEM : P2_ECUDA;
    }
    c->dev_bytes += sizeof(int64_t) * (2 * (size_t)nseg + vseg.size()) +
                    sizeof(double) * (size_t)nseg * c->R;
    if (nseg > 0) {
        P2_CUDA_TRY(cudaMemcpyAsync(c->X.seg_start, s_lo.data(), sizeof(int64_t) * (size_t)nseg,
                                    cudaMemcpyHostToDevice, s));
        P2_CUDA_TRY(cudaMemcpyAsync(c->X.seg_end, s_hi.data(), sizeof(int64_t) * (size_t)nseg,
                                    cudaMemcpyHostToDevice, s));
    }
    P2_CUDA_TRY(cudaMemcpyAsync(c->X.col_seg, vseg.data(), sizeof(int64_t) * vseg.size(),
                                cudaMemcpyHostToDevice, s));
    P2_CUDA_TRY(cudaStreamSynchronize(s));
    return P2_OK;
}

int launch_load(p2_ctx *c, const int64_t *d_subj_ptr, const int64_t *d_row_ptr,
                const int32_t *d_col, const float *d_val, int64_t K, int32_t J, int64_t N,
                int64_t nnz) {
    cudaStream_t s = c->stream;
    const int nsm = c->geo.nsm;
    LoadScratch *ls = nullptr;
    P2_CUDA_TRY(ctx_malloc(c, (void **)&ls, sizeof(LoadScratch)));
    P2_CUDA_TRY(cudaMemsetAsync(ls, 0, sizeof(LoadScratch), s));
    P2_CUDA_TRY(cudaMemsetAsync(c->d_colcount, 0, sizeof(int) * (size_t)J, s));
    k_check_subjects<<<4 * nsm, 256, 0, s>>>(d_subj_ptr, d_row_ptr, K, N, c->X.subj_row,
                                             c->X.subj_nnz, ls);
    if (N > 0) {
        const int smem_hist = J <= 12288 ? 1 : 0;            // within the default 48 KB
        k_check_rows<<<8 * nsm, 256, smem_hist ? (size_t)J * sizeof(int) : 0, s>>>(
            d_row_ptr, d_col, d_val, N, nnz, J, c->X.row_len, c->d_colcount, ls, smem_hist);
    }
    const int nb = c->geo.red_blocks;
    k_sumsq<<<nb, 256, 0, s>>>(d_val, nnz, c->d_part);
    P2_CUDA_TRY(cudaGetLastError());
    LoadScratch h{};
    P2_CUDA_TRY(cudaMemcpyAsync(&h, ls, sizeof(h), cudaMemcpyDeviceToHost, s));
    double *hp = new double[nb];
    int *cc = new int[J];
    cudaError_t e1 = cudaMemcpyAsync(hp, c->d_part, sizeof(double) * nb, cudaMemcpyDeviceToHost, s);
    cudaError_t e2 = cudaMemcpyAsync(cc, c->d_colcount, sizeof(int) * (size_t)J,
                                     cudaMemcpyDeviceToHost, s);
    cudaError_t e3 = cudaStreamSynchronize(s);
    ctx_free(c, ls);
    if (e1 != cudaSuccess || e2 != cudaSuccess || e3 != cudaSuccess) {
        delete[] hp;
        delete[] cc;
        set_error("load: device copy failed: %s",
                  cudaGetErrorString(e3 != cudaSuccess ? e3 : (e1 != cudaSuccess ? e1 : e2)));
        return P2_ECUDA;
    }
    if (h.flags) {
        delete[] hp;
        delete[] cc;
        set_error("p2_load_slices: malformed input (%s%s%s)",
                  (h.flags & FLAG_BAD_PTR) ? "bad subject/row pointers or row longer than 65535; " : "",
                  (h.flags & FLAG_BAD_COL) ? "column out of range or not strictly increasing in a row; " : "",
                  (h.flags & FLAG_BAD_VAL) ? "non-finite value; " : "");
        return P2_EINVAL;
    }
    double nx2 = 0.0;
    for (int b = 0; b < nb; ++b) nx2 += hp[b];
    delete[] hp;
    // The relabel's key: the column counts, summed over all shards for a
    // sharded context (every shard then relabels alike), together with ||X||^2.
    std::vector<double> key((size_t)J + 1);
    for (int j = 0; j < J; ++j) key[j] = (double)cc[j];
    key[J] = nx2;
    if (c->xfn) {
        double *dk = nullptr;
        cudaError_t e = ctx_malloc(c, (void **)&dk, sizeof(double) * ((size_t)J + 1));
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(dk, key.data(), sizeof(double) * ((size_t)J + 1),
                                cudaMemcpyHostToDevice, s);
        int rc = e == cudaSuccess ? exchange(c, dk, (int64_t)J + 1) : P2_OK;
        if (e == cudaSuccess && rc == P2_OK)
            e = cudaMemcpyAsync(key.data(), dk, sizeof(double) * ((size_t)J + 1),
                                cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess && rc == P2_OK) e = cudaStreamSynchronize(s);
        if (dk) ctx_free(c, dk);
        if (rc != P2_OK) {
            delete[] cc;
            return rc;
        }
        if (e != cudaSuccess) {
            delete[] cc;
            set_error("load: exchange of the column counts failed: %s", cudaGetErrorString(e));
            return P2_ECUDA;
        }
        nx2 = key[J];
    }
    // relabel: decreasing frequency, ties by original id
    {
        int32_t *order = c->h_perm_new2old;
        for (int j = 0; j < J; ++j) order[j] = j;
        // bottom-up stable merge sort on count, descending
        int32_t *tmp = new int32_t[J];
        for (int w = 1; w < J; w <<= 1) {
            for (int lo = 0; lo < J; lo += 2 * w) {
                int mid = lo + w < J ? lo + w : J, hi = lo + 2 * w < J ? lo + 2 * w : J;
                int a = lo, b = mid, o = lo;
                while (a < mid && b < hi) {
                    if (key[order[b]] > key[order[a]]) tmp[o++] = order[b++];
                    else tmp[o++] = order[a++];
                }
                while (a < mid) tmp[o++] = order[a++];
                while (b < hi) tmp[o++] = order[b++];
            }
            for (int j = 0; j < J; ++j) order[j] = tmp[j];
        }
        delete[] tmp;
        for (int r = 0; r < J; ++r) c->h_perm_old2new[order[r]] = r;
    }
    std::vector<int32_t> count_new((size_t)J);
    for (int r = 0; r < J; ++r) count_new[r] = cc[c->h_perm_new2old[r]];
    delete[] cc;
    P2_CUDA_TRY(cudaMemcpyAsync(c->d_perm_old2new, c->h_perm_old2new, sizeof(int32_t) * (size_t)J,
                                cudaMemcpyHostToDevice, s));
    if (nnz > 0) k_relabel<<<8 * nsm, 256, 0, s>>>(d_col, c->d_perm_old2new, nnz, c->X.col);
    P2_CUDA_TRY(cudaGetLastError());
    {
        int rc = build_csc(c, d_row_ptr, count_new.data(), N, nnz, J);
        if (rc != P2_OK) return rc;
    }
    P2_CUDA_TRY(cudaMemcpyAsync(&c->d_s->normx2, &nx2, sizeof(double), cudaMemcpyHostToDevice, s));
    P2_CUDA_TRY(cudaStreamSynchronize(s));
    return P2_OK;
}

}  // namespace p2
