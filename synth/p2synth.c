/*
 * Seeded synthetic generators for irregular sparse tensors {X_k}.
 *
 * This module only draws random inputs: subject sizes I_k, per-row non-zero
 * counts, distinct column ids and values, plus uniform initial factors.  It
 * holds none of the PARAFAC2 arithmetic.  Both the FP64 oracle and the CUDA
 * path consume what it produces.
 *
 * Randomness is counter based: every draw is a SplitMix64 sequence
 * (Steele, Lea & Flood, "Fast splittable pseudorandom number generators",
 * OOPSLA 2014) whose starting state is a hash of (seed, stream, index).  So a
 * row's draws depend only on the seed and the row's global index, and the
 * output is identical for any number of OpenMP threads.
 *
 * Shapes follow the paper's synthetic workload (Section 5, "Synthetic Data":
 * K subjects, J variables, at most 100 observations per subject) with the
 * column/value distributions stated for each workload in the Python wrapper.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define GOLDEN 0x9E3779B97F4A7C15ULL

/* Portable elementary functions built from IEEE basic operations only (the
 * file is compiled with -ffp-contract=off), so that x86-64 and AArch64 hosts
 * draw bit-identical samples.  exp: Cody-Waite reduction by ln 2 and a Taylor
 * polynomial; log: the atanh series log(m) = 2 atanh((m-1)/(m+1)); cos: Taylor
 * series after reduction to [-pi, pi]. */
static const double LN2_HI = 6.93147180369123816490e-01;
static const double LN2_LO = 1.90821492927058770002e-10;

static double p_exp(double x) {
    if (x < -745.0) return 0.0;
    if (x > 709.0) return HUGE_VAL;
    double kf = floor(x / 0.6931471805599453 + 0.5);
    double r = (x - kf * LN2_HI) - kf * LN2_LO;
    double s = 1.0, t = 1.0;
    for (int i = 1; i <= 22; i++) { t = t * r / (double)i; s += t; }
    return ldexp(s, (int)kf);
}

static double p_log(double x) {
    int e;
    double m = frexp(x, &e);               /* x = m 2^e, m in [0.5, 1) */
    if (m < 0.7071067811865476) { m *= 2.0; e -= 1; }
    double s = (m - 1.0) / (m + 1.0), s2 = s * s, t = s, acc = 0.0;
    for (int i = 1; i <= 41; i += 2) { acc += t / (double)i; t *= s2; }
    return 2.0 * acc + ((double)e * LN2_LO + (double)e * LN2_HI);
}

static double p_cos_2pi(double u) {          /* cos(2 pi u) */
    double t = u - floor(u + 0.5);           /* t in [-0.5, 0.5] */
    double x = 6.283185307179586 * t, x2 = x * x, term = 1.0, acc = 1.0;
    for (int i = 2; i <= 46; i += 2) { term = -term * x2 / (double)((i - 1) * i); acc += term; }
    return acc;
}

static double p_pow_neg(double r, double s) { return p_exp(-s * p_log(r)); }  /* r^-s */

static inline uint64_t mix64(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

typedef struct { uint64_t s; } sm64_t;

static inline uint64_t sm64_next(sm64_t *g) {
    g->s += GOLDEN;
    return mix64(g->s);
}

static inline sm64_t sm64_for(uint64_t seed, uint64_t stream, uint64_t index) {
    sm64_t g;
    g.s = mix64(seed + GOLDEN * (stream + 1)) ^ mix64(index * GOLDEN + stream);
    return g;
}

/* uniform double in [0,1) with 53 random bits */
static inline double u01(sm64_t *g) { return (double)(sm64_next(g) >> 11) * 0x1.0p-53; }
/* uniform double in (0,1] */
static inline double u01_open0(sm64_t *g) { return ((double)(sm64_next(g) >> 11) + 1.0) * 0x1.0p-53; }

/* Poisson(lambda) by sequential inversion; lambda is small (<= 20) here. */
static int poisson(sm64_t *g, double lambda) {
    if (lambda <= 0.0) return 0;
    double u = u01(g);
    double p = p_exp(-lambda), F = p;
    int k = 0;
    while (u > F && k < 10000) {
        k++;
        p *= lambda / k;
        F += p;
        if (p < 1e-300) break;
    }
    return k;
}

enum { STREAM_SUBJ = 1, STREAM_ROWNNZ = 2, STREAM_ROWCOLS = 3, STREAM_PERM = 4,
       STREAM_INIT = 5, STREAM_VALS = 6 };

typedef struct {
    int64_t K;          /* subjects */
    int32_t J;          /* variables (columns) */
    int32_t imin, imax; /* I_k ~ U{imin..imax} when size_mode == 0 */
    int32_t size_mode;  /* 0 uniform, 1 round(lognormal(mu, sigma)) clipped to [imin, imax] */
    double mu, sigma;
    double lam;         /* non-zeros per row = Poisson(lam) + 1, capped at J */
    int32_t col_mode;   /* 0 uniform over J, 1 Zipf(zipf_s) over ranks mapped by a seeded permutation */
    double zipf_s;
    double val_lam;     /* values = 1 + Poisson(val_lam) */
    uint64_t seed;
} p2synth_cfg;

static int64_t subject_rows(const p2synth_cfg *c, int64_t k) {
    sm64_t g = sm64_for(c->seed, STREAM_SUBJ, (uint64_t)k);
    if (c->size_mode == 0) {
        uint64_t span = (uint64_t)(c->imax - c->imin + 1);
        return c->imin + (int64_t)(sm64_next(&g) % span);
    }
    /* Box-Muller normal */
    double u1 = u01_open0(&g), u2 = u01(&g);
    double n = sqrt(-2.0 * p_log(u1)) * p_cos_2pi(u2);
    double x = p_exp(c->mu + c->sigma * n);
    int64_t r = (int64_t)floor(x + 0.5);
    if (r < c->imin) r = c->imin;
    if (r > c->imax) r = c->imax;
    return r;
}

static int32_t row_nnz(const p2synth_cfg *c, int64_t grow) {
    sm64_t g = sm64_for(c->seed, STREAM_ROWNNZ, (uint64_t)grow);
    int64_t n = (int64_t)poisson(&g, c->lam) + 1;
    if (n > c->J) n = c->J;
    return (int32_t)n;
}

/* Pass 1: subject row offsets (subj_ptr has K+1 entries). Returns total rows. */
int64_t p2synth_subjects(const p2synth_cfg *c, int64_t *subj_ptr) {
    int64_t K = c->K;
    #pragma omp parallel for schedule(static)
    for (int64_t k = 0; k < K; k++) subj_ptr[k + 1] = subject_rows(c, k);
    subj_ptr[0] = 0;
    for (int64_t k = 0; k < K; k++) subj_ptr[k + 1] += subj_ptr[k];
    return subj_ptr[K];
}

/* Pass 2: row offsets (row_ptr has N+1 entries). Returns nnz. */
int64_t p2synth_rows(const p2synth_cfg *c, int64_t N, int64_t *row_ptr) {
    #pragma omp parallel for schedule(static)
    for (int64_t r = 0; r < N; r++) row_ptr[r + 1] = row_nnz(c, r);
    row_ptr[0] = 0;
    for (int64_t r = 0; r < N; r++) row_ptr[r + 1] += row_ptr[r];
    return row_ptr[N];
}

static int cmp_i32(const void *a, const void *b) {
    int32_t x = *(const int32_t *)a, y = *(const int32_t *)b;
    return (x > y) - (x < y);
}

/* Column sampler: cumulative Zipf table over ranks 1..J and the rank->column map. */
typedef struct { double *cdf; int32_t *perm; } colsampler;

static int32_t draw_col(const p2synth_cfg *c, const colsampler *cs, sm64_t *g) {
    if (c->col_mode == 0) return (int32_t)(sm64_next(g) % (uint64_t)c->J);
    double u = u01(g);
    int32_t lo = 0, hi = c->J - 1;      /* first rank whose cdf > u */
    while (lo < hi) {
        int32_t mid = (lo + hi) >> 1;
        if (cs->cdf[mid] > u) hi = mid; else lo = mid + 1;
    }
    return cs->perm[lo];
}

/* Pass 3: distinct sorted columns per row (drawn without replacement by
 * rejecting repeats) and values 1 + Poisson(val_lam). */
int p2synth_fill(const p2synth_cfg *c, int64_t N, const int64_t *row_ptr,
                 int32_t *col, float *val) {
    colsampler cs = {0, 0};
    int32_t J = c->J;
    if (c->col_mode == 1) {
        cs.cdf = (double *)malloc(sizeof(double) * (size_t)J);
        cs.perm = (int32_t *)malloc(sizeof(int32_t) * (size_t)J);
        if (!cs.cdf || !cs.perm) { free(cs.cdf); free(cs.perm); return -1; }
        double acc = 0.0;
        for (int32_t r = 0; r < J; r++) { acc += p_pow_neg((double)(r + 1), c->zipf_s); cs.cdf[r] = acc; }
        for (int32_t r = 0; r < J; r++) cs.cdf[r] /= acc;
        cs.cdf[J - 1] = 2.0;  /* guard: every u < 1 lands inside the table */
        for (int32_t r = 0; r < J; r++) cs.perm[r] = r;
        sm64_t g = sm64_for(c->seed, STREAM_PERM, 0);
        for (int32_t r = J - 1; r > 0; r--) {    /* Fisher-Yates */
            int32_t s = (int32_t)(sm64_next(&g) % (uint64_t)(r + 1));
            int32_t t = cs.perm[r]; cs.perm[r] = cs.perm[s]; cs.perm[s] = t;
        }
    }
    #pragma omp parallel for schedule(dynamic, 4096)
    for (int64_t r = 0; r < N; r++) {
        int64_t b = row_ptr[r], e = row_ptr[r + 1];
        int32_t n = (int32_t)(e - b);
        int32_t *cc = col + b;
        sm64_t g = sm64_for(c->seed, STREAM_ROWCOLS, (uint64_t)r);
        int32_t have = 0;
        int64_t tries = 0, max_tries = 64LL * n + 1024;
        while (have < n && tries < max_tries) {
            int32_t j = draw_col(c, &cs, &g);
            tries++;
            int dup = 0;
            for (int32_t t = 0; t < have; t++) if (cc[t] == j) { dup = 1; break; }
            if (!dup) cc[have++] = j;
        }
        /* extremely dense rows only: complete with the smallest unused ids */
        for (int32_t j = 0; have < n && j < J; j++) {
            int dup = 0;
            for (int32_t t = 0; t < have; t++) if (cc[t] == j) { dup = 1; break; }
            if (!dup) cc[have++] = j;
        }
        qsort(cc, (size_t)n, sizeof(int32_t), cmp_i32);
        sm64_t gv = sm64_for(c->seed, STREAM_VALS, (uint64_t)r);
        for (int32_t t = 0; t < n; t++) val[b + t] = (float)(1 + poisson(&gv, c->val_lam));
    }
    free(cs.cdf); free(cs.perm);
    return 0;
}

/* ---- planted PARAFAC2 workload (the paper's synthetic recipe) -------------
 * Section 5 ("Synthetic Data") builds its tensors from planted factors: each
 * subject k has dense_rows observations of J variables, X_k = Q_k H S_k V^T
 * with Q_k^T Q_k = I at rank Rp, and the entries are then sparsified
 * uniformly with keep probability p; empty rows are dropped (which is why the
 * paper's mean I_k is 46.9 at 63M non-zeros and 99.3 at 500M).  Here H
 * (Rp x Rp), V (J x Rp) and the diagonal of S_k are uniform in [0, 1); Q_k is
 * the first Rp columns of the Householder reflector I - 2 v v^T with v a
 * uniformly random unit vector (orthonormal columns, one entry per O(1)
 * work: Q_k(i, r) = [i == r] - 2 v_i v_r); the number of kept entries of a
 * dense row is Poisson(J p) (capped at J) over distinct uniform columns. */
typedef struct {
    int64_t K;
    int32_t J;
    int32_t dense_rows;   /* observations per subject before sparsification */
    int32_t rank;         /* planted rank Rp <= dense_rows */
    double keep_p;        /* keep probability of an entry */
    uint64_t seed;
} p2synth_pcfg;

enum { STREAM_PLANT_H = 7, STREAM_PLANT_V = 8, STREAM_PLANT_W = 9, STREAM_PLANT_Q = 10 };

static int32_t planted_count(const p2synth_pcfg *c, int64_t k, int32_t i) {
    sm64_t g = sm64_for(c->seed, STREAM_ROWNNZ, (uint64_t)(k * c->dense_rows + i));
    int64_t n = (int64_t)poisson(&g, (double)c->J * c->keep_p);
    return (int32_t)(n > c->J ? c->J : n);
}

static float planted_u01(uint64_t seed, uint64_t stream, uint64_t i) {
    sm64_t g = sm64_for(seed, stream, i);
    return (float)((double)(sm64_next(&g) >> 40) * 0x1.0p-24);
}

/* H (Rp x Rp), V (J x Rp) and, for subject k, w (Rp) and the unit vector v
 * (dense_rows); any pointer may be NULL. */
void p2synth_planted_factors(const p2synth_pcfg *c, int64_t k, float *H, float *V, float *w,
                             double *v) {
    const int32_t Rp = c->rank;
    if (H) for (int64_t e = 0; e < (int64_t)Rp * Rp; e++) H[e] = planted_u01(c->seed, STREAM_PLANT_H, (uint64_t)e);
    if (V) for (int64_t e = 0; e < (int64_t)c->J * Rp; e++) V[e] = planted_u01(c->seed, STREAM_PLANT_V, (uint64_t)e);
    if (w) for (int32_t s = 0; s < Rp; s++) w[s] = planted_u01(c->seed, STREAM_PLANT_W, (uint64_t)(k * Rp + s));
    if (v) {
        sm64_t g = sm64_for(c->seed, STREAM_PLANT_Q, (uint64_t)k);
        double nrm = 0.0;
        for (int32_t i = 0; i < c->dense_rows; i += 2) {      /* Box-Muller pairs */
            double u1 = u01_open0(&g), u2 = u01(&g);
            double rr = sqrt(-2.0 * p_log(u1));
            v[i] = rr * p_cos_2pi(u2);
            if (i + 1 < c->dense_rows) v[i + 1] = rr * p_cos_2pi(u2 + 0.25);
        }
        for (int32_t i = 0; i < c->dense_rows; i++) nrm += v[i] * v[i];
        nrm = sqrt(nrm);
        for (int32_t i = 0; i < c->dense_rows; i++) v[i] /= nrm;
    }
}

/* Pass 1: rows per subject = non-empty dense rows. Returns total rows. */
int64_t p2synth_planted_subjects(const p2synth_pcfg *c, int64_t *subj_ptr) {
    #pragma omp parallel for schedule(static)
    for (int64_t k = 0; k < c->K; k++) {
        int64_t n = 0;
        for (int32_t i = 0; i < c->dense_rows; i++) n += planted_count(c, k, i) > 0;
        subj_ptr[k + 1] = n;
    }
    subj_ptr[0] = 0;
    for (int64_t k = 0; k < c->K; k++) subj_ptr[k + 1] += subj_ptr[k];
    return subj_ptr[c->K];
}

/* Pass 2: row offsets. Returns nnz. */
int64_t p2synth_planted_rows(const p2synth_pcfg *c, const int64_t *subj_ptr, int64_t N,
                             int64_t *row_ptr) {
    #pragma omp parallel for schedule(static)
    for (int64_t k = 0; k < c->K; k++) {
        int64_t r = subj_ptr[k];
        for (int32_t i = 0; i < c->dense_rows; i++) {
            int32_t n = planted_count(c, k, i);
            if (n > 0) row_ptr[++r] = n;
        }
    }
    row_ptr[0] = 0;
    for (int64_t r = 0; r < N; r++) row_ptr[r + 1] += row_ptr[r];
    return row_ptr[N];
}

/* Pass 3: distinct sorted uniform columns and the planted values
 * x_ij = sum_s U_k(i, s) w_s V(j, s), U_k = Q_k H, computed in double. */
int p2synth_planted_fill(const p2synth_pcfg *c, const int64_t *subj_ptr, const int64_t *row_ptr,
                         int32_t *col, float *val) {
    const int32_t Rp = c->rank, J = c->J, D = c->dense_rows;
    float *H = (float *)malloc(sizeof(float) * (size_t)Rp * Rp);
    float *V = (float *)malloc(sizeof(float) * (size_t)J * Rp);
    if (!H || !V) { free(H); free(V); return -1; }
    p2synth_planted_factors(c, 0, H, V, NULL, NULL);
    int fail = 0;
    #pragma omp parallel
    {
        double *v = (double *)malloc(sizeof(double) * (size_t)D);
        double *cs = (double *)malloc(sizeof(double) * (size_t)Rp);
        double *u = (double *)malloc(sizeof(double) * (size_t)Rp);
        float *w = (float *)malloc(sizeof(float) * (size_t)Rp);
        if (!v || !cs || !u || !w) {
            #pragma omp atomic write
            fail = 1;
        } else {
            #pragma omp for schedule(dynamic, 256)
            for (int64_t k = 0; k < c->K; k++) {
                p2synth_planted_factors(c, k, NULL, NULL, w, v);
                for (int32_t s = 0; s < Rp; s++) {          /* c = v_{0:Rp}^T H */
                    double a = 0.0;
                    for (int32_t r = 0; r < Rp; r++) a += v[r] * (double)H[r * Rp + s];
                    cs[s] = a;
                }
                int64_t r = subj_ptr[k];
                for (int32_t i = 0; i < D; i++) {
                    int32_t n = planted_count(c, k, i);
                    if (n == 0) continue;
                    for (int32_t s = 0; s < Rp; s++)       /* u_i = Q_k(i,:) H, times S_k */
                        u[s] = ((i < Rp ? (double)H[i * Rp + s] : 0.0) - 2.0 * v[i] * cs[s]) * (double)w[s];
                    int64_t b = row_ptr[r];
                    int32_t *cc = col + b;
                    sm64_t g = sm64_for(c->seed, STREAM_ROWCOLS, (uint64_t)(k * D + i));
                    int32_t have = 0;
                    int64_t tries = 0, max_tries = 64LL * n + 1024;
                    while (have < n && tries < max_tries) {
                        int32_t j = (int32_t)(sm64_next(&g) % (uint64_t)J);
                        tries++;
                        int dup = 0;
                        for (int32_t t = 0; t < have; t++) if (cc[t] == j) { dup = 1; break; }
                        if (!dup) cc[have++] = j;
                    }
                    for (int32_t j = 0; have < n && j < J; j++) {
                        int dup = 0;
                        for (int32_t t = 0; t < have; t++) if (cc[t] == j) { dup = 1; break; }
                        if (!dup) cc[have++] = j;
                    }
                    qsort(cc, (size_t)n, sizeof(int32_t), cmp_i32);
                    for (int32_t t = 0; t < n; t++) {
                        const float *vj = V + (size_t)cc[t] * Rp;
                        double x = 0.0;
                        for (int32_t s = 0; s < Rp; s++) x += u[s] * (double)vj[s];
                        val[b + t] = (float)x;
                    }
                    r++;
                }
            }
        }
        free(v); free(cs); free(u); free(w);
    }
    free(H); free(V);
    return fail ? -1 : 0;
}

/* n values uniform in [0,1), each a multiple of 2^-24 so that it is exact in
 * FP32 and FP64 alike; used for initial factors H, V, W. */
void p2synth_uniform(uint64_t seed, uint64_t stream, int64_t n, float *out) {
    #pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; i++) {
        sm64_t g = sm64_for(seed, STREAM_INIT + 16 * stream, (uint64_t)i);
        out[i] = (float)((double)(sm64_next(&g) >> 40) * 0x1.0p-24);
    }
}

int p2synth_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
