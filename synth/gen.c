/*
 * Seeded synthetic inputs: power-law graphs (Chung-Lu, R-MAT), their CSR form,
 * and the largest adjacency eigenvalue.  Host C, OpenMP-parallel, deterministic
 * for any thread count.
 *
 * This module holds none of the diffusion method's arithmetic.  It stands in for
 * the SNAP/OGB graphs of the paper's experiments (Section 5, Table 3), which are
 * not available here, with graphs of the same kind (undirected, no self-loops,
 * heavy-tailed degrees) at the sizes the workloads name.
 *
 * Random numbers: SplitMix64 (Steele, Lea, Flood 2014) expands a 64-bit key into
 * the 256-bit state of xoshiro256** (Blackman, Vigna 2018).  Every block of
 * GEN_BLOCK items draws from its own generator keyed by (seed, stream, block), so
 * the output does not depend on how blocks are spread over threads.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>
#include <omp.h>

#define GEN_BLOCK 65536

/* ---------------------------------------------------------------- RNG ---- */

static inline uint64_t splitmix64_next(uint64_t *s) {
    uint64_t z = (*s += 0x9E3779B97F4A7C15ULL);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

typedef struct { uint64_t s[4]; } xo256;

static inline uint64_t rotl64(uint64_t x, int k) { return (x << k) | (x >> (64 - k)); }

static inline uint64_t xo_next(xo256 *g) {
    uint64_t *s = g->s;
    const uint64_t result = rotl64(s[1] * 5, 7) * 9;
    const uint64_t t = s[1] << 17;
    s[2] ^= s[0];
    s[3] ^= s[1];
    s[1] ^= s[2];
    s[0] ^= s[3];
    s[2] ^= t;
    s[3] = rotl64(s[3], 45);
    return result;
}

/* generator for (seed, stream, block): a SplitMix64 walk from a mixed key */
static void xo_init(xo256 *g, uint64_t seed, uint64_t stream, uint64_t block) {
    uint64_t k = seed;
    uint64_t m = splitmix64_next(&k);
    m ^= stream * 0xD1B54A32D192ED03ULL;
    m ^= block * 0x8CB92BA72F3D8DD7ULL;
    for (int i = 0; i < 4; i++) g->s[i] = splitmix64_next(&m);
}

/* uniform double in [0,1) from the top 53 bits */
static inline double xo_unif(xo256 *g) { return (double)(xo_next(g) >> 11) * 0x1.0p-53; }

/* uniform integer in [0, bound) by Lemire's multiply-shift with rejection */
static inline uint64_t xo_below(xo256 *g, uint64_t bound) {
    uint64_t x = xo_next(g);
    __uint128_t m = (__uint128_t)x * bound;
    uint64_t l = (uint64_t)m;
    if (l < bound) {
        uint64_t t = (0 - bound) % bound;
        while (l < t) {
            x = xo_next(g);
            m = (__uint128_t)x * bound;
            l = (uint64_t)m;
        }
    }
    return (uint64_t)(m >> 64);
}

/* ------------------------------------------------------------ Chung-Lu ---- */

/*
 * Endpoint pairs of a Chung-Lu graph: node i has weight w_i = (i+1)^(-1/(gamma-1))
 * (rescaled so the weights average mean_deg), and each of the m pairs draws both
 * endpoints independently with probability proportional to w.  Sampling uses a
 * Walker/Vose alias table.  Returns 0, or -1 on allocation failure.
 */
int synth_chung_lu_pairs(int64_t n, double mean_deg, double gamma, uint64_t seed,
                         int64_t m, int32_t *src, int32_t *dst) {
    double *prob = (double *)malloc(sizeof(double) * n);
    int32_t *alias = (int32_t *)malloc(sizeof(int32_t) * n);
    int32_t *small = (int32_t *)malloc(sizeof(int32_t) * n);
    int32_t *large = (int32_t *)malloc(sizeof(int32_t) * n);
    if (!prob || !alias || !small || !large) {
        free(prob); free(alias); free(small); free(large);
        return -1;
    }
    const double ex = -1.0 / (gamma - 1.0);
    double total = 0.0;
    for (int64_t i = 0; i < n; i++) {
        prob[i] = pow((double)(i + 1), ex);
        total += prob[i];
    }
    (void)mean_deg; /* the pair count m carries the mean degree */
    /* Vose: scaled weights p_i = n w_i / sum w */
    int64_t ns = 0, nl = 0;
    for (int64_t i = 0; i < n; i++) {
        prob[i] = prob[i] * (double)n / total;
        if (prob[i] < 1.0) small[ns++] = (int32_t)i; else large[nl++] = (int32_t)i;
    }
    while (ns > 0 && nl > 0) {
        int32_t s = small[--ns];
        int32_t l = large[--nl];
        alias[s] = l;
        prob[l] = (prob[l] + prob[s]) - 1.0;
        if (prob[l] < 1.0) small[ns++] = l; else large[nl++] = l;
    }
    while (nl > 0) { int32_t l = large[--nl]; prob[l] = 1.0; alias[l] = l; }
    while (ns > 0) { int32_t s = small[--ns]; prob[s] = 1.0; alias[s] = s; }
    free(small); free(large);

    const int64_t nblocks = (m + GEN_BLOCK - 1) / GEN_BLOCK;
#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t b = 0; b < nblocks; b++) {
        xo256 g;
        xo_init(&g, seed, 1, (uint64_t)b);
        int64_t lo = b * GEN_BLOCK, hi = lo + GEN_BLOCK < m ? lo + GEN_BLOCK : m;
        for (int64_t e = lo; e < hi; e++) {
            int32_t ends[2];
            for (int k = 0; k < 2; k++) {
                int64_t i = (int64_t)xo_below(&g, (uint64_t)n);
                double u = xo_unif(&g);
                ends[k] = u < prob[i] ? (int32_t)i : alias[i];
            }
            src[e] = ends[0];
            dst[e] = ends[1];
        }
    }
    free(prob); free(alias);
    return 0;
}

/* --------------------------------------------------------------- R-MAT ---- */

/*
 * Endpoint pairs of an R-MAT graph with 2^scale nodes: each pair descends scale
 * levels of the adjacency quadrants with probabilities (a, b, c, 1-a-b-c).
 */
int synth_rmat_pairs(int scale, double a, double b, double c, uint64_t seed,
                     int64_t m, int32_t *src, int32_t *dst) {
    const double ab = a + b, abc = a + b + c;
    const int64_t nblocks = (m + GEN_BLOCK - 1) / GEN_BLOCK;
#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t blk = 0; blk < nblocks; blk++) {
        xo256 g;
        xo_init(&g, seed, 2, (uint64_t)blk);
        int64_t lo = blk * GEN_BLOCK, hi = lo + GEN_BLOCK < m ? lo + GEN_BLOCK : m;
        for (int64_t e = lo; e < hi; e++) {
            uint32_t u = 0, v = 0;
            for (int lev = 0; lev < scale; lev++) {
                double p = xo_unif(&g);
                uint32_t bit = 1u << (scale - 1 - lev);
                if (p < a) {
                } else if (p < ab) {
                    v |= bit;
                } else if (p < abc) {
                    u |= bit;
                } else {
                    u |= bit;
                    v |= bit;
                }
            }
            src[e] = (int32_t)u;
            dst[e] = (int32_t)v;
        }
    }
    return 0;
}

/* Fisher-Yates permutation of 0..n-1 (sequential, one generator) */
int synth_permutation(int64_t n, uint64_t seed, int32_t *perm) {
    for (int64_t i = 0; i < n; i++) perm[i] = (int32_t)i;
    xo256 g;
    xo_init(&g, seed, 3, 0);
    for (int64_t i = n - 1; i > 0; i--) {
        int64_t j = (int64_t)xo_below(&g, (uint64_t)(i + 1));
        int32_t t = perm[i]; perm[i] = perm[j]; perm[j] = t;
    }
    return 0;
}

/* relabel both endpoint arrays through perm */
void synth_relabel(int64_t m, const int32_t *perm, int32_t *src, int32_t *dst) {
#pragma omp parallel for schedule(static)
    for (int64_t e = 0; e < m; e++) {
        src[e] = perm[src[e]];
        dst[e] = perm[dst[e]];
    }
}

/* ----------------------------------------------------------------- CSR ---- */

static int cmp_i32(const void *p, const void *q) {
    int32_t a = *(const int32_t *)p, b = *(const int32_t *)q;
    return (a > b) - (a < b);
}

static void sort_row(int32_t *a, int64_t len) {
    if (len < 24) {
        for (int64_t i = 1; i < len; i++) {
            int32_t key = a[i];
            int64_t j = i - 1;
            while (j >= 0 && a[j] > key) { a[j + 1] = a[j]; j--; }
            a[j + 1] = key;
        }
    } else {
        qsort(a, (size_t)len, sizeof(int32_t), cmp_i32);
    }
}

/*
 * Undirected simple graph from endpoint pairs: drop self-loops, add both
 * directions, sort each row and remove duplicates.  offsets has n+1 entries;
 * cols must hold 2m entries (the final nnz is returned, <= 2m).  Returns -1 on
 * allocation failure.
 */
int64_t synth_csr_from_pairs(int64_t n, int64_t m, const int32_t *src, const int32_t *dst,
                             int64_t *offsets, int32_t *cols) {
    int64_t *cnt = (int64_t *)calloc((size_t)n + 1, sizeof(int64_t));
    if (!cnt) return -1;
#pragma omp parallel for schedule(static)
    for (int64_t e = 0; e < m; e++) {
        int32_t u = src[e], v = dst[e];
        if (u == v) continue;
        __atomic_fetch_add(&cnt[u], 1, __ATOMIC_RELAXED);
        __atomic_fetch_add(&cnt[v], 1, __ATOMIC_RELAXED);
    }
    /* raw row starts in offsets; cursor in cnt */
    int64_t acc = 0;
    for (int64_t u = 0; u < n; u++) {
        int64_t c = cnt[u];
        offsets[u] = acc;
        cnt[u] = acc;
        acc += c;
    }
    offsets[n] = acc;
#pragma omp parallel for schedule(static)
    for (int64_t e = 0; e < m; e++) {
        int32_t u = src[e], v = dst[e];
        if (u == v) continue;
        int64_t pu = __atomic_fetch_add(&cnt[u], 1, __ATOMIC_RELAXED);
        int64_t pv = __atomic_fetch_add(&cnt[v], 1, __ATOMIC_RELAXED);
        cols[pu] = v;
        cols[pv] = u;
    }
    /* sort + unique per row; unique length into cnt[u] */
#pragma omp parallel for schedule(dynamic, 1024)
    for (int64_t u = 0; u < n; u++) {
        int32_t *row = cols + offsets[u];
        int64_t len = offsets[u + 1] - offsets[u];
        sort_row(row, len);
        int64_t k = 0;
        for (int64_t i = 0; i < len; i++)
            if (k == 0 || row[i] != row[k - 1]) row[k++] = row[i];
        cnt[u] = k;
    }
    /* compact: new offsets are the prefix sums of the unique lengths */
    int64_t *newoff = (int64_t *)malloc(sizeof(int64_t) * ((size_t)n + 1));
    if (!newoff) { free(cnt); return -1; }
    acc = 0;
    for (int64_t u = 0; u < n; u++) { newoff[u] = acc; acc += cnt[u]; }
    newoff[n] = acc;
    /* rows only move left, so a sequential in-place pass is safe */
    for (int64_t u = 0; u < n; u++) {
        if (newoff[u] != offsets[u] && cnt[u] > 0)
            memmove(cols + newoff[u], cols + offsets[u], sizeof(int32_t) * (size_t)cnt[u]);
    }
    memcpy(offsets, newoff, sizeof(int64_t) * ((size_t)n + 1));
    free(newoff);
    free(cnt);
    return acc;
}

/* ------------------------------------------------------ largest eigenvalue */

/*
 * Largest eigenvalue of the adjacency matrix by power iteration on A + I from
 * the all-ones vector (the shift keeps bipartite parts from oscillating).  The
 * Rayleigh quotient of A + I is tracked; iteration stops when it changes by less
 * than rel_tol relative, or after max_iter steps.  Sums use fixed blocks so the
 * result does not depend on the thread count.  Returns lambda_max(A); *iters
 * receives the number of steps.
 */
double synth_lambda_max(int64_t n, const int64_t *off, const int32_t *col,
                        double rel_tol, int64_t max_iter, int64_t *iters) {
    double *v = (double *)malloc(sizeof(double) * n);
    double *w = (double *)malloc(sizeof(double) * n);
    const int64_t nb = (n + GEN_BLOCK - 1) / GEN_BLOCK;
    double *part = (double *)malloc(sizeof(double) * (nb > 0 ? nb : 1) * 2);
    if (!v || !w || !part) { free(v); free(w); free(part); return -1.0; }
    double inv = 1.0 / sqrt((double)n);
    for (int64_t i = 0; i < n; i++) v[i] = inv;
    double rho_prev = 0.0, rho = 0.0;
    int64_t it = 0;
    for (it = 1; it <= max_iter; it++) {
#pragma omp parallel for schedule(dynamic, 1)
        for (int64_t b = 0; b < nb; b++) {
            int64_t lo = b * GEN_BLOCK, hi = lo + GEN_BLOCK < n ? lo + GEN_BLOCK : n;
            double sq = 0.0, rq = 0.0;
            for (int64_t i = lo; i < hi; i++) {
                double s = v[i];
                for (int64_t e = off[i]; e < off[i + 1]; e++) s += v[col[e]];
                w[i] = s;
                sq += s * s;
                rq += s * v[i];
            }
            part[2 * b] = sq;
            part[2 * b + 1] = rq;
        }
        double sq = 0.0, rq = 0.0;
        for (int64_t b = 0; b < nb; b++) { sq += part[2 * b]; rq += part[2 * b + 1]; }
        rho = rq; /* v has unit norm, so v'(A+I)v is the Rayleigh quotient */
        double nrm = sqrt(sq);
#pragma omp parallel for schedule(static)
        for (int64_t i = 0; i < n; i++) v[i] = w[i] / nrm;
        if (it > 1 && fabs(rho - rho_prev) <= rel_tol * fabs(rho)) break;
        rho_prev = rho;
    }
    if (iters) *iters = it > max_iter ? max_iter : it;
    free(v); free(w); free(part);
    return rho - 1.0;
}

int synth_num_threads(void) { return omp_get_max_threads(); }
