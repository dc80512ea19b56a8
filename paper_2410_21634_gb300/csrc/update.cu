// Edge insertion into the device CSR: the dynamic setting of Section 4, where a snapshot
// G_t becomes G_{t+1} through a batch of insertion events.  Each undirected edge adds the
// adjacencies u -> v and v -> u; self-loops and adjacencies already present are skipped,
// so rows stay sorted and duplicate-free (the store's invariant).
//
// The batch is normalised on the host (it is small next to the graph), then the device
// drops adjacencies already in their row (binary search) and rebuilds the CSR into spare
// buffers that are kept between batches: new offsets and the old columns' new places come
// from binary searches over the few changed rows (the rest of the CSR only shifts), and a
// thread per added adjacency drops it into its gap.
#include <algorithm>
#include <utility>
#include <vector>

#include "common.cuh"

namespace gde {

// keep[i] = 1 if (u[i], v[i]) is not yet in row u[i]
__global__ void k_mark_new(int64_t m, const int32_t *__restrict__ u, const int32_t *__restrict__ v,
                           const int64_t *__restrict__ off, const int32_t *__restrict__ col,
                           uint8_t *__restrict__ keep) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= m) return;
    const int32_t a = u[i], b = v[i];
    int64_t lo = off[a], hi = off[a + 1];
    while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        if (col[mid] < b) lo = mid + 1; else hi = mid;
    }
    keep[i] = (lo < off[a + 1] && col[lo] == b) ? 0 : 1;
}

__global__ void k_gather_deg(int64_t rows, const int32_t *__restrict__ row, const int32_t *__restrict__ deg,
                             int32_t *__restrict__ out) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < rows) out[i] = deg[row[i]];
}

// old row bounds of the changed rows
__global__ void k_row_bounds(int64_t rows, const int32_t *__restrict__ row, const int64_t *__restrict__ off,
                             int64_t *__restrict__ rb, int64_t *__restrict__ re) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= rows) return;
    rb[i] = off[row[i]];
    re[i] = off[row[i] + 1];
}

// first index in [lo, hi) of the ascending array a whose value is >= x (hi if none)
__device__ __forceinline__ int64_t lower_index(const int32_t *__restrict__ a, int64_t lo, int64_t hi, int64_t x) {
    while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        if (a[mid] < x) lo = mid + 1; else hi = mid;
    }
    return lo;
}

constexpr int kOffsetTile = 1024;  // offsets per warp tile

// noff[u] = off[u] + (adjacencies added to rows before u): the number of changed rows below
// u (a search over the ascending changed rows) indexes row_start, the running total of
// their additions.  A warp searches once for its tile of consecutive u, then each u only
// within the changed rows that fall inside the tile.
__global__ void k_new_offsets(int64_t n, const int64_t *__restrict__ off, const int32_t *__restrict__ row,
                              const int64_t *__restrict__ row_start, int64_t rows, int64_t added,
                              int64_t *__restrict__ noff) {
    const int lane = threadIdx.x & 31;
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t t0 = warp * kOffsetTile; t0 <= n; t0 += nwarps * kOffsetTile) {
        const int64_t t1 = t0 + kOffsetTile < n + 1 ? t0 + kOffsetTile : n + 1;
        const int64_t first = lower_index(row, 0, rows, t0);        // changed rows below t0
        const int64_t last = lower_index(row, first, rows, t1);     // changed rows below t1
        for (int64_t u = t0 + lane; u < t1; u += 32) {
            const int64_t lo = lower_index(row, first, last, u);    // changed rows below u
            noff[u] = off[u] + (lo < rows ? row_start[lo] : added);
        }
    }
}

// first index in [lo, hi) of the ascending array a whose value exceeds x (hi if none)
__device__ __forceinline__ int64_t upper_index(const int64_t *__restrict__ a, int64_t lo, int64_t hi, int64_t x) {
    while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        if (a[mid] <= x) lo = mid + 1; else hi = mid;
    }
    return lo;
}

constexpr int kShiftTile = 1024;  // CSR entries per warp tile of the column shift

// Each old CSR entry e moves by the additions to earlier rows, plus, inside a changed row, by
// that row's added columns that sort before it.  Rows are sorted, so the copy is a shift that
// changes only at the changed rows: a coalesced streaming pass.  A warp takes a tile of
// consecutive entries and finds the changed rows that reach into it once (one search over
// the row starts); each entry then only searches that short range, which is empty unless a
// changed row starts inside the tile.
// The packed columns (when colp is not NULL) move with their columns: a column's packed word
// only changes if its node's degree changed, which k_fix_codes handles.
__global__ void k_shift_columns(int64_t nnz, const int32_t *__restrict__ col, const int64_t *__restrict__ rb,
                                const int64_t *__restrict__ re, const int64_t *__restrict__ row_start,
                                const int32_t *__restrict__ row_cnt, int64_t rows,
                                const int32_t *__restrict__ added, int32_t *__restrict__ ncol,
                                const uint32_t *__restrict__ colp, uint32_t *__restrict__ ncolp) {
    const int lane = threadIdx.x & 31;
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t t0 = warp * kShiftTile; t0 < nnz; t0 += nwarps * kShiftTile) {
        const int64_t t1 = t0 + kShiftTile < nnz ? t0 + kShiftTile : nnz;
        const int64_t first = upper_index(rb, 0, rows, t0);          // rows starting after t0
        const int64_t last = upper_index(rb, first, rows, t1 - 1);   // rows starting after t1 - 1
        for (int64_t e = t0 + lane; e < t1; e += 32) {
            const int32_t c = col[e];
            const int64_t i = upper_index(rb, first, last, e) - 1;  // last changed row starting at or before e
            int64_t shift = 0;
            if (i >= 0) {
                if (e < re[i]) {
                    const int32_t *a = added + row_start[i];
                    int32_t l = 0, h = row_cnt[i];  // added columns of that row below c
                    while (l < h) {
                        const int32_t m = (l + h) >> 1;
                        if (a[m] < c) l = m + 1; else h = m;
                    }
                    shift = row_start[i] + l;
                } else {
                    shift = row_start[i] + row_cnt[i];
                }
            }
            ncol[e + shift] = c;
            if (ncolp) ncolp[e + shift] = colp[e];
        }
    }
}

__global__ void k_deg_add(int64_t rows, const int32_t *__restrict__ row, const int32_t *__restrict__ cnt,
                          int32_t *__restrict__ deg, int *max_deg) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= rows) return;
    const int32_t d = deg[row[i]] + cnt[i];
    deg[row[i]] = d;
    atomicMax(max_deg, d);
}

// one thread per added adjacency i (row u, column v; the list is sorted by (u, v)): its place
// is noff[u] + (its index among u's added) + (old columns of u below v).  With packed columns
// (ncolp not NULL) it also writes v's packed word from v's degree after the batch.
__global__ void k_place_added(int64_t m, const int32_t *__restrict__ u, const int32_t *__restrict__ v,
                              const int64_t *__restrict__ off, const int32_t *__restrict__ col,
                              const int64_t *__restrict__ noff, const int32_t *__restrict__ row,
                              const int64_t *__restrict__ row_start, int64_t rows, int32_t *__restrict__ ncol,
                              const int32_t *__restrict__ deg, uint32_t *__restrict__ ncolp, int idbits,
                              int code_exact) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= m) return;
    const int32_t a = u[i], c = v[i];
    int64_t rl = 0, rh = rows;  // a's position among the changed rows
    while (rl < rh) {
        const int64_t mid = (rl + rh) >> 1;
        if (row[mid] < a) rl = mid + 1; else rh = mid;
    }
    int64_t lo = off[a], hi = off[a + 1];
    while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        if (col[mid] < c) lo = mid + 1; else hi = mid;
    }
    const int64_t at = noff[a] + (i - row_start[rl]) + (lo - off[a]);
    ncol[at] = c;
    if (ncolp) ncolp[at] = (uint32_t)c | (degree_code(deg[c], code_exact) << idbits);
}

// Packed words of the columns that name a node whose degree code the batch changed.  The
// graph is symmetric, so the entries naming c sit in the rows of c's neighbours: one warp per
// changed row c walks c's new row and, for each neighbour u, finds c in u's new row (binary
// search) and rewrites its word.  An entry that is not found (the graph was not symmetric
// after all) sets *missing, and the caller then drops the packed array.
__global__ void k_fix_codes(int64_t rows, const int32_t *__restrict__ row, const int32_t *__restrict__ old_deg,
                            const int32_t *__restrict__ deg, const int64_t *__restrict__ noff,
                            const int32_t *__restrict__ ncol, uint32_t *__restrict__ ncolp, int idbits,
                            int code_exact, unsigned *missing) {
    const int lane = threadIdx.x & 31;
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t i = warp; i < rows; i += nwarps) {
        const int32_t c = row[i];
        const uint32_t code = degree_code(deg[c], code_exact);
        if (code == degree_code(old_deg[i], code_exact)) continue;
        const uint32_t word = (uint32_t)c | (code << idbits);
        for (int64_t k = noff[c] + lane; k < noff[c + 1]; k += 32) {
            const int32_t u = ncol[k];
            int64_t lo = noff[u], hi = noff[u + 1];
            while (lo < hi) {
                const int64_t mid = (lo + hi) >> 1;
                if (ncol[mid] < c) lo = mid + 1; else hi = mid;
            }
            if (lo < noff[u + 1] && ncol[lo] == c) ncolp[lo] = word;
            else atomicOr(missing, 1u);
        }
    }
}

static unsigned blocks_for(int64_t m) {
    const int64_t b = (m + kThreads - 1) / kThreads;
    return (unsigned)(b > 0 ? b : 1);
}

// Buffers of the CSR rebuild, kept between batches so that a batch allocates nothing: the
// spare column array (the merge writes there, then it swaps with the graph's), the spare
// offsets, and an arena for the batch's own arrays (its adjacencies, the changed rows and
// their bounds), which grows only when a larger batch arrives.
struct UpdateScratch {
    int32_t *col = nullptr;
    int64_t col_cap = 0;         // entries of the spare column array
    int64_t graph_col_cap = 0;   // entries of the array the graph's columns sit in
    int64_t *off = nullptr;      // n + 1
    int *dmax = nullptr;         // [0]: max degree, [1]: packed-word entries not found
    uint32_t *colp = nullptr;    // spare packed columns
    int64_t colp_cap = 0;
    uint8_t *arena = nullptr;
    size_t arena_cap = 0;
    int64_t n = -1;
};

void update_scratch_free(Graph &g) {
    UpdateScratch *u = g.upd;
    if (!u) return;
    dfree(u->col); dfree(u->off); dfree(u->dmax); dfree(u->colp); dfree(u->arena);
    delete u;
    g.upd = nullptr;
}

// Hands out 256-byte aligned pieces of the arena in order.
struct Carver {
    uint8_t *base;
    size_t cap, used = 0;
    template <typename T> T *take(int64_t count) {
        const size_t at = (used + 255) & ~(size_t)255;
        const size_t bytes = sizeof(T) * (size_t)(count > 0 ? count : 1);
        GDE_REQUIRE(at + bytes <= cap, GDE_ECUDA, "edge batch arena too small");
        used = at + bytes;
        return reinterpret_cast<T *>(base + at);
    }
};

// bytes of the arena a batch of mp directed adjacencies may need (every per-adjacency and
// per-row array at its largest, plus alignment)
static size_t arena_bytes(int64_t mp) {
    return (size_t)mp * (4 + 4 + 1 + 4 + 4 + 4 + 4 + 8 + 4 + 8 + 8) + 12 * 256;
}

static UpdateScratch *update_scratch_base(Graph &g) {
    if (g.upd && g.upd->n != g.n) update_scratch_free(g);
    if (!g.upd) {
        UpdateScratch *u = new UpdateScratch();
        g.upd = u;
        const int64_t n = g.n;
        u->n = n;
        u->off = (int64_t *)dmalloc(8 * (size_t)(n + 1), "CSR offsets");
        u->dmax = (int *)dmalloc(2 * sizeof(int), "max degree");
        u->graph_col_cap = g.nnz;  // the graph's columns were allocated to size
    }
    return g.upd;
}

static Carver batch_arena(Graph &g, int64_t mp) {
    UpdateScratch *u = update_scratch_base(g);
    const size_t need = arena_bytes(mp);
    if (u->arena_cap < need) {
        const size_t cap = need + need / 2;
        dfree(u->arena);
        u->arena = nullptr;
        u->arena_cap = 0;
        u->arena = (uint8_t *)dmalloc(cap, "edge batch");
        u->arena_cap = cap;
    }
    return Carver{u->arena, u->arena_cap};
}

static UpdateScratch *update_scratch(Graph &g, int64_t nnz_new) {
    UpdateScratch *u = update_scratch_base(g);
    if (u->col_cap < nnz_new) {
        // room for growth: later batches reuse the buffer
        const int64_t cap = nnz_new + nnz_new / 4 + 1024;
        dfree(u->col);
        u->col = nullptr;
        u->col = (int32_t *)dmalloc(4 * (size_t)cap, "CSR columns");
        u->col_cap = cap;
    }
    return u;
}

void edge_batch_free(EdgeBatch &b) {
    if (b.owned) {
        dfree(b.u); dfree(b.v); dfree(b.row); dfree(b.row_cnt); dfree(b.row_start); dfree(b.old_deg);
    }
    b = EdgeBatch{};
}

// Sorts keys below `bound` ascending: least-significant-digit radix sort, 12-bit digits, as
// many passes as bound has digits (a batch's keys are few, so counting passes beat comparisons).
static void radix_sort_keys(std::vector<uint64_t> &k, uint64_t bound) {
    constexpr int kBits = 12;
    constexpr size_t kBuckets = (size_t)1 << kBits;
    std::vector<uint64_t> tmp(k.size());
    std::vector<size_t> cnt(kBuckets);
    for (int shift = 0; shift < 64 && (shift == 0 || (bound - 1) >> shift); shift += kBits) {
        std::fill(cnt.begin(), cnt.end(), 0);
        for (uint64_t x : k) cnt[(x >> shift) & (kBuckets - 1)]++;
        size_t sum = 0;
        for (size_t b = 0; b < kBuckets; b++) {
            const size_t c = cnt[b];
            cnt[b] = sum;
            sum += c;
        }
        for (uint64_t x : k) tmp[cnt[(x >> shift) & (kBuckets - 1)]++] = x;
        k.swap(tmp);
    }
}

int64_t graph_insert_edges(Graph &g, const int32_t *src, const int32_t *dst, int64_t m, bool dev_ptrs,
                           EdgeBatch *out) {
    GDE_REQUIRE(m >= 0, GDE_EINVAL, "edge count must be >= 0");
    GDE_REQUIRE(m == 0 || (src && dst), GDE_EINVAL, "src or dst is NULL");
    cudaStream_t s = g.stream;
    std::vector<int32_t> hs((size_t)m), hd((size_t)m);
    if (m > 0) {
        const cudaMemcpyKind k = dev_ptrs ? cudaMemcpyDeviceToHost : cudaMemcpyHostToHost;
        GDE_CUDA(cudaMemcpyAsync(hs.data(), src, 4 * (size_t)m, k, s));
        GDE_CUDA(cudaMemcpyAsync(hd.data(), dst, 4 * (size_t)m, k, s));
        GDE_CUDA(cudaStreamSynchronize(s));
    }
    // both directions, no self-loops, sorted by (u, v), unique: (u, v) packed as u n + v
    const uint64_t n64 = (uint64_t)g.n;
    std::vector<uint64_t> p;
    p.reserve(2 * (size_t)m);
    for (int64_t i = 0; i < m; i++) {
        const int32_t a = hs[(size_t)i], b = hd[(size_t)i];
        GDE_REQUIRE(a >= 0 && a < g.n && b >= 0 && b < g.n, GDE_EINVAL, "edge endpoint out of range");
        if (a == b) continue;
        p.push_back((uint64_t)a * n64 + (uint64_t)b);
        p.push_back((uint64_t)b * n64 + (uint64_t)a);
    }
    radix_sort_keys(p, n64 * n64);
    p.erase(std::unique(p.begin(), p.end()), p.end());
    const int64_t mp = (int64_t)p.size();
    if (out) *out = EdgeBatch{};
    if (mp == 0) return 0;

    int64_t added = 0;
    {
        Carver arena = batch_arena(g, mp);
        std::vector<int32_t> pu((size_t)mp), pv((size_t)mp);
        for (int64_t i = 0; i < mp; i++) {
            pu[(size_t)i] = (int32_t)(p[(size_t)i] / n64);
            pv[(size_t)i] = (int32_t)(p[(size_t)i] % n64);
        }
        int32_t *du = arena.take<int32_t>(mp);
        int32_t *dv = arena.take<int32_t>(mp);
        uint8_t *keep = arena.take<uint8_t>(mp);
        GDE_CUDA(cudaMemcpyAsync(du, pu.data(), 4 * (size_t)mp, cudaMemcpyHostToDevice, s));
        GDE_CUDA(cudaMemcpyAsync(dv, pv.data(), 4 * (size_t)mp, cudaMemcpyHostToDevice, s));
        k_mark_new<<<blocks_for(mp), kThreads, 0, s>>>(mp, du, dv, g.off, g.col, keep);
        GDE_CUDA(cudaGetLastError());
        g.prof.launched();
        std::vector<uint8_t> hk((size_t)mp);
        GDE_CUDA(cudaMemcpyAsync(hk.data(), keep, (size_t)mp, cudaMemcpyDeviceToHost, s));
        GDE_CUDA(cudaStreamSynchronize(s));
        // the new adjacencies (still sorted) and the rows that gain them
        std::vector<int32_t> nu, nv, rows, rcnt;
        std::vector<int64_t> rstart;
        for (int64_t i = 0; i < mp; i++) {
            if (!hk[(size_t)i]) continue;
            const int32_t a = pu[(size_t)i];
            if (rows.empty() || rows.back() != a) {
                rows.push_back(a);
                rcnt.push_back(0);
                rstart.push_back((int64_t)nu.size());
            }
            rcnt.back()++;
            nu.push_back(a);
            nv.push_back(pv[(size_t)i]);
        }
        added = (int64_t)nu.size();
        if (added == 0) return 0;
        GDE_REQUIRE(g.nnz + added < ((int64_t)1 << 40), GDE_EINVAL, "graph too large");
        const int64_t nrows = (int64_t)rows.size();
        EdgeBatch eb{};
        eb.owned = false;
        eb.m = added;
        eb.rows = nrows;
        eb.u = arena.take<int32_t>(added);
        eb.v = arena.take<int32_t>(added);
        eb.row = arena.take<int32_t>(nrows);
        eb.row_cnt = arena.take<int32_t>(nrows);
        eb.row_start = arena.take<int64_t>(nrows);
        eb.old_deg = arena.take<int32_t>(nrows);
        {
            GDE_CUDA(cudaMemcpyAsync(eb.u, nu.data(), 4 * (size_t)added, cudaMemcpyHostToDevice, s));
            GDE_CUDA(cudaMemcpyAsync(eb.v, nv.data(), 4 * (size_t)added, cudaMemcpyHostToDevice, s));
            GDE_CUDA(cudaMemcpyAsync(eb.row, rows.data(), 4 * (size_t)nrows, cudaMemcpyHostToDevice, s));
            GDE_CUDA(cudaMemcpyAsync(eb.row_cnt, rcnt.data(), 4 * (size_t)nrows, cudaMemcpyHostToDevice, s));
            GDE_CUDA(cudaMemcpyAsync(eb.row_start, rstart.data(), 8 * (size_t)nrows, cudaMemcpyHostToDevice, s));
            // new offsets, shifted columns, the degrees of the changed rows, placed additions;
            // on a symmetric graph the packed columns are carried along and then patched where
            // a degree code changed, else they are dropped and rebuilt on next use
            const int64_t n = g.n;
            UpdateScratch *u = update_scratch(g, g.nnz + added);
            int64_t *noff = u->off;
            int *dmax = u->dmax;
            const bool keep_colp = g.colp_valid && g.colp && g.symmetric && g.colp_idbits > 0;
            uint32_t *ncolp = nullptr;
            if (keep_colp) {
                const int64_t need = g.nnz + added;
                if (u->colp_cap < need) {
                    const int64_t cap = need + need / 4 + 1024;
                    dfree(u->colp);
                    u->colp = nullptr;
                    u->colp_cap = 0;
                    u->colp = (uint32_t *)dmalloc(4 * (size_t)cap, "packed columns");
                    u->colp_cap = cap;
                }
                ncolp = u->colp;
            }
            int64_t *rb = arena.take<int64_t>(nrows);
            int64_t *re = arena.take<int64_t>(nrows);
            const int hstate[2] = {g.max_degree, 0};
            GDE_CUDA(cudaMemcpyAsync(dmax, hstate, sizeof(hstate), cudaMemcpyHostToDevice, s));
            k_gather_deg<<<blocks_for(nrows), kThreads, 0, s>>>(nrows, eb.row, g.deg, eb.old_deg);
            GDE_CUDA(cudaGetLastError());
            k_row_bounds<<<blocks_for(nrows), kThreads, 0, s>>>(nrows, eb.row, g.off, rb, re);
            GDE_CUDA(cudaGetLastError());
            k_new_offsets<<<kSMs * 16, kThreads, 0, s>>>(n, g.off, eb.row, eb.row_start, nrows, added, noff);
            GDE_CUDA(cudaGetLastError());
            int32_t *ncol = u->col;
            int launched = 5;
            if (g.nnz > 0) {
                k_shift_columns<<<kSMs * 16, kThreads, 0, s>>>(g.nnz, g.col, rb, re, eb.row_start, eb.row_cnt, nrows,
                                                               eb.v, ncol, keep_colp ? g.colp : nullptr, ncolp);
                GDE_CUDA(cudaGetLastError());
                launched++;
            }
            k_deg_add<<<blocks_for(nrows), kThreads, 0, s>>>(nrows, eb.row, eb.row_cnt, g.deg, dmax);
            GDE_CUDA(cudaGetLastError());
            k_place_added<<<blocks_for(added), kThreads, 0, s>>>(added, eb.u, eb.v, g.off, g.col, noff, eb.row,
                                                                 eb.row_start, nrows, ncol, g.deg, ncolp,
                                                                 g.colp_idbits, g.colp_exact);
            GDE_CUDA(cudaGetLastError());
            if (keep_colp) {
                k_fix_codes<<<blocks_for(32 * nrows), kThreads, 0, s>>>(nrows, eb.row, eb.old_deg, g.deg, noff, ncol,
                                                                       ncolp, g.colp_idbits, g.colp_exact,
                                                                       reinterpret_cast<unsigned *>(dmax + 1));
                GDE_CUDA(cudaGetLastError());
                launched++;
            }
            int hres[2] = {0, 0};
            GDE_CUDA(cudaMemcpyAsync(hres, dmax, sizeof(hres), cudaMemcpyDeviceToHost, s));
            GDE_CUDA(cudaStreamSynchronize(s));
            g.prof.launched(launched);
            // the rebuilt arrays become the graph's, the old ones the next batch's spares
            std::swap(g.col, u->col);
            std::swap(g.off, u->off);
            std::swap(u->col_cap, u->graph_col_cap);
            if (keep_colp && hres[1] == 0) {
                std::swap(g.colp, u->colp);
                std::swap(g.colp_cap, u->colp_cap);
            } else {
                g.colp_valid = false;
                if (keep_colp) g.symmetric = false;  // an entry had no mirror
            }
            g.nnz += added;
            g.max_degree = hres[0];
        }
        if (out) *out = eb;
    }
    graph_changed(g);
    return added;
}

}  // namespace gde
