// Edge insertion into the device CSR: the dynamic setting of Section 4, where a snapshot
// G_t becomes G_{t+1} through a batch of insertion events.  Each undirected edge adds the
// adjacencies u -> v and v -> u; self-loops and adjacencies already present are skipped,
// so rows stay sorted and duplicate-free (the store's invariant).
//
// The batch is normalised on the host (it is small next to the graph), then the device
// drops adjacencies already in their row (binary search), computes the new degrees and
// offsets (scan), and rebuilds the column array in one pass: a warp per row moves the old
// columns to their new places (shifted past the added columns that sort before them), and
// a thread per added adjacency drops it into its gap.
#include <algorithm>
#include <utility>
#include <vector>

#include "common.cuh"
#include "detsort.cuh"

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

// per-row added counts and first-added index, from the sorted list of rows that gained
__global__ void k_scatter_rows(int64_t rows, const int32_t *__restrict__ row, const int32_t *__restrict__ cnt,
                               const int64_t *__restrict__ start, int32_t *__restrict__ add_cnt,
                               int64_t *__restrict__ add_start) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= rows) return;
    add_cnt[row[i]] = cnt[i];
    add_start[row[i]] = start[i];
}

__global__ void k_gather_deg(int64_t rows, const int32_t *__restrict__ row, const int32_t *__restrict__ deg,
                             int32_t *__restrict__ out) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < rows) out[i] = deg[row[i]];
}

__global__ void k_new_degrees(int64_t n, int32_t *__restrict__ deg, const int32_t *__restrict__ add_cnt,
                              int64_t *__restrict__ deg64, int *max_deg) {
    const int64_t u = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (u >= n) return;
    const int32_t d = deg[u] + add_cnt[u];
    deg[u] = d;
    deg64[u] = d;
    if (add_cnt[u]) atomicMax(max_deg, d);
}

// one warp per row: old column k of row u goes to noff[u] + k + (added columns of u below it)
__global__ void k_merge_rows(int64_t n, const int64_t *__restrict__ off, const int32_t *__restrict__ col,
                             const int64_t *__restrict__ noff, int32_t *__restrict__ ncol,
                             const int32_t *__restrict__ add_cnt, const int64_t *__restrict__ add_start,
                             const int32_t *__restrict__ added) {
    const int lane = threadIdx.x & 31;
    const int64_t w0 = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t u = w0; u < n; u += nw) {
        const int64_t b = off[u], e = off[u + 1], nb = noff[u];
        const int32_t k = add_cnt[u];
        const int32_t *a = added + (k ? add_start[u] : 0);
        for (int64_t i = b + lane; i < e; i += 32) {
            const int32_t c = col[i];
            int32_t lo = 0, hi = k;  // added columns below c
            while (lo < hi) {
                const int32_t mid = (lo + hi) >> 1;
                if (a[mid] < c) lo = mid + 1; else hi = mid;
            }
            ncol[nb + (i - b) + lo] = c;
        }
    }
}

// one thread per added adjacency (u, v): its place is noff[u] + (its index among u's added)
// + (old columns of u below v)
__global__ void k_place_added(int64_t m, const int32_t *__restrict__ u, const int32_t *__restrict__ v,
                              const int64_t *__restrict__ off, const int32_t *__restrict__ col,
                              const int64_t *__restrict__ noff, const int64_t *__restrict__ add_start,
                              int32_t *__restrict__ ncol) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= m) return;
    const int32_t a = u[i], c = v[i];
    int64_t lo = off[a], hi = off[a + 1];
    while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        if (col[mid] < c) lo = mid + 1; else hi = mid;
    }
    ncol[noff[a] + (i - add_start[a]) + (lo - off[a])] = c;
}

static unsigned blocks_for(int64_t m) {
    const int64_t b = (m + kThreads - 1) / kThreads;
    return (unsigned)(b > 0 ? b : 1);
}

void edge_batch_free(EdgeBatch &b) {
    dfree(b.u); dfree(b.v); dfree(b.row); dfree(b.row_cnt); dfree(b.row_start); dfree(b.old_deg);
    b = EdgeBatch{};
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
    // both directions, no self-loops, sorted by (u, v), unique
    std::vector<std::pair<int32_t, int32_t>> p;
    p.reserve(2 * (size_t)m);
    for (int64_t i = 0; i < m; i++) {
        const int32_t a = hs[(size_t)i], b = hd[(size_t)i];
        GDE_REQUIRE(a >= 0 && a < g.n && b >= 0 && b < g.n, GDE_EINVAL, "edge endpoint out of range");
        if (a == b) continue;
        p.emplace_back(a, b);
        p.emplace_back(b, a);
    }
    std::sort(p.begin(), p.end());
    p.erase(std::unique(p.begin(), p.end()), p.end());
    const int64_t mp = (int64_t)p.size();
    if (out) *out = EdgeBatch{};
    if (mp == 0) return 0;

    std::vector<void *> tmp;
    auto alloc = [&](size_t bytes, const char *what) {
        void *q = dmalloc(bytes, what);
        tmp.push_back(q);
        return q;
    };
    int64_t added = 0;
    try {
        std::vector<int32_t> pu((size_t)mp), pv((size_t)mp);
        for (int64_t i = 0; i < mp; i++) { pu[(size_t)i] = p[(size_t)i].first; pv[(size_t)i] = p[(size_t)i].second; }
        int32_t *du = (int32_t *)alloc(4 * (size_t)mp, "edge batch");
        int32_t *dv = (int32_t *)alloc(4 * (size_t)mp, "edge batch");
        uint8_t *keep = (uint8_t *)alloc((size_t)mp, "edge batch");
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
        if (added == 0) {
            for (void *q : tmp) dfree(q);
            return 0;
        }
        GDE_REQUIRE(g.nnz + added < ((int64_t)1 << 40), GDE_EINVAL, "graph too large");
        const int64_t nrows = (int64_t)rows.size();
        EdgeBatch eb{};
        eb.m = added;
        eb.rows = nrows;
        eb.u = (int32_t *)dmalloc(4 * (size_t)added, "edge batch");
        eb.v = (int32_t *)dmalloc(4 * (size_t)added, "edge batch");
        eb.row = (int32_t *)dmalloc(4 * (size_t)nrows, "edge batch");
        eb.row_cnt = (int32_t *)dmalloc(4 * (size_t)nrows, "edge batch");
        eb.row_start = (int64_t *)dmalloc(8 * (size_t)nrows, "edge batch");
        eb.old_deg = (int32_t *)dmalloc(4 * (size_t)nrows, "edge batch");
        try {
            GDE_CUDA(cudaMemcpyAsync(eb.u, nu.data(), 4 * (size_t)added, cudaMemcpyHostToDevice, s));
            GDE_CUDA(cudaMemcpyAsync(eb.v, nv.data(), 4 * (size_t)added, cudaMemcpyHostToDevice, s));
            GDE_CUDA(cudaMemcpyAsync(eb.row, rows.data(), 4 * (size_t)nrows, cudaMemcpyHostToDevice, s));
            GDE_CUDA(cudaMemcpyAsync(eb.row_cnt, rcnt.data(), 4 * (size_t)nrows, cudaMemcpyHostToDevice, s));
            GDE_CUDA(cudaMemcpyAsync(eb.row_start, rstart.data(), 8 * (size_t)nrows, cudaMemcpyHostToDevice, s));
            // per-row counts and starts over all n rows; new degrees, offsets, columns
            const int64_t n = g.n;
            int32_t *add_cnt = (int32_t *)alloc(4 * (size_t)n, "row adds");
            int64_t *add_start = (int64_t *)alloc(8 * (size_t)n, "row adds");
            int64_t *deg64 = (int64_t *)alloc(8 * (size_t)n, "new degrees");
            int64_t *noff = (int64_t *)alloc(8 * (size_t)(n + 1), "CSR offsets");
            int64_t *scr = (int64_t *)alloc(scan_scratch_bytes(n), "scan scratch");
            int *dmax = (int *)alloc(sizeof(int), "max degree");
            GDE_CUDA(cudaMemsetAsync(add_cnt, 0, 4 * (size_t)n, s));
            GDE_CUDA(cudaMemcpyAsync(dmax, &g.max_degree, sizeof(int), cudaMemcpyHostToDevice, s));
            k_scatter_rows<<<blocks_for(nrows), kThreads, 0, s>>>(nrows, eb.row, eb.row_cnt, eb.row_start,
                                                                   add_cnt, add_start);
            GDE_CUDA(cudaGetLastError());
            // degrees before the update, for the caller's state corrections
            k_gather_deg<<<blocks_for(nrows), kThreads, 0, s>>>(nrows, eb.row, g.deg, eb.old_deg);
            GDE_CUDA(cudaGetLastError());
            k_new_degrees<<<blocks_for(n), kThreads, 0, s>>>(n, g.deg, add_cnt, deg64, dmax);
            GDE_CUDA(cudaGetLastError());
            exclusive_scan_i64(deg64, noff, n, noff + n, scr, s);
            int32_t *ncol = (int32_t *)dmalloc(4 * (size_t)(g.nnz + added), "CSR columns");
            try {
                k_merge_rows<<<kSMs * 8, kThreads, 0, s>>>(n, g.off, g.col, noff, ncol, add_cnt, add_start, eb.v);
                GDE_CUDA(cudaGetLastError());
                k_place_added<<<blocks_for(added), kThreads, 0, s>>>(added, eb.u, eb.v, g.off, g.col, noff,
                                                                     add_start, ncol);
                GDE_CUDA(cudaGetLastError());
                int hmax = 0;
                GDE_CUDA(cudaMemcpyAsync(&hmax, dmax, sizeof(int), cudaMemcpyDeviceToHost, s));
                GDE_CUDA(cudaStreamSynchronize(s));
                g.prof.launched(7);
                // swap in the new arrays (noff leaves the temporaries)
                dfree(g.col);
                g.col = ncol;
                dfree(g.off);
                g.off = noff;
                tmp.erase(std::find(tmp.begin(), tmp.end(), (void *)noff));
                g.nnz += added;
                g.max_degree = hmax;
            } catch (...) {
                dfree(ncol);
                throw;
            }
        } catch (...) {
            edge_batch_free(eb);
            throw;
        }
        if (out) *out = eb; else edge_batch_free(eb);
    } catch (...) {
        for (void *q : tmp) dfree(q);
        throw;
    }
    for (void *q : tmp) dfree(q);
    graph_changed(g);
    return added;
}

}  // namespace gde
