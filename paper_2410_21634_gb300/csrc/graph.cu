// CSR graph store: upload, degree array, validation (Section 2 notation: A symmetric,
// no self-loops, d_u = |N(u)|).
#include "common.cuh"

namespace gde {

// one thread per row: offsets monotone, columns in range, strictly increasing, no u in N(u);
// also writes d_u and tracks the maximum degree
__global__ void k_validate_rows(int64_t n, int64_t nnz, const int64_t *__restrict__ off,
                                const int32_t *__restrict__ col, int32_t *__restrict__ deg,
                                unsigned *bits, int *max_deg) {
    int64_t u = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (u == 0 && (off[0] != 0 || off[n] != nnz)) atomicOr(bits, kBadOffsets);
    if (u >= n) return;
    int64_t b = off[u], e = off[u + 1];
    if (e < b || b < 0 || e > nnz) {
        atomicOr(bits, kBadOffsets);
        deg[u] = 0;
        return;
    }
    int64_t d = e - b;
    if (d >= (int64_t)1 << 31) {
        atomicOr(bits, kBadOffsets);
        deg[u] = 0;
        return;
    }
    deg[u] = (int32_t)d;
    atomicMax(max_deg, (int)d);
    unsigned local = 0;
    int32_t prev = -1;
    for (int64_t k = b; k < e; k++) {
        int32_t v = col[k];
        if (v < 0 || v >= n) local |= kBadColRange;
        if (v <= prev) local |= kUnsorted;
        if (v == (int32_t)u) local |= kSelfLoop;
        prev = v;
    }
    if (local) atomicOr(bits, local);
}

// one thread per CSR entry (u,v): u must appear in row v (binary search)
__global__ void k_check_symmetric(int64_t n, int64_t nnz, const int64_t *__restrict__ off,
                                  const int32_t *__restrict__ col, unsigned *bits) {
    int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (k >= nnz) return;
    // row of entry k: largest u with off[u] <= k
    int64_t lo = 0, hi = n;  // off[lo] <= k < off[hi]
    while (hi - lo > 1) {
        int64_t mid = (lo + hi) >> 1;
        if (off[mid] <= k) lo = mid; else hi = mid;
    }
    int32_t u = (int32_t)lo, v = col[k];
    if (v < 0 || v >= n) return;  // reported by the row check
    int64_t a = off[v], b = off[v + 1];
    while (a < b) {
        int64_t mid = (a + b) >> 1;
        int32_t c = col[mid];
        if (c == u) return;
        if (c < u) a = mid + 1; else b = mid;
    }
    atomicOr(bits, kAsymmetric);
}

void graph_validate(Graph &g, bool check_symmetric, unsigned *bits_out) {
    unsigned *d_bits = nullptr;
    int *d_max = nullptr;
    d_bits = (unsigned *)dmalloc(sizeof(unsigned) * 2, "validation flags");
    d_max = (int *)(d_bits + 1);
    try {
        GDE_CUDA(cudaMemsetAsync(d_bits, 0, sizeof(unsigned) * 2, g.stream));
        int64_t blocks = (g.n + kThreads - 1) / kThreads;
        if (blocks > 0)
            k_validate_rows<<<(unsigned)blocks, kThreads, 0, g.stream>>>(g.n, g.nnz, g.off, g.col,
                                                                        g.deg, d_bits, d_max);
        else
            k_validate_rows<<<1, kThreads, 0, g.stream>>>(g.n, g.nnz, g.off, g.col, g.deg, d_bits,
                                                          d_max);
        GDE_CUDA(cudaGetLastError());
        unsigned h[2] = {0, 0};
        GDE_CUDA(cudaMemcpyAsync(h, d_bits, sizeof(h), cudaMemcpyDeviceToHost, g.stream));
        GDE_CUDA(cudaStreamSynchronize(g.stream));
        if (h[0] == 0 && check_symmetric && g.nnz > 0) {
            int64_t eb = (g.nnz + kThreads - 1) / kThreads;
            k_check_symmetric<<<(unsigned)eb, kThreads, 0, g.stream>>>(g.n, g.nnz, g.off, g.col,
                                                                       d_bits);
            GDE_CUDA(cudaGetLastError());
            GDE_CUDA(cudaMemcpyAsync(h, d_bits, sizeof(unsigned), cudaMemcpyDeviceToHost,
                                     g.stream));
            GDE_CUDA(cudaStreamSynchronize(g.stream));
        }
        *bits_out = h[0];
        g.max_degree = (int32_t)h[1];
        g.symmetric = h[0] == 0 && check_symmetric;
    } catch (...) {
        dfree(d_bits);
        throw;
    }
    dfree(d_bits);
}

}  // namespace gde
