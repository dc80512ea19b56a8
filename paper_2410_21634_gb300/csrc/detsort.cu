// Stable LSD radix sort (4-bit digits) and exclusive scans for the deterministic scatter.
//
// A tile is kSortThreads x kSortItems keys; thread t holds keys t*kSortItems .. +kSortItems-1 of
// its tile, so (thread, item) order is the input order.  Per pass: k_sort_hist counts the
// digits of every tile (digit-major table), an exclusive scan turns the table into global
// offsets, and k_sort_scatter ranks every key among the equal digits of its tile (a block-wide
// scan over per-thread digit counts) and writes it to offset + rank.  Equal keys keep their
// input order, which the deterministic scatter relies on.
#include "common.cuh"
#include "detsort.cuh"

namespace gde {

constexpr int kSortThreads = 256;
constexpr int kSortItems = 8;
constexpr int kSortTile = kSortThreads * kSortItems;
constexpr int kRadix = 16;
constexpr int kScanTile = 2048;

__global__ void __launch_bounds__(kSortThreads) k_sort_hist(const uint32_t *__restrict__ keys, int64_t n,
                                                            int shift, int64_t ntiles,
                                                            int64_t *__restrict__ table) {
    __shared__ unsigned cnt[kRadix];
    if (threadIdx.x < kRadix) cnt[threadIdx.x] = 0;
    __syncthreads();
    const int64_t tile = blockIdx.x;
    const int64_t base = tile * kSortTile;
    for (int i = threadIdx.x; i < kSortTile; i += kSortThreads) {
        const int64_t k = base + i;
        if (k < n) atomicAdd(&cnt[(keys[k] >> shift) & (kRadix - 1)], 1u);
    }
    __syncthreads();
    if (threadIdx.x < kRadix) table[(int64_t)threadIdx.x * ntiles + tile] = cnt[threadIdx.x];
}

template <typename V>
__global__ void __launch_bounds__(kSortThreads) k_sort_scatter(const uint32_t *__restrict__ keys_in,
                                                               const V *__restrict__ vals_in,
                                                               uint32_t *__restrict__ keys_out,
                                                               V *__restrict__ vals_out, int64_t n,
                                                               int shift, int64_t ntiles,
                                                               const int64_t *__restrict__ offsets) {
    __shared__ unsigned cnt[kRadix * kSortThreads];  // [digit][thread]
    __shared__ unsigned warp_tot[kSortThreads / 32];
    const int t = threadIdx.x;
    const int64_t tile = blockIdx.x;
    const int64_t base = tile * kSortTile + (int64_t)t * kSortItems;
    uint32_t k[kSortItems];
    unsigned local[kRadix];
#pragma unroll
    for (int d = 0; d < kRadix; d++) local[d] = 0;
#pragma unroll
    for (int i = 0; i < kSortItems; i++) {
        const int64_t idx = base + i;
        k[i] = idx < n ? keys_in[idx] : 0u;
        if (idx < n) {
            const unsigned d = (k[i] >> shift) & (kRadix - 1);
#pragma unroll
            for (int dd = 0; dd < kRadix; dd++) local[dd] += (d == (unsigned)dd);
        }
    }
#pragma unroll
    for (int d = 0; d < kRadix; d++) cnt[d * kSortThreads + t] = local[d];
    __syncthreads();
    // block-wide exclusive scan of cnt in (digit, thread) order: each thread owns 16 consecutive
    // entries of the 4096-entry table
    const int lane = t & 31, wid = t >> 5;
    unsigned run[kRadix];
    unsigned sum = 0;
#pragma unroll
    for (int q = 0; q < kRadix; q++) {
        run[q] = sum;
        sum += cnt[t * kRadix + q];
    }
    unsigned incl = sum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
    }
    if (lane == 31) warp_tot[wid] = incl;
    __syncthreads();
    unsigned wbase = 0;
    for (int w = 0; w < wid; w++) wbase += warp_tot[w];
    const unsigned excl = wbase + incl - sum;
    __syncthreads();
#pragma unroll
    for (int q = 0; q < kRadix; q++) cnt[t * kRadix + q] = excl + run[q];
    __syncthreads();
    // cnt[d][t] is now (keys of the tile with digit < d) + (digit-d keys of threads < t)
#pragma unroll
    for (int d = 0; d < kRadix; d++) local[d] = cnt[d * kSortThreads + t] - cnt[d * kSortThreads];
#pragma unroll
    for (int i = 0; i < kSortItems; i++) {
        const int64_t idx = base + i;
        if (idx < n) {
            const unsigned d = (k[i] >> shift) & (kRadix - 1);
            unsigned r = 0;
#pragma unroll
            for (int dd = 0; dd < kRadix; dd++)
                if (d == (unsigned)dd) { r = local[dd]; local[dd] = r + 1; }
            const int64_t pos = offsets[(int64_t)d * ntiles + tile] + r;
            keys_out[pos] = k[i];
            if (vals_in) vals_out[pos] = vals_in[idx];
        }
    }
}

// exclusive scan, three phases: per-tile sums, a single-block scan of the tile sums, per-tile
// scan plus the tile's offset
template <typename T>
__global__ void __launch_bounds__(256) k_scan_tiles(const T *__restrict__ in, int64_t n, T *__restrict__ sums) {
    __shared__ T s[256];
    const int64_t base = (int64_t)blockIdx.x * kScanTile;
    T acc = 0;
    for (int i = threadIdx.x; i < kScanTile; i += 256) {
        const int64_t k = base + i;
        if (k < n) acc += in[k];
    }
    s[threadIdx.x] = acc;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (threadIdx.x < o) s[threadIdx.x] += s[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) sums[blockIdx.x] = s[0];
}

template <typename T>
__device__ T block_excl_scan_256(T v, T *total, T *s_warp) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    T x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const T y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) s_warp[wid] = x;
    __syncthreads();
    T before = 0, all = 0;
    for (int w = 0; w < 8; w++) {
        if (w < wid) before += s_warp[w];
        all += s_warp[w];
    }
    __syncthreads();
    *total = all;
    return before + x - v;
}

template <typename T>
__global__ void __launch_bounds__(256) k_scan_sums(T *sums, int64_t m, T *grand_total) {
    __shared__ T s_warp[8];
    T carry = 0;
    for (int64_t base = 0; base < m; base += 256) {
        const int64_t i = base + threadIdx.x;
        const T v = i < m ? sums[i] : T(0);
        T tot;
        const T e = block_excl_scan_256(v, &tot, s_warp);
        if (i < m) sums[i] = carry + e;
        carry += tot;
    }
    if (threadIdx.x == 0 && grand_total) *grand_total = carry;
}

template <typename T>
__global__ void __launch_bounds__(256) k_scan_apply(const T *__restrict__ in, T *__restrict__ out, int64_t n,
                                                    const T *__restrict__ sums) {
    __shared__ T s_warp[8];
    const int64_t base = (int64_t)blockIdx.x * kScanTile;
    T carry = sums[blockIdx.x];
    for (int c = 0; c < kScanTile; c += 256) {
        const int64_t i = base + c + threadIdx.x;
        const T v = i < n ? in[i] : T(0);
        T tot;
        const T e = block_excl_scan_256(v, &tot, s_warp);
        if (i < n) out[i] = carry + e;
        carry += tot;
    }
}

static int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }

size_t scan_scratch_bytes(int64_t n) { return sizeof(int64_t) * (size_t)(ceil_div(n, kScanTile) + 1); }

void exclusive_scan_i64(const int64_t *in, int64_t *out, int64_t n, int64_t *total, int64_t *scratch,
                        cudaStream_t s) {
    if (n <= 0) {
        GDE_CUDA(cudaMemsetAsync(total, 0, sizeof(int64_t), s));
        return;
    }
    const int64_t tiles = ceil_div(n, kScanTile);
    k_scan_tiles<int64_t><<<(unsigned)tiles, 256, 0, s>>>(in, n, scratch);
    GDE_CUDA(cudaGetLastError());
    k_scan_sums<int64_t><<<1, 256, 0, s>>>(scratch, tiles, total);
    GDE_CUDA(cudaGetLastError());
    k_scan_apply<int64_t><<<(unsigned)tiles, 256, 0, s>>>(in, out, n, scratch);
    GDE_CUDA(cudaGetLastError());
}

size_t sort_scratch_bytes(int64_t n) {
    const int64_t tiles = ceil_div(n > 0 ? n : 1, kSortTile);
    const int64_t table = (int64_t)kRadix * tiles;
    return sizeof(int64_t) * (size_t)(2 * table + ceil_div(table, kScanTile) + 1);
}

template <typename V>
int radix_sort(uint32_t *keys, V *vals, uint32_t *keys_tmp, V *vals_tmp, int64_t n, int key_bits,
               void *scratch, cudaStream_t s) {
    if (n <= 1) return 0;
    const int64_t tiles = ceil_div(n, kSortTile);
    const int64_t table_n = (int64_t)kRadix * tiles;
    int64_t *table = (int64_t *)scratch;
    int64_t *offs = table + table_n;
    int64_t *sums = offs + table_n;
    int passes = (key_bits + 3) / 4;
    uint32_t *kin = keys, *kout = keys_tmp;
    V *vin = vals, *vout = vals_tmp;
    for (int p = 0; p < passes; p++) {
        const int shift = 4 * p;
        k_sort_hist<<<(unsigned)tiles, kSortThreads, 0, s>>>(kin, n, shift, tiles, table);
        GDE_CUDA(cudaGetLastError());
        const int64_t st = ceil_div(table_n, kScanTile);
        k_scan_tiles<int64_t><<<(unsigned)st, 256, 0, s>>>(table, table_n, sums);
        GDE_CUDA(cudaGetLastError());
        k_scan_sums<int64_t><<<1, 256, 0, s>>>(sums, st, nullptr);
        GDE_CUDA(cudaGetLastError());
        k_scan_apply<int64_t><<<(unsigned)st, 256, 0, s>>>(table, offs, table_n, sums);
        GDE_CUDA(cudaGetLastError());
        k_sort_scatter<V><<<(unsigned)tiles, kSortThreads, 0, s>>>(kin, vin, kout, vout, n, shift, tiles, offs);
        GDE_CUDA(cudaGetLastError());
        uint32_t *tk = kin; kin = kout; kout = tk;
        V *tv = vin; vin = vout; vout = tv;
    }
    // the sorted data is in `kin` / `vin`: 0 = in keys/vals, 1 = in the temporaries
    return (passes & 1) ? 1 : 0;
}

template int radix_sort<double>(uint32_t *, double *, uint32_t *, double *, int64_t, int, void *, cudaStream_t);
template int radix_sort<float>(uint32_t *, float *, uint32_t *, float *, int64_t, int, void *, cudaStream_t);
template int radix_sort<uint32_t>(uint32_t *, uint32_t *, uint32_t *, uint32_t *, int64_t, int, void *, cudaStream_t);

}  // namespace gde
