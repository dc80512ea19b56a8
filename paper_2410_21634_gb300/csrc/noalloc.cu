// Top-k of a dense float vector without any device allocation: the per-block partial
// lists live in a fixed file-scope device array instead of a cudaMalloc buffer.  For
// callers that cannot allocate device memory (see gde_topk_f32_noalloc in gde.h).
#include <mutex>

#include "common.cuh"

namespace gde {

constexpr int kNoallocParts = 512;  // partial top-64 lists (one per block)
static_assert(GDE_TOPK_NOALLOC_SCRATCH_BYTES == kNoallocParts * 64 * 8, "scratch size");

// one copy per device that loads the library, held until process exit
static __device__ __align__(256) unsigned long long g_topk_scratch[kNoallocParts * 64];

constexpr int kMaxDevices = 64;
static std::mutex g_scratch_mu;
static unsigned long long *g_scratch_addr[kMaxDevices] = {};

// device address of this device's scratch; looked up once per device with it current
static unsigned long long *scratch_for_current_device() {
    int dev = 0;
    GDE_CUDA(cudaGetDevice(&dev));
    GDE_REQUIRE(dev >= 0 && dev < kMaxDevices, GDE_EINVAL, "device ordinal too large");
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    if (!g_scratch_addr[dev]) {
        void *p = nullptr;
        GDE_CUDA(cudaGetSymbolAddress(&p, g_topk_scratch));
        g_scratch_addr[dev] = static_cast<unsigned long long *>(p);
    }
    return g_scratch_addr[dev];
}

}  // namespace gde

using namespace gde;

extern "C" gde_status gde_topk_f32_noalloc(const float *x, int64_t n, int32_t k, int32_t *out_ids,
                                           float *out_vals, void *cuda_stream) {
    try {
        clear_error();
        GDE_REQUIRE(x != nullptr && out_ids != nullptr && out_vals != nullptr, GDE_EINVAL,
                    "gde_topk_f32_noalloc: x, out_ids and out_vals must be device pointers");
        GDE_REQUIRE(k >= 1 && k <= GDE_TOPK_NOALLOC_MAX_K, GDE_EINVAL,
                    "gde_topk_f32_noalloc: k must be in [1, 64] (the scratch holds 64 keys per list)");
        GDE_REQUIRE(n >= 1 && n <= (int64_t)0x7FFFFFFF, GDE_EINVAL,
                    "gde_topk_f32_noalloc: n must be in [1, 2^31 - 1]");
        unsigned long long *scratch = scratch_for_current_device();
        cudaStream_t s = (cudaStream_t)cuda_stream;
        // fewer lists for small inputs; every list the merge reads is written by this call
        int64_t parts = (n + 4095) / 4096;
        if (parts > kNoallocParts) parts = kNoallocParts;
        k_topk_dense_partial<<<(unsigned)parts, kThreads, 0, s>>>(n, x, scratch);
        GDE_CUDA(cudaGetLastError());
        k_topk_dense_final<<<1, kThreads, 0, s>>>(parts, scratch, k, out_ids, out_vals);
        GDE_CUDA(cudaGetLastError());
    } catch (const Fail &f) {
        return f.st;
    } catch (...) {
        set_error("gde_topk_f32_noalloc: unexpected C++ exception");
        return GDE_ECUDA;
    }
    return GDE_OK;
}
