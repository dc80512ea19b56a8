// Random-access calibration of device memory.  The batched scatter's cost is set by how
// many random 32-byte sectors per second the memory system can serve, not by streaming
// bandwidth: a copy moves whole lines in order, a hash-table insert touches one sector at an
// unpredictable address.  This probe measures that rate with the scatter's own access forms
// (two 16-byte L1-bypassing loads of one sector, then an FP32 atomic add into it; a 64-bit
// integer add alone, as into the hub slab; each add with and without its result used), so
// the roofline of the round kernel can be read against both ceilings.
#include "common.cuh"

namespace gde {

// splitmix64 (Steele, Lea and Flood, "Fast splittable pseudorandom number generators",
// OOPSLA 2014): the access index spread over the whole buffer
__device__ __forceinline__ uint64_t probe_mix(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

__global__ void __launch_bounds__(kThreads) k_probe_random(unsigned long long *buf, uint64_t smask, int64_t nops,
                                                           int mode, uint64_t salt, unsigned long long *sink) {
    unsigned long long acc = 0ull;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nops; i += (int64_t)gridDim.x * blockDim.x) {
        unsigned long long *p = buf + 4 * (probe_mix((uint64_t)i + salt) & smask);
        unsigned long long w = 0ull;
        if (mode <= 1) {
            const ulonglong2 lo = __ldcg(reinterpret_cast<const ulonglong2 *>(p));
            const ulonglong2 hi = __ldcg(reinterpret_cast<const ulonglong2 *>(p + 2));
            w = lo.x ^ lo.y ^ hi.x ^ hi.y;
        }
        if (mode == 0) {
            acc += w;
        } else if (mode <= 3) {
            // the word the read picked (mode 1) or the sector's first word (modes 2 and 3)
            float *f = reinterpret_cast<float *>(p + (w & 3ull)) + 1;
            if (mode == 3) atomicAdd(f, 1.0f);
            else acc += (unsigned long long)atomicAdd(f, 1.0f);
        } else if (mode == 4) {
            acc += atomicAdd(p, 1ull);
        } else {
            atomicAdd(p, 1ull);
        }
    }
    // keeps the loads live; the sink is written only if the sum hits this one value
    if (acc == 0x5DEECE66Dull) *sink = acc;
}

}  // namespace gde

using namespace gde;

extern "C" gde_status gde_probe_random_access(void *buf, uint64_t bytes, int64_t nops, int32_t mode, int32_t grid,
                                              int32_t reps, int32_t l2_fetch_bytes, void *cuda_stream,
                                              double *ms_out) {
    bool limit_set = false;
    size_t limit_old = 0;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    gde_status st = GDE_OK;
    try {
        clear_error();
        GDE_REQUIRE(buf != nullptr && ms_out != nullptr, GDE_EINVAL, "gde_probe_random_access: buf and ms_out are required");
        GDE_REQUIRE(((uintptr_t)buf & 255u) == 0, GDE_EINVAL, "gde_probe_random_access: buf must be 256-byte aligned");
        GDE_REQUIRE(bytes >= 64, GDE_EINVAL, "gde_probe_random_access: bytes must be at least 64");
        GDE_REQUIRE(nops >= 1, GDE_EINVAL, "gde_probe_random_access: nops must be >= 1");
        GDE_REQUIRE(mode >= 0 && mode <= 5, GDE_EINVAL, "gde_probe_random_access: mode is 0 .. 5");
        GDE_REQUIRE(grid >= 1 && grid <= 65535, GDE_EINVAL, "gde_probe_random_access: grid in [1, 65535]");
        GDE_REQUIRE(reps >= 1 && reps <= 1000, GDE_EINVAL, "gde_probe_random_access: reps in [1, 1000]");
        GDE_REQUIRE(l2_fetch_bytes == 0 || l2_fetch_bytes == 32 || l2_fetch_bytes == 64 || l2_fetch_bytes == 128,
                    GDE_EINVAL, "gde_probe_random_access: l2_fetch_bytes is 0, 32, 64 or 128");
        // the largest power-of-two number of 32-byte sectors inside the buffer
        uint64_t nsec = 1;
        while ((nsec << 1) <= bytes / 32) nsec <<= 1;
        cudaStream_t s = (cudaStream_t)cuda_stream;
        unsigned long long *sink = reinterpret_cast<unsigned long long *>(buf);  // never written in practice
        if (l2_fetch_bytes) {
            GDE_CUDA(cudaStreamSynchronize(s));
            GDE_CUDA(cudaDeviceGetLimit(&limit_old, cudaLimitMaxL2FetchGranularity));
            GDE_CUDA(cudaDeviceSetLimit(cudaLimitMaxL2FetchGranularity, (size_t)l2_fetch_bytes));
            limit_set = true;
        }
        GDE_CUDA(cudaMemsetAsync(buf, 0, nsec * 32, s));
        GDE_CUDA(cudaEventCreate(&e0));
        GDE_CUDA(cudaEventCreate(&e1));
        unsigned long long *b = reinterpret_cast<unsigned long long *>(buf);
        k_probe_random<<<grid, kThreads, 0, s>>>(b, nsec - 1, nops, mode, 0ull, sink);  // untimed
        GDE_CUDA(cudaGetLastError());
        GDE_CUDA(cudaEventRecord(e0, s));
        for (int r = 1; r <= reps; r++) {
            // a different salt per launch: each touches sectors the previous one did not leave in L2
            k_probe_random<<<grid, kThreads, 0, s>>>(b, nsec - 1, nops, mode, 0x9E3779B97F4A7C15ull * (uint64_t)r, sink);
            GDE_CUDA(cudaGetLastError());
        }
        GDE_CUDA(cudaEventRecord(e1, s));
        GDE_CUDA(cudaEventSynchronize(e1));
        float ms = 0.0f;
        GDE_CUDA(cudaEventElapsedTime(&ms, e0, e1));
        *ms_out = (double)ms / reps;
    } catch (const Fail &f) {
        st = f.st;
    } catch (...) {
        set_error("gde_probe_random_access: unexpected C++ exception");
        st = GDE_ECUDA;
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (limit_set) cudaDeviceSetLimit(cudaLimitMaxL2FetchGranularity, limit_old);
    return st;
}
