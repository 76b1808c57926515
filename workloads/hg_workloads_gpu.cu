/*
 * Device-side copies of two input recipes of hg_workloads.c, for inputs too
 * large to generate on the host and copy (the serving trace's tables).  The
 * same counter-based definition as the host code: the i-th SplitMix64 output
 * of a stream is mix(state + (i + 1) * GAMMA), so element i of any array is
 * computed independently and equals the host's element i.  Holds none of the
 * hash table's arithmetic.
 */
#include <cstdint>
#include <cuda_runtime.h>

namespace {

constexpr uint64_t GAMMA = 0x9E3779B97F4A7C15ULL;

__device__ __forceinline__ uint64_t sm64_mix(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

__device__ __forceinline__ uint64_t sm64_at(uint64_t state, uint64_t i) { return sm64_mix(state + (i + 1) * GAMMA); }

__global__ void k_uniform_u32(uint64_t state, uint64_t n, uint32_t* out) {
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x)
        out[i] = (uint32_t)(sm64_at(state, i) >> 32);
}

// hgw_probe_mix_u32 over keys = uniform_u32(key_state, n_keys), without
// materialising the keys: a hit's key is regenerated from its index.
__global__ void k_probe_mix_uniform_u32(uint64_t key_state, uint64_t n_keys, uint64_t sel, uint64_t miss,
                                        uint64_t thr, uint64_t q, uint32_t* out) {
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < q; i += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t x = sm64_at(sel, i);
        if (n_keys > 0 && (x >> 32) < thr) {
            const uint64_t idx = ((x & 0xffffffffULL) * n_keys) >> 32;
            out[i] = (uint32_t)(sm64_at(key_state, idx) >> 32);
        } else {
            out[i] = (uint32_t)(sm64_at(miss, i) >> 32);
        }
    }
}

unsigned grid_for(uint64_t n) {
    const uint64_t g = (n + 255) / 256;
    return (unsigned)(g < 4096 ? (g ? g : 1) : 4096);
}

}  // namespace

extern "C" {

int hgw_gpu_uniform_u32(uint64_t state, uint64_t n, uint32_t* out, void* stream) {
    if (n == 0) return 0;
    k_uniform_u32<<<grid_for(n), 256, 0, static_cast<cudaStream_t>(stream)>>>(state, n, out);
    return (int)cudaGetLastError();
}

int hgw_gpu_probe_mix_uniform_u32(uint64_t key_state, uint64_t n_keys, uint64_t sel, uint64_t miss, uint64_t thr,
                                  uint64_t q, uint32_t* out, void* stream) {
    if (q == 0) return 0;
    k_probe_mix_uniform_u32<<<grid_for(q), 256, 0, static_cast<cudaStream_t>(stream)>>>(key_state, n_keys, sel, miss,
                                                                                     thr, q, out);
    return (int)cudaGetLastError();
}

}  // extern "C"
