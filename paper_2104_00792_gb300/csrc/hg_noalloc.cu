// hg_build_noalloc: the direct build for callers that cannot allocate device
// memory.  Some callers run inside a framework that owns every byte of device
// memory (an inference or serving engine with a fixed memory plan, a plugin
// that may only use buffers its host hands it), or must not allocate once
// they are running (a real-time loop where growing a memory pool would stall
// it).  They can still pass in their own input and output buffers, but not
// the scratch the build's prefix sum needs.  This entry point takes that
// scratch from a fixed array compiled into the library instead.
//
// The scratch is a file-scope __device__ array of 64 KiB (NOALLOC_SCRATCH_BYTES).
// Every GPU that loads the library holds it until the process exits.  Host
// code cannot use the array's name as a device address (on the host it names
// a host-side stand-in), so the first call on each device looks up the real
// address with cudaGetSymbolAddress, with that device current, and caches it
// for the life of the process (so the device's primary context must not be
// reset while the library is loaded).  That first call should therefore happen
// before any stream capture.  Device-side errors are not returned as a status:
// a build whose prefix sum gave up a bounded wait leaves d_offsets[V] != n.
//
// All calls share the one array and it keeps the last call's contents: each
// call clears the parts that must start at zero.  Calls whose work overlaps
// on the GPU (different streams, or different host threads) race on it; order
// them on one stream or serialise them.
#include <cstdio>
#include <mutex>

#include "hg_internal.h"

namespace hg {
namespace {

// Bytes 0..255: the device error word.  From byte 256: the prefix sum's tile
// flags, tile counter and per-tile sums (12 bytes per tile of 2048 or 4096
// offsets, so 4096 tiles cover NOALLOC_MAX_BUCKETS + 1 offsets either way).
constexpr size_t NOALLOC_SCRATCH_BYTES = 64 * 1024;
constexpr size_t NOALLOC_ERR_BYTES = 256;
constexpr uint64_t NOALLOC_MAX_BUCKETS = (1ull << 23) - 1;

static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_SCRATCH_BYTES];

std::mutex g_mu;
void* g_addr[64] = {nullptr};

cudaError_t scratch_address(void** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_addr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_addr[dev] = p;
    }
    *out = g_addr[dev];
    return cudaSuccess;
}

thread_local char g_msg[256];

}  // namespace
}  // namespace hg

using namespace hg;

extern "C" {

hg_status hg_build_noalloc(const hg_config* cfg, const void* d_keys, const void* d_values, uint64_t n,
                           uint32_t* d_offsets, void* d_keys_out, uint32_t* d_values_out, hg_stream_t s) {
    auto bad = [](const char* m) {
        set_error_message(m);
        return HG_ERR_INVALID_ARG;
    };
    if (!cfg) return bad("hg_build_noalloc: cfg is NULL");
    if (cfg->key_bytes != 4 && cfg->key_bytes != 8) return bad("hg_build_noalloc: key_bytes must be 4 or 8");
    if (cfg->value_bytes != 0 && cfg->value_bytes != 4) return bad("hg_build_noalloc: value_bytes must be 0 or 4");
    if (cfg->num_buckets < 1 || cfg->num_buckets > NOALLOC_MAX_BUCKETS) {
        snprintf(g_msg, sizeof(g_msg),
                 "hg_build_noalloc: num_buckets = %llu is outside [1, %llu], the most its fixed scratch supports",
                 (unsigned long long)cfg->num_buckets, (unsigned long long)NOALLOC_MAX_BUCKETS);
        return bad(g_msg);
    }
    if (n >= (1ull << 32)) return bad("hg_build_noalloc: n must be < 2^32");
    if (cfg->flags & ~HG_INDEX_VALUES) return bad("hg_build_noalloc: only HG_INDEX_VALUES is supported");
    const bool want_vals = cfg->value_bytes == 4 || (cfg->flags & HG_INDEX_VALUES);
    if ((cfg->flags & HG_INDEX_VALUES) && cfg->value_bytes) return bad("hg_build_noalloc: HG_INDEX_VALUES needs value_bytes = 0");
    if (!d_offsets) return bad("hg_build_noalloc: d_offsets is NULL");
    if (n > 0 && (!d_keys || !d_keys_out)) return bad("hg_build_noalloc: d_keys and d_keys_out are required");
    if (cfg->value_bytes == 4 && n > 0 && !d_values) return bad("hg_build_noalloc: d_values is NULL");
    if (cfg->value_bytes == 0 && d_values) return bad("hg_build_noalloc: d_values given with value_bytes = 0");
    if (want_vals && n > 0 && !d_values_out) return bad("hg_build_noalloc: d_values_out is required");
    if (!want_vals && d_values_out) return bad("hg_build_noalloc: d_values_out given for a key-only table");
    const uintptr_t kb = cfg->key_bytes;
    if ((reinterpret_cast<uintptr_t>(d_keys) % kb) || (reinterpret_cast<uintptr_t>(d_keys_out) % kb) ||
        (reinterpret_cast<uintptr_t>(d_offsets) % 4) || (reinterpret_cast<uintptr_t>(d_values) % 4) ||
        (reinterpret_cast<uintptr_t>(d_values_out) % 4))
        return bad("hg_build_noalloc: a buffer is not aligned to its element size");

    cudaStream_t st = reinterpret_cast<cudaStream_t>(s);
    void* scratch = nullptr;
    cudaError_t e = scratch_address(&scratch);
    if (e != cudaSuccess) {
        snprintf(g_msg, sizeof(g_msg), "hg_build_noalloc: cudaGetSymbolAddress failed: %s", cudaGetErrorString(e));
        set_error_message(g_msg);
        return HG_ERR_CUDA;
    }
    uint32_t* err = static_cast<uint32_t*>(scratch);
    void* scan_scratch = static_cast<char*>(scratch) + NOALLOC_ERR_BYTES;
    const size_t scan_bytes = NOALLOC_SCRATCH_BYTES - NOALLOC_ERR_BYTES;
    if (scan_u32_scratch_bytes(d_offsets, cfg->num_buckets + 1) > scan_bytes)
        return bad("hg_build_noalloc: internal scratch too small for num_buckets");  // unreachable by the limit
    e = cudaMemsetAsync(err, 0, sizeof(uint32_t), st);
    if (e == cudaSuccess) {
        const Hasher H = make_hasher(cfg->key_bytes, cfg->num_buckets, cfg->seed);
        e = build_direct_into(H, cfg->key_bytes, d_keys, static_cast<const uint32_t*>(d_values),
                              (cfg->flags & HG_INDEX_VALUES) != 0, n, cfg->num_buckets, d_offsets, d_keys_out,
                              d_values_out, scan_scratch, scan_bytes, err, st);
    }
    if (e != cudaSuccess) {
        snprintf(g_msg, sizeof(g_msg), "hg_build_noalloc: %s", cudaGetErrorString(e));
        set_error_message(g_msg);
        return HG_ERR_CUDA;
    }
    return HG_OK;
}

}  // extern "C"
