// Exclusive prefix sum in place, single pass with decoupled look-back
// (Merrill and Garland, "Single-pass Parallel Prefix Scan with Decoupled
// Look-back", NVIDIA TR 2016).  Used for Algorithm 1's
// offset = PrefixSum(CounterArray) and for the gather's output offsets.
//
// Tiles take their index from an atomic counter in launch order, so a tile
// only ever waits on tiles that are already running; every wait is bounded
// and, if it runs out, the tile records DEVERR_TIMEOUT and carries on with a
// zero contribution instead of spinning forever.
#include <cstdint>

#include "hg_device.cuh"

namespace hg {

namespace {

constexpr int SCAN_WARPS = 8;
constexpr int SCAN_THREADS = SCAN_WARPS * 32;
constexpr uint32_t FLAG_AGG = 1, FLAG_PREFIX = 2;
constexpr uint32_t SPIN_LIMIT = 1u << 20;  // polls per lane, each ~0.5-1 us: about a second at most

template <typename T>
__device__ __forceinline__ T warp_reduce_add(T v) {
    return warp_sum(v);
}

// Sum of the inclusive prefixes/aggregates of all tiles before `tile`.
// Called by all 32 lanes of one warp.
template <typename T>
__device__ T lookback(uint64_t tile, const uint32_t* flags, const T* aggs, const T* pres, uint32_t* err) {
    T excl = 0;
    int64_t pred = (int64_t)tile - 1;
    const int lane = (int)lane_id();
    uint32_t polls = 0;
    while (true) {
        const int64_t t = pred - lane;  // lane 0 looks at the nearest predecessor
        uint32_t f = FLAG_PREFIX;
        if (t >= 0) {
            f = ld_acquire_u32(flags + t);
            while (f == 0 && polls < SPIN_LIMIT) {
                ++polls;
                __nanosleep(64);
                f = ld_acquire_u32(flags + t);
            }
        }
        const bool gave_up = (f == 0);
        if (__any_sync(FULL_MASK, gave_up) && lane == 0) atomicOr(err, DEVERR_TIMEOUT);
        T v = 0;
        if (t >= 0 && !gave_up) v = (f == FLAG_PREFIX) ? pres[t] : aggs[t];
        const unsigned stop_mask = __ballot_sync(FULL_MASK, f == FLAG_PREFIX || gave_up);
        const int stop = stop_mask ? __ffs(stop_mask) - 1 : 31;
        excl += warp_reduce_add<T>(lane <= stop ? v : (T)0);
        if (stop_mask) break;
        pred -= 32;
    }
    return excl;
}

template <typename T>
__device__ __forceinline__ void publish(uint32_t* flags, T* slot, uint64_t tile, T v, uint32_t flag) {
    slot[tile] = v;
    st_release_u32(flags + tile, flag);
}

// V: elements per 16-byte vector (1 when the array is not 16-byte aligned).
template <typename T, int V, int ROWS>
__global__ void __launch_bounds__(SCAN_THREADS)
k_scan_exclusive(T* data, uint64_t n, uint32_t* flags, T* aggs, T* pres, uint32_t* tile_ctr, uint32_t* err) {
    constexpr int ROW = 32 * V;
    constexpr int WARP_ITEMS = ROWS * ROW;
    constexpr uint64_t TILE = (uint64_t)SCAN_WARPS * WARP_ITEMS;
    __shared__ uint32_t s_tile;
    __shared__ T s_warp[SCAN_WARPS];
    __shared__ T s_excl;

    if (threadIdx.x == 0) s_tile = atomicAdd(tile_ctr, 1u);
    __syncthreads();
    const uint64_t tile = s_tile;
    const int w = threadIdx.x >> 5;
    const int lane = (int)lane_id();
    const uint64_t wbase = tile * TILE + (uint64_t)w * WARP_ITEMS;

    T x[ROWS][V];
#pragma unroll
    for (int r = 0; r < ROWS; ++r) {
        const uint64_t idx = wbase + (uint64_t)r * ROW + (uint64_t)lane * V;
        if (V > 1 && idx + V <= n) {
            uint4 raw = *reinterpret_cast<const uint4*>(data + idx);
            const T* e = reinterpret_cast<const T*>(&raw);
#pragma unroll
            for (int v = 0; v < V; ++v) x[r][v] = e[v];
        } else {
#pragma unroll
            for (int v = 0; v < V; ++v) x[r][v] = (idx + v < n) ? data[idx + v] : (T)0;
        }
    }

    T lane_excl[ROWS], row_prefix[ROWS];
    T warp_total = 0;
#pragma unroll
    for (int r = 0; r < ROWS; ++r) {
        T s = 0;
#pragma unroll
        for (int v = 0; v < V; ++v) s += x[r][v];
        const T incl = warp_inclusive_scan(s);
        lane_excl[r] = incl - s;
        row_prefix[r] = warp_total;
        warp_total += __shfl_sync(FULL_MASK, incl, 31);
    }
    if (lane == 0) s_warp[w] = warp_total;
    __syncthreads();

    if (w == 0) {
        const T mine = lane < SCAN_WARPS ? s_warp[lane] : (T)0;
        const T incl = warp_inclusive_scan(mine);
        const T tile_agg = __shfl_sync(FULL_MASK, incl, 31);
        if (lane < SCAN_WARPS) s_warp[lane] = incl - mine;
        T excl = 0;
        if (tile == 0) {
            if (lane == 0) publish(flags, pres, tile, tile_agg, FLAG_PREFIX);
        } else {
            if (lane == 0) publish(flags, aggs, tile, tile_agg, FLAG_AGG);
            excl = lookback<T>(tile, flags, aggs, pres, err);
            if (lane == 0) publish(flags, pres, tile, excl + tile_agg, FLAG_PREFIX);
        }
        if (lane == 0) s_excl = excl;
    }
    __syncthreads();

    const T prefix = s_excl + s_warp[w];
#pragma unroll
    for (int r = 0; r < ROWS; ++r) {
        T run = prefix + row_prefix[r] + lane_excl[r];
        T out[V];
#pragma unroll
        for (int v = 0; v < V; ++v) {
            out[v] = run;
            run += x[r][v];
        }
        const uint64_t idx = wbase + (uint64_t)r * ROW + (uint64_t)lane * V;
        if (V > 1 && idx + V <= n) {
            *reinterpret_cast<uint4*>(data + idx) = *reinterpret_cast<const uint4*>(out);
        } else {
#pragma unroll
            for (int v = 0; v < V; ++v)
                if (idx + v < n) data[idx + v] = out[v];
        }
    }
}

template <typename T, int V, int ROWS>
cudaError_t launch_scan(T* data, uint64_t n, uint32_t* err, cudaStream_t s) {
    constexpr uint64_t TILE = (uint64_t)SCAN_WARPS * ROWS * 32 * V;
    const uint64_t ntiles = (n + TILE - 1) / TILE;
    if (ntiles > 0x7fffffffull) return cudaErrorInvalidValue;
    // scratch: flags[ntiles] u32 | tile counter u32 | pad | aggs[ntiles] T | pres[ntiles] T
    const size_t flag_bytes = ((ntiles + 1) * sizeof(uint32_t) + 15) & ~size_t(15);
    const size_t bytes = flag_bytes + 2 * ntiles * sizeof(T);
    void* scratch = nullptr;
    cudaError_t e = dev_alloc(&scratch, bytes, s);
    if (e != cudaSuccess) return e;
    uint32_t* flags = static_cast<uint32_t*>(scratch);
    uint32_t* ctr = flags + ntiles;
    T* aggs = reinterpret_cast<T*>(static_cast<char*>(scratch) + flag_bytes);
    T* pres = aggs + ntiles;
    e = cudaMemsetAsync(flags, 0, (ntiles + 1) * sizeof(uint32_t), s);
    if (e == cudaSuccess) {
        launch_begin("scan", s);
        k_scan_exclusive<T, V, ROWS><<<(unsigned)ntiles, SCAN_THREADS, 0, s>>>(data, n, flags, aggs, pres, ctr, err);
        launch_end("scan", s);
        e = cudaGetLastError();
    }
    dev_free(scratch, s);
    return e;
}

// Same kernel, scratch supplied by the caller (no allocation).  The flags and
// the tile counter are cleared here; the aggregate/prefix slots need no clearing.
template <typename T, int V, int ROWS>
cudaError_t launch_scan_into(T* data, uint64_t n, void* scratch, size_t scratch_bytes, uint32_t* err,
                             cudaStream_t s) {
    constexpr uint64_t TILE = (uint64_t)SCAN_WARPS * ROWS * 32 * V;
    const uint64_t ntiles = (n + TILE - 1) / TILE;
    const size_t flag_bytes = ((ntiles + 1) * sizeof(uint32_t) + 15) & ~size_t(15);
    if (flag_bytes + 2 * ntiles * sizeof(T) > scratch_bytes || (reinterpret_cast<uintptr_t>(scratch) & 15))
        return cudaErrorInvalidValue;
    uint32_t* flags = static_cast<uint32_t*>(scratch);
    uint32_t* ctr = flags + ntiles;
    T* aggs = reinterpret_cast<T*>(static_cast<char*>(scratch) + flag_bytes);
    T* pres = aggs + ntiles;
    cudaError_t e = cudaMemsetAsync(flags, 0, (ntiles + 1) * sizeof(uint32_t), s);
    if (e != cudaSuccess) return e;
    launch_begin("scan", s);
    k_scan_exclusive<T, V, ROWS><<<(unsigned)ntiles, SCAN_THREADS, 0, s>>>(data, n, flags, aggs, pres, ctr, err);
    launch_end("scan", s);
    return cudaGetLastError();
}

}  // namespace

// Self-test of the bounded look-back wait: one CTA of the scan takes tile 1 of
// a two-tile array while tile 0 never runs, so its wait for tile 0's flag (a
// flag nothing sets) runs out after SPIN_LIMIT polls, about a second, and the
// CTA records DEVERR_TIMEOUT in *err and finishes.
cudaError_t scan_wait_limit_selftest(uint32_t* err, cudaStream_t s) {
    constexpr uint64_t TILE = (uint64_t)SCAN_WARPS * 4 * 32 * 4;
    const uint64_t n = 2 * TILE;
    const size_t flag_bytes = (3 * sizeof(uint32_t) + 15) & ~size_t(15);
    const size_t bytes = 4 * n + flag_bytes + 2 * 2 * sizeof(uint32_t);
    void* mem = nullptr;
    cudaError_t e = dev_alloc(&mem, bytes, s);
    if (e != cudaSuccess) return e;
    uint32_t* data = static_cast<uint32_t*>(mem);
    uint32_t* flags = data + n;
    uint32_t* ctr = flags + 2;
    uint32_t* aggs = reinterpret_cast<uint32_t*>(reinterpret_cast<char*>(flags) + flag_bytes);
    uint32_t* pres = aggs + 2;
    static const uint32_t one = 1;
    e = cudaMemsetAsync(mem, 0, bytes, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(ctr, &one, sizeof(one), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) {
        launch_begin("scan", s);
        k_scan_exclusive<uint32_t, 4, 4><<<1, SCAN_THREADS, 0, s>>>(data, n, flags, aggs, pres, ctr, err);
        launch_end("scan", s);
        e = cudaGetLastError();
    }
    dev_free(mem, s);
    return e;
}

size_t scan_u32_scratch_bytes(const uint32_t* data, uint64_t n) {
    const uint64_t tile = (reinterpret_cast<uintptr_t>(data) & 15) == 0 ? (uint64_t)SCAN_WARPS * 4 * 32 * 4
                                                                          : (uint64_t)SCAN_WARPS * 8 * 32 * 1;
    const uint64_t ntiles = (n + tile - 1) / tile;
    return (((ntiles + 1) * sizeof(uint32_t) + 15) & ~size_t(15)) + 2 * ntiles * sizeof(uint32_t);
}

cudaError_t scan_exclusive_u32_into(uint32_t* data, uint64_t n, void* scratch, size_t scratch_bytes, uint32_t* err,
                                    cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    if ((reinterpret_cast<uintptr_t>(data) & 15) == 0)
        return launch_scan_into<uint32_t, 4, 4>(data, n, scratch, scratch_bytes, err, s);
    return launch_scan_into<uint32_t, 1, 8>(data, n, scratch, scratch_bytes, err, s);
}

cudaError_t scan_exclusive_u32(uint32_t* data, uint64_t n, uint32_t* err, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    if ((reinterpret_cast<uintptr_t>(data) & 15) == 0) return launch_scan<uint32_t, 4, 4>(data, n, err, s);
    return launch_scan<uint32_t, 1, 8>(data, n, err, s);
}

cudaError_t scan_exclusive_u64(uint64_t* data, uint64_t n, uint32_t* err, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    if ((reinterpret_cast<uintptr_t>(data) & 15) == 0) return launch_scan<uint64_t, 2, 4>(data, n, err, s);
    return launch_scan<uint64_t, 1, 8>(data, n, err, s);
}

}  // namespace hg
