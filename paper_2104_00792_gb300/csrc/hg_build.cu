// HashGraph build (Algorithm 1) on one GPU.
//
// The CSR offsets double as the counters: offsets[0..B] starts at zero, the
// histogram adds each key to offsets[1 + bucket], an exclusive scan over the
// whole array turns offsets[1 + b] into the start of bucket b, and the
// scatter's atomic cursor for bucket b is offsets[1 + b] itself, so that when
// the scatter ends offsets[1 + b] = start(b) + count(b) = start(b + 1).  No
// separate CounterArray is allocated and the offsets are final when the
// scatter completes.
//
// Hashes are recomputed in each pass instead of materialising H_A (the hash
// costs a handful of integer operations; storing it would cost 8 bytes/key).
#include <cstdint>

#include "hg_device.cuh"

namespace hg {

namespace {

constexpr int BUILD_THREADS = 256;

// Calls f(i, key, mask) for every element i of keys[0, n).  Elements in the
// 16-byte aligned body are loaded 16 bytes at a time; the few elements before
// and after it go to the first warp of the grid.  `mask` is the set of lanes
// of the calling warp that call f together (for warp-aggregated atomics).
template <typename K, typename F>
__device__ __forceinline__ void for_each_key(const K* keys, uint64_t n, uint64_t head, uint64_t nvec, F&& f) {
    constexpr int VEC = KeyVec<K>::N;
    const unsigned lane = lane_id();
    const uint64_t gw = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint64_t nw = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    const K* body = keys + head;
    for (uint64_t b0 = gw * 32; b0 < nvec; b0 += nw * 32) {
        const uint64_t v = b0 + lane;
        const bool ok = v < nvec;
        const unsigned m = __ballot_sync(FULL_MASK, ok);
        if (ok) {
            const KeyVec<K> kv = load_keys16(body + v * VEC);
#pragma unroll
            for (int j = 0; j < VEC; ++j) f(head + v * VEC + j, kv.k[j], m);
        }
    }
    if (gw == 0) {
        const uint64_t tail0 = head + nvec * VEC;
        const uint64_t nrem = head + (n - tail0);  // < 2 * VEC <= 8
        const bool ok = lane < nrem;
        const unsigned m = __ballot_sync(FULL_MASK, ok);
        if (ok) {
            const uint64_t i = lane < head ? lane : tail0 + (lane - head);
            f(i, keys[i], m);
        }
    }
}

// Algorithm 1, loops 2-3: CounterArray[hash(A[i]) mod V] += 1, into offsets[1 + b].
template <typename K>
__global__ void __launch_bounds__(BUILD_THREADS)
k_hist(const K* keys, uint64_t n, uint64_t head, uint64_t nvec, Hasher H, uint32_t* cnt) {
    for_each_key(keys, n, head, nvec, [&](uint64_t, K k, unsigned m) { agg_count(cnt, bucket_of(k, H), m); });
}

// Algorithm 1, loop 5: pos = AtomicAdd(cursor[b], 1); keys[pos] = A[i] (cursor = offsets + 1,
// already holding each bucket's start).  VM: 0 keys only, 1 caller values, 2 input index as value.
// A position outside [0, n) can only come from inconsistent offsets (a scan
// that gave up a wait); it is skipped and flagged instead of written.
template <typename K, int VM>
__global__ void __launch_bounds__(BUILD_THREADS)
k_scatter(const K* keys, const uint32_t* vals, uint64_t n, uint64_t head, uint64_t nvec, Hasher H, uint32_t* cur,
          K* keys_out, uint32_t* vals_out, uint32_t* err) {
    for_each_key(keys, n, head, nvec, [&](uint64_t i, K k, unsigned m) {
        const uint32_t pos = agg_inc(cur, bucket_of(k, H), m);
        if (pos >= n) {
            atomicOr(err, DEVERR_BOUNDS);
            return;
        }
        keys_out[pos] = k;
        if (VM == 1) vals_out[pos] = __ldg(vals + i);
        if (VM == 2) vals_out[pos] = (uint32_t)i;
    });
}

template <typename Kern>
unsigned stream_grid(Kern kern, uint64_t work_items) {
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, BUILD_THREADS, 0) != cudaSuccess || per_sm < 1)
        per_sm = 1;
    uint64_t g = (uint64_t)num_sms() * per_sm;
    const uint64_t need = (work_items + BUILD_THREADS - 1) / BUILD_THREADS;
    if (need < g) g = need;
    return (unsigned)(g < 1 ? 1 : g);
}

template <typename K>
cudaError_t build_plain(Table& t, const K* keys, const uint32_t* vals, cudaStream_t s) {
    constexpr int VEC = KeyVec<K>::N;
    const uint64_t n = t.n;
    const uintptr_t a = reinterpret_cast<uintptr_t>(keys);
    uint64_t head = ((16 - (a & 15)) & 15) / sizeof(K);
    if (head > n) head = n;
    const uint64_t nvec = (n - head) / VEC;
    uint32_t* cnt = t.offsets + 1;

    {
        auto kern = k_hist<K>;
        const unsigned g = stream_grid(kern, nvec + 1);
        launch_begin("hist", s);
        kern<<<g, BUILD_THREADS, 0, s>>>(keys, n, head, nvec, t.H, cnt);
        launch_end("hist", s);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    cudaError_t e = scan_exclusive_u32(t.offsets, t.B + 1, t.err, s);
    if (e != cudaSuccess) return e;
    K* kout = static_cast<K*>(t.keys);
    auto launch = [&](auto kern) {
        const unsigned g = stream_grid(kern, nvec + 1);
        launch_begin("scatter", s);
        kern<<<g, BUILD_THREADS, 0, s>>>(keys, vals, n, head, nvec, t.H, cnt, kout, t.values, t.err);
        launch_end("scatter", s);
        return cudaGetLastError();
    };
    if (vals) return launch(k_scatter<K, 1>);
    if (t.has_values) return launch(k_scatter<K, 2>);
    return launch(k_scatter<K, 0>);
}

// The direct build writing into caller-provided arrays, with the scan's scratch
// supplied by the caller.
template <typename K>
cudaError_t build_direct_into_impl(const Hasher& H, const K* keys, const uint32_t* vals, bool index_values,
                                   uint64_t n, uint64_t B, uint32_t* offsets, K* kout, uint32_t* vout,
                                   void* scan_scratch, size_t scan_scratch_bytes, uint32_t* err, cudaStream_t s) {
    constexpr int VEC = KeyVec<K>::N;
    const uintptr_t a = reinterpret_cast<uintptr_t>(keys);
    uint64_t head = ((16 - (a & 15)) & 15) / sizeof(K);
    if (head > n) head = n;
    const uint64_t nvec = (n - head) / VEC;
    uint32_t* cnt = offsets + 1;
    {
        auto kern = k_hist<K>;
        const unsigned g = stream_grid(kern, nvec + 1);
        launch_begin("hist", s);
        kern<<<g, BUILD_THREADS, 0, s>>>(keys, n, head, nvec, H, cnt);
        launch_end("hist", s);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    cudaError_t e = scan_exclusive_u32_into(offsets, B + 1, scan_scratch, scan_scratch_bytes, err, s);
    if (e != cudaSuccess) return e;
    auto launch = [&](auto kern) {
        const unsigned g = stream_grid(kern, nvec + 1);
        launch_begin("scatter", s);
        kern<<<g, BUILD_THREADS, 0, s>>>(keys, vals, n, head, nvec, H, cnt, kout, vout, err);
        launch_end("scatter", s);
        return cudaGetLastError();
    };
    if (vals && vout) return launch(k_scatter<K, 1>);
    if (index_values && vout) return launch(k_scatter<K, 2>);
    return launch(k_scatter<K, 0>);
}

}  // namespace

cudaError_t build_direct_into(const Hasher& H, uint32_t key_bytes, const void* keys, const uint32_t* vals,
                              bool index_values, uint64_t n, uint64_t B, uint32_t* offsets, void* keys_out,
                              uint32_t* vals_out, void* scan_scratch, size_t scan_scratch_bytes, uint32_t* err,
                              cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(offsets, 0, (B + 1) * sizeof(uint32_t), s);
    if (e != cudaSuccess || n == 0) return e;
    if (key_bytes == 4)
        return build_direct_into_impl<uint32_t>(H, static_cast<const uint32_t*>(keys), vals, index_values, n, B,
                                                offsets, static_cast<uint32_t*>(keys_out), vals_out, scan_scratch,
                                                scan_scratch_bytes, err, s);
    return build_direct_into_impl<uint64_t>(H, static_cast<const uint64_t*>(keys), vals, index_values, n, B, offsets,
                                            static_cast<uint64_t*>(keys_out), vals_out, scan_scratch,
                                            scan_scratch_bytes, err, s);
}

// The partitioned build (Sec. 3.2 binning) pays off once the offsets array no
// longer fits in L2; forced either way by HG_PARTITION_BUILD / HG_PLAIN_BUILD.
static bool use_partition(const Table& t) {
    if (t.flags & HG_PLAIN_BUILD) return false;
    if (!partition_supported(t.B)) return false;
    if (t.flags & HG_PARTITION_BUILD) return true;
    return t.B >= (1ull << 21);
}

cudaError_t build_table(Table& t, const void* d_keys, const void* d_values, cudaStream_t s) {
    if (t.n > 0 && use_partition(t)) return build_partitioned(t, d_keys, d_values, s);
    cudaError_t e = cudaMemsetAsync(t.offsets, 0, (t.B + 1) * sizeof(uint32_t), s);
    if (e != cudaSuccess || t.n == 0) return e;
    const uint32_t* vals = static_cast<const uint32_t*>(d_values);
    if (t.key_bytes == 4) return build_plain<uint32_t>(t, static_cast<const uint32_t*>(d_keys), vals, s);
    return build_plain<uint64_t>(t, static_cast<const uint64_t*>(d_keys), vals, s);
}

}  // namespace hg
