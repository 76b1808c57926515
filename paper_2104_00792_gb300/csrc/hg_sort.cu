// Sorted buckets (HG_SORTED_BUCKETS): after the build, the keys of every
// bucket of at most SORT_MAX keys are put in ascending order (values move
// with their keys).  A query can then count its key in such a bucket with
// two binary searches (first position >= key, first position > key) instead
// of walking it, which removes the walk that grows with the number of copies
// of a key (the duplicate-key regime of Sec. 5.4).  Offsets and each bucket's
// multiset are unchanged; only the order inside a bucket, which Algorithm 1
// leaves free, is fixed.
//
//  * buckets of 2..TINY_MAX keys: one lane each, a sorting network in registers;
//  * buckets of TINY_MAX+1..SMALL_MAX keys: the warp that found them, a bitonic
//    sort across its lanes;
//  * buckets of SMALL_MAX+1..MID_MAX keys: listed, then one warp each, bitonic
//    sort in its own slice of shared memory;
//  * buckets of MID_MAX+1..SORT_MAX keys: listed, then one CTA each, bitonic
//    sort in shared memory over the next power of two (padding positions
//    marked, and ordered after real keys of the same value);
//  * longer buckets keep their build order and are walked as before.
#include <algorithm>
#include <cstdint>

#include "hg_device.cuh"

namespace hg {
namespace {

constexpr uint32_t TINY_MAX = 8;    // sorted by one thread in registers
constexpr uint32_t SMALL_MAX = 32;  // sorted by one warp across its lanes
constexpr uint32_t MID_MAX = 1024;  // sorted by one warp in shared memory
constexpr int MID_WARPS = 8;
constexpr int SORT_THREADS = 512;

// (key, pad) order: padding after every real key of the same value.
template <typename K>
__device__ __forceinline__ bool after(K a, bool pa, K b, bool pb) {
    return a > b || (a == b && pa && !pb);
}

// Bitonic sort of one (key, pad, value) per lane across the warp, ascending by
// lane: 15 compare-exchange steps with the partner lane (lane ^ j).
template <typename K, bool HV>
__device__ __forceinline__ void warp_bitonic(K& key, bool& pad, uint32_t& val) {
    const unsigned lane = lane_id();
#pragma unroll
    for (unsigned k = 2; k <= 32; k <<= 1) {
#pragma unroll
        for (unsigned j = k >> 1; j > 0; j >>= 1) {
            const K pk = __shfl_xor_sync(FULL_MASK, key, j);
            const bool pp = __shfl_xor_sync(FULL_MASK, pad ? 1u : 0u, j) != 0;
            const uint32_t pv = HV ? __shfl_xor_sync(FULL_MASK, val, j) : 0u;
            const bool ascending = (lane & k) == 0;
            const bool lower = (lane & j) == 0;
            // the lower lane of an ascending pair keeps the smaller element
            const bool take = (lower == ascending) ? after(key, pad, pk, pp) : after(pk, pp, key, pad);
            if (take) {
                key = pk;
                pad = pp;
                if (HV) val = pv;
            }
        }
    }
}

// A warp takes 32 consecutive buckets, one per lane.  Buckets of 2..TINY_MAX
// keys are sorted by their lane in registers (Batcher's odd-even merge
// network for 8 inputs); buckets of TINY_MAX+1..SMALL_MAX keys are then sorted
// one after another by the whole warp (one key per lane, a bitonic sort across
// lanes); longer ones up to sort_max are listed (one atomic per warp) for the
// CTA pass.
template <typename K, bool HV>
__global__ void __launch_bounds__(256) k_sort_small(K* keys, uint32_t* vals, const uint32_t* __restrict__ offs,
                                                    uint64_t B, uint32_t n, uint32_t sort_max, uint32_t* mlist,
                                                    uint32_t* mlist_n, uint32_t mcap, uint32_t* clist,
                                                    uint32_t* clist_n, uint32_t ccap) {
    const unsigned lane = lane_id();
    const uint64_t gw = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint64_t nw = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    for (uint64_t b0 = gw * 32; b0 < B; b0 += nw * 32) {
        const uint64_t b = b0 + lane;
        uint32_t lo = 0, len = 0;
        if (b < B) {
            const uint32_t hi = min(offs[b + 1], n);
            lo = min(offs[b], hi);
            len = hi - lo;
        }
        // lists for the warp pass (up to MID_MAX keys) and the CTA pass, warp-aggregated
        const unsigned mm = __ballot_sync(FULL_MASK, len > SMALL_MAX && len <= MID_MAX && len <= sort_max);
        if (mm) {
            uint32_t base = 0;
            if (lane == 0) base = atomicAdd(mlist_n, (uint32_t)__popc(mm));
            base = __shfl_sync(FULL_MASK, base, 0);
            if ((mm >> lane) & 1u) {
                const uint32_t pos = base + __popc(mm & lanemask_lt());
                if (pos < mcap) mlist[pos] = (uint32_t)b;
            }
        }
        const unsigned cm = __ballot_sync(FULL_MASK, len > MID_MAX && len <= sort_max);
        if (cm) {
            uint32_t base = 0;
            if (lane == 0) base = atomicAdd(clist_n, (uint32_t)__popc(cm));
            base = __shfl_sync(FULL_MASK, base, 0);
            if ((cm >> lane) & 1u) {
                const uint32_t pos = base + __popc(cm & lanemask_lt());
                if (pos < ccap) clist[pos] = (uint32_t)b;
            }
        }
        if (len >= 2 && len <= TINY_MAX) {
            K k[TINY_MAX];
            uint32_t v[TINY_MAX];
            bool p[TINY_MAX];
#pragma unroll
            for (int i = 0; i < (int)TINY_MAX; ++i) {
                p[i] = (uint32_t)i >= len;
                k[i] = p[i] ? ~(K)0 : keys[lo + i];
                v[i] = (HV && !p[i]) ? vals[lo + i] : 0u;
            }
            constexpr int NET[19][2] = {{0, 1}, {2, 3}, {4, 5}, {6, 7}, {0, 2}, {1, 3}, {4, 6}, {5, 7}, {1, 2},
                                        {5, 6}, {0, 4}, {1, 5}, {2, 6}, {3, 7}, {2, 4}, {3, 5}, {1, 2}, {3, 4},
                                        {5, 6}};
#pragma unroll
            for (int c = 0; c < 19; ++c) {
                const int i = NET[c][0], j = NET[c][1];
                if (after(k[i], p[i], k[j], p[j])) {
                    const K tk = k[i]; k[i] = k[j]; k[j] = tk;
                    const bool tp = p[i]; p[i] = p[j]; p[j] = tp;
                    if (HV) { const uint32_t tv = v[i]; v[i] = v[j]; v[j] = tv; }
                }
            }
#pragma unroll
            for (int i = 0; i < (int)TINY_MAX; ++i)
                if ((uint32_t)i < len) {
                    keys[lo + i] = k[i];
                    if (HV) vals[lo + i] = v[i];
                }
        }
        unsigned wm = __ballot_sync(FULL_MASK, len > TINY_MAX && len <= SMALL_MAX);
        while (wm) {
            const int src = __ffs(wm) - 1;
            wm &= wm - 1;
            const uint32_t blo = __shfl_sync(FULL_MASK, lo, src);
            const uint32_t blen = __shfl_sync(FULL_MASK, len, src);
            bool pad = lane >= blen;
            K kk = pad ? ~(K)0 : keys[blo + lane];
            uint32_t vv = (HV && !pad) ? vals[blo + lane] : 0u;
            warp_bitonic<K, HV>(kk, pad, vv);
            __syncwarp();
            if (!pad) {  // lane i holds the i-th smallest; real keys come before the padding
                keys[blo + lane] = kk;
                if (HV) vals[blo + lane] = vv;
            }
            __syncwarp();
        }
    }
}

// Bitonic sort of P (a power of two) (key, pad, value) entries in shared
// memory by `nthreads` threads numbered `tid`; `sync` orders the steps.
template <typename K, bool HV, typename Sync>
__device__ __forceinline__ void smem_bitonic(K* s_k, uint8_t* s_pad, uint32_t* s_v, uint32_t P, uint32_t tid,
                                             uint32_t nthreads, Sync sync) {
    for (uint32_t size = 2; size <= P; size <<= 1) {
        for (uint32_t stride = size >> 1; stride > 0; stride >>= 1) {
            for (uint32_t t = tid; t < P / 2; t += nthreads) {
                const uint32_t i = 2 * t - (t & (stride - 1));  // lower element of the pair
                const uint32_t j = i + stride;
                const bool up = (i & size) == 0;
                const K ki = s_k[i], kj = s_k[j];
                const uint8_t pi = s_pad[i], pj = s_pad[j];
                if (after(ki, pi != 0, kj, pj != 0) == up) {
                    s_k[i] = kj;
                    s_k[j] = ki;
                    s_pad[i] = pj;
                    s_pad[j] = pi;
                    if (HV) {
                        const uint32_t vi = s_v[i];
                        s_v[i] = s_v[j];
                        s_v[j] = vi;
                    }
                }
            }
            sync();
        }
    }
}

// One warp per listed bucket of SMALL_MAX+1..MID_MAX keys, in its own slice of shared memory.
template <typename K, bool HV>
__global__ void __launch_bounds__(MID_WARPS * 32) k_sort_mid(K* keys, uint32_t* vals,
                                                             const uint32_t* __restrict__ offs, uint32_t n,
                                                             const uint32_t* __restrict__ list,
                                                             const uint32_t* __restrict__ list_n, uint32_t cap) {
    extern __shared__ __align__(16) unsigned char smem[];
    const unsigned lane = lane_id();
    const uint32_t w = threadIdx.x >> 5;
    K* s_k = reinterpret_cast<K*>(smem) + (size_t)w * MID_MAX;
    uint32_t* s_v = reinterpret_cast<uint32_t*>(reinterpret_cast<K*>(smem) + MID_WARPS * MID_MAX) +
                    (HV ? (size_t)w * MID_MAX : 0);
    uint8_t* s_pad = reinterpret_cast<uint8_t*>(reinterpret_cast<uint32_t*>(reinterpret_cast<K*>(smem) +
                                                                          MID_WARPS * MID_MAX) +
                                                (HV ? MID_WARPS * MID_MAX : 0)) +
                     (size_t)w * MID_MAX;
    const uint32_t count = min(*list_n, cap);
    const uint64_t gw = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint64_t nw = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    for (uint64_t item = gw; item < count; item += nw) {
        const uint32_t b = list[item];
        const uint32_t hi = min(offs[b + 1], n);
        const uint32_t lo = min(offs[b], hi);
        const uint32_t len = hi - lo;
        uint32_t P = 1;
        while (P < len) P <<= 1;
        if (P > MID_MAX) continue;  // not listed here; kept for safety
        for (uint32_t i = lane; i < P; i += 32) {
            const bool real = i < len;
            s_k[i] = real ? keys[lo + i] : ~(K)0;
            if (HV) s_v[i] = real ? vals[lo + i] : 0u;
            s_pad[i] = real ? 0 : 1;
        }
        __syncwarp();
        smem_bitonic<K, HV>(s_k, s_pad, s_v, P, lane, 32u, [] { __syncwarp(); });
        for (uint32_t i = lane; i < len; i += 32) {
            keys[lo + i] = s_k[i];
            if (HV) vals[lo + i] = s_v[i];
        }
        __syncwarp();
    }
}

// One CTA per listed bucket: bitonic sort of (key, pad, value) in shared memory.
template <typename K, bool HV>
__global__ void __launch_bounds__(SORT_THREADS) k_sort_medium(K* keys, uint32_t* vals,
                                                              const uint32_t* __restrict__ offs, uint32_t n,
                                                              const uint32_t* __restrict__ list,
                                                              const uint32_t* __restrict__ list_n, uint32_t list_cap,
                                                              uint32_t cap_pow2) {
    extern __shared__ __align__(16) unsigned char smem[];
    K* s_k = reinterpret_cast<K*>(smem);
    uint32_t* s_v = reinterpret_cast<uint32_t*>(s_k + cap_pow2);
    uint8_t* s_pad = reinterpret_cast<uint8_t*>(s_v + (HV ? cap_pow2 : 0));
    const uint32_t count = min(*list_n, list_cap);
    for (uint32_t item = blockIdx.x; item < count; item += gridDim.x) {
        const uint32_t b = list[item];
        const uint32_t hi = min(offs[b + 1], n);
        const uint32_t lo = min(offs[b], hi);
        const uint32_t len = hi - lo;
        uint32_t P = 1;
        while (P < len) P <<= 1;
        if (P > cap_pow2) continue;  // not listed by k_sort_small; kept for safety
        for (uint32_t i = threadIdx.x; i < P; i += blockDim.x) {
            const bool real = i < len;
            s_k[i] = real ? keys[lo + i] : ~(K)0;  // padding sorts after every real key
            if (HV) s_v[i] = real ? vals[lo + i] : 0u;
            s_pad[i] = real ? 0 : 1;
        }
        __syncthreads();
        smem_bitonic<K, HV>(s_k, s_pad, s_v, P, threadIdx.x, blockDim.x, [] { __syncthreads(); });
        for (uint32_t i = threadIdx.x; i < len; i += blockDim.x) {
            keys[lo + i] = s_k[i];
            if (HV) vals[lo + i] = s_v[i];
        }
        __syncthreads();
    }
}

template <typename K, bool HV>
cudaError_t sort_impl(Table& t, cudaStream_t s) {
    K* keys = static_cast<K*>(t.keys);
    const uint32_t sort_max = sorted_bucket_max(t.key_bytes);
    const uint32_t mcap = (uint32_t)std::min<uint64_t>(t.B, t.n / (SMALL_MAX + 1) + 1);
    const uint32_t ccap = (uint32_t)std::min<uint64_t>(t.B, t.n / (MID_MAX + 1) + 1);
    void* mem = nullptr;
    cudaError_t e = dev_alloc(&mem, 32 + 4ull * (mcap + ccap), s);
    if (e != cudaSuccess) return e;
    uint32_t* mlist_n = static_cast<uint32_t*>(mem);
    uint32_t* clist_n = mlist_n + 4;
    uint32_t* mlist = mlist_n + 8;
    uint32_t* clist = mlist + mcap;
    e = cudaMemsetAsync(mem, 0, 32, s);
    if (e == cudaSuccess) {
        const uint64_t warps = (t.B + 31) / 32;
        const uint64_t blocks = std::min<uint64_t>((warps + 7) / 8, (uint64_t)num_sms() * 16);
        launch_begin("sort_buckets", s);
        k_sort_small<K, HV><<<(unsigned)std::max<uint64_t>(blocks, 1), 256, 0, s>>>(
            keys, t.values, t.offsets, t.B, (uint32_t)t.n, sort_max, mlist, mlist_n, mcap, clist, clist_n, ccap);
        launch_end("sort_buckets", s);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) {
        const size_t smem = (size_t)MID_WARPS * MID_MAX * (sizeof(K) + (HV ? 4 : 0) + 1);
        auto kern = k_sort_mid<K, HV>;
        e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e == cudaSuccess) {
            launch_begin("sort_buckets", s);
            kern<<<num_sms() * 2, MID_WARPS * 32, smem, s>>>(keys, t.values, t.offsets, (uint32_t)t.n, mlist,
                                                              mlist_n, mcap);
            launch_end("sort_buckets", s);
            e = cudaGetLastError();
        }
    }
    if (e == cudaSuccess) {
        const size_t smem = (size_t)sort_max * (sizeof(K) + (HV ? 4 : 0) + 1);
        auto kern = k_sort_medium<K, HV>;
        e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e == cudaSuccess) {
            launch_begin("sort_buckets", s);
            kern<<<num_sms() * 2, SORT_THREADS, smem, s>>>(keys, t.values, t.offsets, (uint32_t)t.n, clist, clist_n,
                                                           ccap, sort_max);
            launch_end("sort_buckets", s);
            e = cudaGetLastError();
        }
    }
    dev_free(mem, s);
    return e;
}

}  // namespace

uint32_t sorted_bucket_max(uint32_t key_bytes) { return key_bytes == 4 ? 16384u : 8192u; }

cudaError_t sort_buckets(Table& t, cudaStream_t s) {
    if (t.n < 2) return cudaSuccess;
    const bool hv = t.has_values != 0;
    if (t.key_bytes == 4) return hv ? sort_impl<uint32_t, true>(t, s) : sort_impl<uint32_t, false>(t, s);
    return hv ? sort_impl<uint64_t, true>(t, s) : sort_impl<uint64_t, false>(t, s);
}

}  // namespace hg
