// Device-side helpers shared by the build and probe kernels.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "hg_internal.h"

namespace hg {

constexpr unsigned FULL_MASK = 0xffffffffu;

// MurmurHash3 32-bit finaliser.
__device__ __forceinline__ uint32_t fmix32(uint32_t h) {
    h ^= h >> 16;
    h *= 0x85ebca6bu;
    h ^= h >> 13;
    h *= 0xc2b2ae35u;
    h ^= h >> 16;
    return h;
}

// Inverse of fmix32 (a bijection of 32-bit words): its steps undone in reverse
// order.  x ^= x >> 16 is its own inverse; x ^= x >> 13 is undone by
// x ^= (x >> 13) ^ (x >> 26); a product with an odd constant by the product
// with the constant's inverse mod 2^32 (0x85ebca6b * 0xa5cb9243 = 1 and
// 0xc2b2ae35 * 0x7ed1b41d = 1 mod 2^32).
__device__ __forceinline__ uint32_t fmix32_inv(uint32_t h) {
    h ^= h >> 16;
    h *= 0x7ed1b41du;
    h ^= (h >> 13) ^ (h >> 26);
    h *= 0xa5cb9243u;
    h ^= h >> 16;
    return h;
}

// MurmurHash3 64-bit finaliser.
__device__ __forceinline__ uint64_t fmix64(uint64_t k) {
    k ^= k >> 33;
    k *= 0xff51afd7ed558ccdull;
    k ^= k >> 33;
    k *= 0xc4ceb9fe1a85ec53ull;
    k ^= k >> 33;
    return k;
}

// bucket(k) = hash(k) mod B (Algorithm 1, first loop).  B <= 2^31, so a bucket fits 32 bits.
__device__ __forceinline__ uint32_t bucket_of(uint32_t k, const Hasher& H) {
    const uint32_t h = fmix32(k ^ (uint32_t)H.seed);
    if (H.mode == MODE_POW2) return h & (uint32_t)H.mask;
    return (uint32_t)__umul64hi(H.magic * (uint64_t)h, H.B);
}
__device__ __forceinline__ uint32_t bucket_of(uint64_t k, const Hasher& H) {
    const uint64_t h = fmix64(k ^ H.seed);
    if (H.mode == MODE_POW2) return (uint32_t)(h & H.mask);
    return (uint32_t)(h % H.B);
}

// The build's and the query grouping's intermediate arrays of 32-bit keys hold
// each key's hash h = fmix32(k ^ seed) instead of the key, so that later passes
// need no hashing; the key comes back as fmix32_inv(h) ^ seed.
__device__ __forceinline__ uint32_t bucket_of_hash(uint32_t h, const Hasher& H) {
    if (H.mode == MODE_POW2) return h & (uint32_t)H.mask;
    return (uint32_t)__umul64hi(H.magic * (uint64_t)h, H.B);
}
__device__ __forceinline__ uint32_t hash_key32(uint32_t k, const Hasher& H) { return fmix32(k ^ (uint32_t)H.seed); }
__device__ __forceinline__ uint32_t unhash_key32(uint32_t h, const Hasher& H) { return fmix32_inv(h) ^ (uint32_t)H.seed; }

__device__ __forceinline__ unsigned lane_id() { return threadIdx.x & 31u; }
__device__ __forceinline__ unsigned lanemask_lt() { return (1u << lane_id()) - 1u; }

// Streaming 16-byte load that does not allocate in L1.
__device__ __forceinline__ uint4 ld_stream16(const void* p) {
    uint4 v;
    asm volatile("ld.global.nc.L1::no_allocate.v4.u32 {%0,%1,%2,%3}, [%4];"
                 : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
                 : "l"(p));
    return v;
}

// Streaming 16-byte load that asks L2 to keep the line (evict_last): for data
// the same kernel reads again shortly.
__device__ __forceinline__ uint4 ld_keep16(const void* p) {
    uint4 v;
    uint64_t pol;
    asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(pol));
    asm volatile("ld.global.nc.L1::no_allocate.L2::cache_hint.v4.u32 {%0,%1,%2,%3}, [%4], %5;"
                 : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
                 : "l"(p), "l"(pol));
    return v;
}

template <typename K>
struct KeyVec {
    static constexpr int N = 16 / sizeof(K);
    K k[N];
};

template <typename K>
__device__ __forceinline__ KeyVec<K> load_keys16(const K* p) {
    uint4 raw = ld_stream16(p);
    KeyVec<K> v;
    static_assert(sizeof(v) == 16, "");
    *reinterpret_cast<uint4*>(&v) = raw;
    return v;
}

// Warp-aggregated atomic increment: every lane in `mask` adds 1 to ctr[b] and
// gets back a distinct slot (old value + its rank among lanes with the same b).
// Lanes with equal b share one atomic, so hot duplicate keys do not serialise.
__device__ __forceinline__ uint32_t agg_inc(uint32_t* ctr, uint32_t b, unsigned mask) {
    const unsigned peers = __match_any_sync(mask, b);
    const int leader = __ffs(peers) - 1;
    uint32_t base = 0;
    if ((int)lane_id() == leader) base = atomicAdd(ctr + b, (uint32_t)__popc(peers));
    base = __shfl_sync(peers, base, leader);
    return base + __popc(peers & lanemask_lt());
}

// Same, when the old value is not needed (compiles to a reduction).
__device__ __forceinline__ void agg_count(uint32_t* ctr, uint32_t b, unsigned mask) {
    const unsigned peers = __match_any_sync(mask, b);
    if ((int)lane_id() == __ffs(peers) - 1) atomicAdd(ctr + b, (uint32_t)__popc(peers));
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULL_MASK, v, o);
    return v;
}

template <typename T>
__device__ __forceinline__ T warp_inclusive_scan(T v) {
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        T t = __shfl_up_sync(FULL_MASK, v, o);
        if ((int)lane_id() >= o) v += t;
    }
    return v;
}

__device__ __forceinline__ uint32_t ld_acquire_u32(const uint32_t* p) {
    uint32_t v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release_u32(uint32_t* p, uint32_t v) {
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// ---- bulk copies (TMA, non-tensor) completing on a shared-memory mbarrier ----
__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}
// Arrive once and add `bytes` to the transaction count the phase waits for.
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ bool mbar_test_parity(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2; selp.u32 %0, 1, 0, p; }"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// Global -> shared bulk copy; dst and src 16-byte aligned, bytes a multiple of 16.
__device__ __forceinline__ void bulk_load(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_addr(dst)),
                 "l"(src), "r"(bytes), "r"(smem_addr(bar))
                 : "memory");
}
// 4-byte asynchronous global -> shared copy (no register staging); completes at cp_async_wait_all.
__device__ __forceinline__ void cp_async4(void* dst, const void* src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(smem_addr(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }
// Orders earlier generic-proxy accesses of shared memory before later async-proxy (bulk copy) ones.
__device__ __forceinline__ void fence_proxy_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// Slot of bucket b in a long-bucket summary map (linear probing from here).
__device__ __forceinline__ uint32_t summary_slot(uint32_t b, uint32_t mask) { return fmix32(b ^ 0x2c1b3c6du) & mask; }

// Lists long bucket b: next index l, bucket[l] = b, map entry (l << 32 | b).
__device__ __forceinline__ void note_long(const LongFinder& F, uint32_t b) {
    const uint32_t l = atomicAdd(F.n_long, 1u);
    if (l >= F.cap) return;  // cannot happen: each long bucket holds more than n / (cap + 1) keys
    F.bucket[l] = b;
    uint32_t h = summary_slot(b, F.map_mask);
    const unsigned long long w = ((unsigned long long)l << 32) | b;
    for (uint32_t probe = 0; probe <= F.map_mask; ++probe) {
        if (atomicCAS(F.map + h, ~0ull, w) == ~0ull) return;
        h = (h + 1) & F.map_mask;
    }
}

// Index of long bucket b's summary, or SUM_OVERFLOW when it has none usable
// (not a long bucket, or more distinct keys than a summary holds).
__device__ __forceinline__ uint32_t summary_index(const LongSummary& S, uint32_t b) {
    uint32_t h = summary_slot(b, S.map_mask);
    for (uint32_t probe = 0; probe <= S.map_mask; ++probe) {
        const unsigned long long w = __ldg(S.map + h);
        if (w == ~0ull) return SUM_OVERFLOW;
        if ((uint32_t)w == b) {
            const uint32_t l = (uint32_t)(w >> 32);
            return __ldg(S.len + l) <= SUM_SLOTS ? l : SUM_OVERFLOW;
        }
        h = (h + 1) & S.map_mask;
    }
    return SUM_OVERFLOW;
}

// Count of `key` in long bucket b from its summary (HG_LONG_SUMMARY): false
// when the bucket has no summary (too many distinct keys, or none was made),
// so that the caller walks it instead.
template <typename K>
__device__ __forceinline__ bool summary_count(const LongSummary& S, uint32_t b, K key, uint32_t& cnt) {
    uint32_t h = summary_slot(b, S.map_mask);
    uint32_t l = SUM_OVERFLOW;
    for (uint32_t probe = 0; probe <= S.map_mask; ++probe) {
        const unsigned long long w = __ldg(S.map + h);
        if (w == ~0ull) return false;
        if ((uint32_t)w == b) {
            l = (uint32_t)(w >> 32);
            break;
        }
        h = (h + 1) & S.map_mask;
    }
    if (l == SUM_OVERFLOW) return false;
    const uint32_t n = __ldg(S.len + l);
    if (n > SUM_SLOTS) return false;
    const K* k = static_cast<const K*>(S.keys) + (size_t)l * SUM_SLOTS;
    uint32_t a = 0, z = n;  // first entry >= key
    while (a < z) {
        const uint32_t m = (a + z) >> 1;
        if (__ldg(k + m) < key) a = m + 1; else z = m;
    }
    cnt = (a < n && __ldg(k + a) == key) ? __ldg(S.cnt + (size_t)l * SUM_SLOTS + a) : 0u;
    return true;
}

}  // namespace hg
