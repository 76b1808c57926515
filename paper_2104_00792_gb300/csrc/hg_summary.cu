// Long-bucket summaries (HG_LONG_SUMMARY).
//
// Counting a query walks its whole bucket, so a bucket holding millions of
// copies of one key costs millions of compares per query of that key: the
// quadratic duplicate-key regime (Sec. 5.4).  After the build, every bucket of
// more than SUM_MIN_LEN keys is condensed here into its distinct keys with
// their multiplicities, ascending by key; a count query on such a bucket then
// takes a binary search of at most SUM_SLOTS entries instead of the walk.  The
// counts are the ones the walk finds (each entry is the number of copies of
// its key in the bucket).  A bucket with more than SUM_SLOTS distinct keys
// gets the length SUM_OVERFLOW and is walked as before.
//
// Steps, on the build's stream:
//   (listing)     every long bucket takes an index l and enters the bucket -> l
//                 hash map: the partitioned build does it where it writes the
//                 offsets (k_bin_local, k_huge_scan); after the direct build,
//                 k_sum_find makes one pass over the offsets (16-byte loads);
//   k_sum_plan    one CTA: SUM_CHUNK-key chunks of each long bucket, one work
//                 item descriptor (key range, l) per chunk;
//   k_sum_count   persistent: one chunk per CTA work item.  Each thread counts
//                 runs of equal keys in registers and adds each run into a
//                 shared-memory table; the table is then added into the
//                 bucket's global open-addressing table (a few atomics per
//                 chunk, since a long bucket holds few distinct keys);
//   k_sum_finish  one warp per long bucket: compact and sort its table.
// All-ones is the empty slot marker of both tables; the key with all bits set
// is counted on the side and placed last (it is the largest key).
#include <cstdint>

#include "hg_device.cuh"

namespace hg {

namespace {

constexpr uint32_t SUM_CHUNK = 1u << 16;  // keys per k_sum_count work item
constexpr uint32_t SUM_LOCAL = 256;       // slots of a chunk's shared-memory table
constexpr int SUM_THREADS = 512;
constexpr int SUM_UNROLL = 4;             // 16-byte loads in flight per thread

// Scratch and result arrays of one table's summaries (one allocation).
struct SumBuild {
    LongFinder F;            // n_long [1], bucket [cap], map
    uint32_t* total_chunks;  // [1]
    uint4* item;             // [max_items]: (first key, end key, l, 0) of each chunk
    uint32_t max_items;
    uint32_t* spec;          // [cap]: copies of the all-ones key
    uint32_t* len;           // [cap]: 0 while counting, SUM_OVERFLOW on overflow, then the entry count
    void* keys;              // [cap * SUM_SLOTS]
    uint32_t* cnt;           // [cap * SUM_SLOTS]
};

template <typename K>
__device__ __forceinline__ uint32_t key_slot(K k, uint32_t mask) {
    if (sizeof(K) == 4) return fmix32((uint32_t)k ^ 0x7f4a7c15u) & mask;
    return (uint32_t)fmix64((uint64_t)k ^ 0x7f4a7c159e3779b9ull) & mask;
}

__device__ __forceinline__ uint32_t cas_key(uint32_t* p, uint32_t cmp, uint32_t v) { return atomicCAS(p, cmp, v); }
__device__ __forceinline__ uint64_t cas_key(uint64_t* p, uint64_t cmp, uint64_t v) {
    return (uint64_t)atomicCAS(reinterpret_cast<unsigned long long*>(p), (unsigned long long)cmp,
                               (unsigned long long)v);
}

// Long buckets from the offsets: thread v reads offsets [4v, 4v + 4) with one
// 16-byte load and takes the fifth from the next lane.
__global__ void __launch_bounds__(256) k_sum_find(const uint32_t* __restrict__ offs, uint64_t B, uint32_t n_keys,
                                                  LongFinder F) {
    const unsigned lane = lane_id();
    const uint64_t nvec = (B + 3) / 4;
    const uint64_t gw = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint64_t nw = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    for (uint64_t base = gw * 32; base < nvec; base += nw * 32) {
        const uint64_t v = base + lane;
        const bool ok = v < nvec;
        uint4 o = make_uint4(0, 0, 0, 0);
        if (ok) o = __ldg(reinterpret_cast<const uint4*>(offs) + v);
        uint32_t next = __shfl_down_sync(FULL_MASK, o.x, 1);
        // the fifth offset from memory where the next lane holds no vector
        if ((lane == 31 || v + 1 >= nvec) && ok && 4 * v + 4 <= B) next = __ldg(offs + 4 * v + 4);
        if (!ok) continue;
        const uint32_t e[5] = {o.x, o.y, o.z, o.w, next};
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const uint64_t b = 4 * v + u;
            if (b >= B) break;
            const uint32_t hi = min(e[u + 1], n_keys);
            const uint32_t lo = min(e[u], hi);
            if (hi - lo > SUM_MIN_LEN) note_long(F, (uint32_t)b);
        }
    }
}

// One CTA: the chunks of every long bucket l (chunks before it: the running
// prefix of ceil(len / SUM_CHUNK)), each written as a work item descriptor.
__global__ void __launch_bounds__(1024) k_sum_plan(const uint32_t* __restrict__ offs, uint32_t n_keys, SumBuild S) {
    __shared__ uint32_t s_warp[32];
    __shared__ uint32_t s_tot;
    const unsigned lane = lane_id();
    const int w = threadIdx.x >> 5;
    const uint32_t L = min(*S.F.n_long, S.F.cap);
    uint32_t running = 0;
    for (uint32_t base = 0; base < L; base += blockDim.x) {
        const uint32_t l = base + threadIdx.x;
        uint32_t ch = 0, lo = 0, hi = 0;
        if (l < L) {
            const uint32_t b = S.F.bucket[l];
            hi = min(offs[b + 1], n_keys);
            lo = min(offs[b], hi);
            ch = (hi - lo + SUM_CHUNK - 1) / SUM_CHUNK;
        }
        const uint32_t incl = warp_inclusive_scan(ch);
        if (lane == 31) s_warp[w] = incl;
        __syncthreads();
        if (w == 0) {
            const uint32_t wv = lane < (blockDim.x >> 5) ? s_warp[lane] : 0u;
            const uint32_t wi = warp_inclusive_scan(wv);
            if (lane < (blockDim.x >> 5)) s_warp[lane] = wi - wv;
            if (lane == 31) s_tot = wi;
        }
        __syncthreads();
        const uint32_t first = running + s_warp[w] + incl - ch;
        for (uint32_t c = 0; c < ch; ++c) {
            const uint32_t it = first + c;
            const uint32_t p0 = lo + c * SUM_CHUNK;
            if (it < S.max_items) S.item[it] = make_uint4(p0, min(hi, p0 + SUM_CHUNK), l, 0u);
        }
        running += s_tot;
        __syncthreads();
    }
    if (threadIdx.x == 0) *S.total_chunks = min(running, S.max_items);
}

// Chunks of the long buckets: distinct keys and their copies, added into the
// bucket's global table.
template <typename K>
__global__ void __launch_bounds__(SUM_THREADS) k_sum_count(const K* __restrict__ keys,
                                                           const uint32_t* __restrict__ offs, uint32_t n_keys,
                                                           SumBuild S) {
    constexpr int KVEC = 16 / sizeof(K);
    constexpr K EMPTY = ~(K)0;
    __shared__ K s_key[SUM_LOCAL];
    __shared__ uint32_t s_cnt[SUM_LOCAL];
    __shared__ uint32_t s_spec, s_over;
    const uint32_t total = *S.total_chunks;
    for (uint32_t item = blockIdx.x; item < total; item += gridDim.x) {
        const uint4 d = S.item[item];  // same address in every thread: one broadcast load
        const uint32_t p0 = min(d.x, n_keys), p1 = min(d.y, n_keys), l = d.z;
        if (threadIdx.x == 0) {
            s_spec = 0;
            s_over = 0;
        }
        for (uint32_t t = threadIdx.x; t < SUM_LOCAL; t += blockDim.x) {
            s_key[t] = EMPTY;
            s_cnt[t] = 0;
        }
        __syncthreads();
        // add `c` copies of `k` to the chunk's table
        auto flush = [&](K k, uint32_t c) {
            if (c == 0) return;
            if (k == EMPTY) {
                atomicAdd(&s_spec, c);
                return;
            }
            if (*static_cast<volatile uint32_t*>(&s_over)) return;
            uint32_t h = key_slot(k, SUM_LOCAL - 1);
            for (uint32_t probe = 0; probe < SUM_LOCAL; ++probe) {
                K cur = *static_cast<volatile K*>(&s_key[h]);
                if (cur == EMPTY) cur = cas_key(&s_key[h], EMPTY, k);
                if (cur == EMPTY || cur == k) {
                    atomicAdd(&s_cnt[h], c);
                    return;
                }
                h = (h + 1) & (SUM_LOCAL - 1);
            }
            s_over = 1;
        };
        // two keys counted in registers (a bucket often interleaves two values);
        // a third key flushes the older one
        K r0 = 0, r1 = 0;
        uint32_t c0 = 0, c1 = 0;
        const uint32_t a0 = p0 & ~(uint32_t)(KVEC - 1);
        const uint32_t stride = blockDim.x * KVEC;
        for (uint32_t v = a0 + threadIdx.x * KVEC; v < p1; v += SUM_UNROLL * stride) {
            if (*static_cast<volatile uint32_t*>(&s_over)) break;
            KeyVec<K> kv[SUM_UNROLL];  // SUM_UNROLL loads in flight per thread
#pragma unroll
            for (int r = 0; r < SUM_UNROLL; ++r)
                if (v + r * stride < p1) kv[r] = load_keys16(keys + v + r * stride);
#pragma unroll
            for (int r = 0; r < SUM_UNROLL; ++r) {
#pragma unroll
                for (int u = 0; u < KVEC; ++u) {
                    const uint32_t i = v + r * stride + u;
                    if (i < p0 || i >= p1) continue;
                    const K k = kv[r].k[u];
                    if (c0 && k == r0) {
                        ++c0;
                    } else if (c1 && k == r1) {
                        ++c1;
                    } else {
                        flush(r1, c1);
                        r1 = r0;
                        c1 = c0;
                        r0 = k;
                        c0 = 1;
                    }
                }
            }
        }
        flush(r0, c0);
        flush(r1, c1);
        __syncthreads();
        if (s_over) {
            if (threadIdx.x == 0) atomicOr(S.len + l, SUM_OVERFLOW);
        } else {
            K* gk = static_cast<K*>(S.keys) + (size_t)l * SUM_SLOTS;
            uint32_t* gc = S.cnt + (size_t)l * SUM_SLOTS;
            for (uint32_t t = threadIdx.x; t < SUM_LOCAL; t += blockDim.x) {
                const K k = s_key[t];
                if (k == EMPTY) continue;
                uint32_t h = key_slot(k, SUM_SLOTS - 1);
                bool placed = false;
                for (uint32_t probe = 0; probe < SUM_SLOTS && !placed; ++probe) {
                    const K old = cas_key(gk + h, EMPTY, k);
                    if (old == EMPTY || old == k) {
                        atomicAdd(gc + h, s_cnt[t]);
                        placed = true;
                    }
                    h = (h + 1) & (SUM_SLOTS - 1);
                }
                if (!placed) atomicOr(S.len + l, SUM_OVERFLOW);
            }
            if (threadIdx.x == 0 && s_spec) atomicAdd(S.spec + l, s_spec);
        }
        __syncthreads();
    }
}

// One warp per long bucket: its table's entries sorted by key (rank = number
// of smaller keys; the keys are distinct), the all-ones key last.
template <typename K>
__global__ void __launch_bounds__(256) k_sum_finish(SumBuild S) {
    constexpr K EMPTY = ~(K)0;
    constexpr int PER = SUM_SLOTS / 32;
    const unsigned lane = lane_id();
    const uint32_t L = min(*S.F.n_long, S.F.cap);
    const uint32_t gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint32_t nw = (gridDim.x * blockDim.x) >> 5;
    for (uint32_t l = gw; l < L; l += nw) {
        if (S.len[l] == SUM_OVERFLOW) continue;
        K* gk = static_cast<K*>(S.keys) + (size_t)l * SUM_SLOTS;
        uint32_t* gc = S.cnt + (size_t)l * SUM_SLOTS;
        K k[PER];
        uint32_t c[PER], rank[PER];
        uint32_t m = 0;
#pragma unroll
        for (int j = 0; j < PER; ++j) {
            k[j] = gk[j * 32 + lane];
            c[j] = gc[j * 32 + lane];
            rank[j] = 0;
            m += __popc(__ballot_sync(FULL_MASK, k[j] != EMPTY));
        }
#pragma unroll
        for (int jj = 0; jj < PER; ++jj)
            for (int src = 0; src < 32; ++src) {
                const K o = __shfl_sync(FULL_MASK, k[jj], src);
#pragma unroll
                for (int j = 0; j < PER; ++j) rank[j] += (o != EMPTY && o < k[j]) ? 1u : 0u;
            }
        const uint32_t sp = S.spec[l];
        const uint32_t n = m + (sp ? 1u : 0u);
        __syncwarp();
        if (n > SUM_SLOTS) {
            if (lane == 0) S.len[l] = SUM_OVERFLOW;
            continue;
        }
#pragma unroll
        for (int j = 0; j < PER; ++j) {
            if (k[j] == EMPTY) continue;
            gk[rank[j]] = k[j];
            gc[rank[j]] = c[j];
        }
        if (lane == 0) {
            if (sp) {
                gk[m] = EMPTY;
                gc[m] = sp;
            }
            S.len[l] = n;
        }
        __syncwarp();
    }
}

// Capacity: a long bucket holds more than SUM_MIN_LEN keys, so there are at most n / (SUM_MIN_LEN + 1).
uint32_t summary_cap(uint64_t n) { return (uint32_t)(n / (SUM_MIN_LEN + 1)); }

SumBuild sum_build_of(const Table& t) {
    SumBuild S{};
    S.F = t.finder;
    char* base = static_cast<char*>(t.sum_mem);
    const uint32_t cap = t.sum_cap;
    auto al = [](size_t x) { return (x + 255) & ~size_t(255); };
    size_t off = 0;
    off += al((size_t)(S.F.map_mask + 1) * 8);                  // map
    const size_t o_keys = off; off += al((size_t)cap * SUM_SLOTS * t.key_bytes);
    const size_t o_hdr = off; off += 256;
    const size_t o_spec = off; off += al((size_t)cap * 4);
    const size_t o_len = off; off += al((size_t)cap * 4);
    const size_t o_cnt = off; off += al((size_t)cap * SUM_SLOTS * 4);
    off += al((size_t)cap * 4);                                   // bucket
    const size_t o_item = off;
    S.total_chunks = reinterpret_cast<uint32_t*>(base + o_hdr) + 1;
    S.item = reinterpret_cast<uint4*>(base + o_item);
    S.max_items = (uint32_t)(t.n / SUM_CHUNK + cap);
    S.spec = reinterpret_cast<uint32_t*>(base + o_spec);
    S.len = reinterpret_cast<uint32_t*>(base + o_len);
    S.keys = base + o_keys;
    S.cnt = reinterpret_cast<uint32_t*>(base + o_cnt);
    return S;
}

template <typename K>
cudaError_t finish_impl(Table& t, cudaStream_t s) {
    const SumBuild S = sum_build_of(t);
    const uint32_t n_keys = (uint32_t)t.n;
    cudaError_t e;
    if (!t.long_noted) {
        const uint64_t nvec = (t.B + 3) / 4;
        uint64_t blocks = (nvec + 255) / 256;
        const uint64_t maxb = (uint64_t)num_sms() * 8;
        if (blocks > maxb) blocks = maxb;
        if (blocks < 1) blocks = 1;
        launch_begin("sum_find", s);
        k_sum_find<<<(unsigned)blocks, 256, 0, s>>>(t.offsets, t.B, n_keys, S.F);
        launch_end("sum_find", s);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    launch_begin("sum_plan", s);
    k_sum_plan<<<1, 1024, 0, s>>>(t.offsets, n_keys, S);
    launch_end("sum_plan", s);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    {
        uint64_t grid = (uint64_t)num_sms() * 3;
        if (grid > S.max_items) grid = S.max_items;
        launch_begin("sum_count", s);
        k_sum_count<K><<<(unsigned)grid, SUM_THREADS, 0, s>>>(static_cast<const K*>(t.keys), t.offsets, n_keys, S);
        launch_end("sum_count", s);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    uint64_t blocks = ((uint64_t)t.sum_cap * 32 + 255) / 256;
    const uint64_t maxb = (uint64_t)num_sms() * 8;
    if (blocks > maxb) blocks = maxb;
    launch_begin("sum_finish", s);
    k_sum_finish<K><<<(unsigned)blocks, 256, 0, s>>>(S);
    launch_end("sum_finish", s);
    return cudaGetLastError();
}

}  // namespace

cudaError_t summary_prepare(Table& t, cudaStream_t s) {
    const uint32_t cap = summary_cap(t.n);
    if (cap == 0) return cudaSuccess;
    uint32_t map_slots = 2;
    while (map_slots < 2 * cap) map_slots <<= 1;
    auto al = [](size_t x) { return (x + 255) & ~size_t(255); };
    // set to all ones: map, keys; set to zero: header, spec, len, counts; then bucket, items
    size_t off = 0;
    const size_t o_map = off; off += al((size_t)map_slots * 8);
    off += al((size_t)cap * SUM_SLOTS * t.key_bytes);
    const size_t ones_end = off;
    const size_t o_hdr = off; off += 256;
    off += al((size_t)cap * 4);
    off += al((size_t)cap * 4);
    off += al((size_t)cap * SUM_SLOTS * 4);
    const size_t zero_end = off;
    const size_t o_bucket = off; off += al((size_t)cap * 4);
    off += al(((size_t)(t.n / SUM_CHUNK) + cap) * 16);
    void* mem = nullptr;
    cudaError_t e = dev_alloc(&mem, off, s);
    if (e != cudaSuccess) return e;
    char* base = static_cast<char*>(mem);
    t.sum_mem = mem;
    t.sum_cap = cap;
    t.finder.n_long = reinterpret_cast<uint32_t*>(base + o_hdr);
    t.finder.bucket = reinterpret_cast<uint32_t*>(base + o_bucket);
    t.finder.map = reinterpret_cast<unsigned long long*>(base + o_map);
    t.finder.map_mask = map_slots - 1;
    t.finder.cap = cap;
    t.sum_n_long = t.finder.n_long;
    t.sum_bucket = t.finder.bucket;
    const SumBuild S = sum_build_of(t);
    t.sum.map = t.finder.map;
    t.sum.map_mask = t.finder.map_mask;
    t.sum.keys = S.keys;
    t.sum.cnt = S.cnt;
    t.sum.len = S.len;
    e = cudaMemsetAsync(base, 0xFF, ones_end, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(base + ones_end, 0, zero_end - ones_end, s);
    return e;
}

cudaError_t summary_finish(Table& t, cudaStream_t s) {
    if (!t.sum_mem) return cudaSuccess;
    if (t.key_bytes == 4) return finish_impl<uint32_t>(t, s);
    return finish_impl<uint64_t>(t, s);
}

}  // namespace hg
