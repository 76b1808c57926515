// HashGraph query (Sec. 3.3): hash the probe key, read offset[b] and
// offset[b + 1], walk keys[offset[b] .. offset[b + 1]) and count (or gather
// the values of) every key equal to the probe, duplicates included (Sec. 5.4).
//
// Buckets are walked by one of three workers, chosen by the bucket's length:
//   <= WALK_LANE  keys : the query's own lane walks it;
//   <= WALK_WARP  keys : the whole warp walks it with 16-byte loads;
//   longer             : the slot goes to a work list, and a second kernel
//                        splits each listed bucket into LONG_CHUNK-key chunks
//                        spread over every warp of the GPU, adding partial
//                        counts atomically.  This keeps a heavily duplicated
//                        key (millions of copies in one bucket) from holding a
//                        single warp for milliseconds.
#include <cstdint>

#include "hg_device.cuh"

namespace hg {

namespace {

constexpr int PROBE_THREADS = 256;
constexpr uint32_t WALK_LANE = 16;
constexpr uint32_t WALK_WARP = 8192;
constexpr uint32_t LONG_CHUNK = 4096;
constexpr uint32_t COUNT_LONG_CAP = 1u << 22;  // count/join list capacity; overflow -> the warp walks it

enum { OUT_U32 = 0, OUT_U64 = 1, OUT_NONE = 2 };
enum : uint8_t { CLS_NONE = 0, CLS_LANE = 1, CLS_WARP = 2, CLS_LONG = 3 };

struct LongList {
    uint32_t* n;             // entries appended (may exceed cap)
    uint32_t* n_uniq;        // entries that are walked (written by k_long_prep)
    uint64_t* total_chunks;  // written by k_long_prep
    uint32_t* slot;          // [cap] query slot of each entry
    uint64_t* chunk_start;   // [cap] exclusive prefix of chunk counts, over the walked entries
    uint32_t* uniq;          // [cap] walked entries (each distinct query key once when deduplicated)
    uint32_t* rep;           // [cap] entry whose walk answers entry e
    uint32_t* mult;          // [cap] number of entries a walked entry answers
    uint32_t* cursor;        // [cap] gather write cursors (or null)
    uint32_t cap;
    uint64_t qunhash = 0;    // the queries are hashes of 32-bit keys (BinWork::qunhash)
};

// A query as its key: grouped 32-bit queries are held as their hashes (qunhash
// = 1 << 32 | seed), which fmix32_inv undoes; otherwise the word itself.
__device__ __forceinline__ uint32_t query_key(uint32_t w, uint64_t qunhash) {
    return (qunhash >> 32) ? fmix32_inv(w) ^ (uint32_t)qunhash : w;
}
__device__ __forceinline__ uint64_t query_key(uint64_t w, uint64_t) { return w; }
constexpr uint32_t DEDUP_SLOTS = 16384;  // shared-memory hash table of k_long_prep

// The part of a LongList the probe kernels append to.
struct LongSink {
    uint32_t* n;
    uint32_t* slot;
    uint32_t cap;
};
inline LongSink sink_of(const LongList& L) { return LongSink{L.n, L.slot, L.cap}; }

// Longest bucket a probe may count by binary search (0: the table's buckets are not sorted).
inline uint32_t sorted_limit(const Table& t) {
    return (t.flags & HG_SORTED_BUCKETS) ? sorted_bucket_max(t.key_bytes) : 0u;
}

template <typename K>
__device__ __forceinline__ uint32_t lane_count(const K* __restrict__ keys, uint32_t lo, uint32_t hi, K key) {
    uint32_t c = 0;
#pragma unroll 4
    for (uint32_t p = lo; p < hi; ++p) c += (__ldg(keys + p) == key);
    return c;
}

// Number of keys equal to `key` in keys[p0, p1); all 32 lanes call, all get the total.
template <typename K>
__device__ __forceinline__ uint32_t warp_count(const K* __restrict__ keys, uint64_t p0, uint64_t p1, K key) {
    constexpr int VEC = KeyVec<K>::N;
    const unsigned lane = lane_id();
    uint32_t c = 0;
    const uint64_t mis = (reinterpret_cast<uintptr_t>(keys + p0) & 15) / sizeof(K);
    uint64_t a = p0;
    if (mis) {
        uint64_t e = p0 + (VEC - mis);
        if (e > p1) e = p1;
        if (a + lane < e) c += (__ldg(keys + a + lane) == key);
        a = e;
    }
    const uint64_t nv = (p1 - a) / VEC;
    const K* body = keys + a;
#pragma unroll 4
    for (uint64_t v = lane; v < nv; v += 32) {
        const KeyVec<K> kv = load_keys16(body + v * VEC);
#pragma unroll
        for (int j = 0; j < VEC; ++j) c += (kv.k[j] == key);
    }
    a += nv * VEC;
    if (a + lane < p1) c += (__ldg(keys + a + lane) == key);
    return __reduce_add_sync(FULL_MASK, c);
}

// Writes vals[p] for every p in [p0, p1) with keys[p] == key to dst[0, 1, ...] in walk order.
template <typename K>
__device__ __forceinline__ void warp_write_matches(const K* __restrict__ keys, const uint32_t* __restrict__ vals,
                                                   uint64_t p0, uint64_t p1, K key, uint32_t* dst) {
    const unsigned lane = lane_id();
    uint64_t w = 0;
    for (uint64_t base = p0; base < p1; base += 32) {
        const uint64_t p = base + lane;
        const bool match = p < p1 && __ldg(keys + p) == key;
        const unsigned m = __ballot_sync(FULL_MASK, match);
        if (match) dst[w + __popc(m & lanemask_lt())] = __ldg(vals + p);
        w += __popc(m);
    }
}

template <typename T>
__device__ __forceinline__ T block_sum(T v) {
    __shared__ T s_part[32];
    v = warp_sum(v);
    const int w = threadIdx.x >> 5;
    if (lane_id() == 0) s_part[w] = v;
    __syncthreads();
    T r = 0;
    if (w == 0) {
        r = (lane_id() < (blockDim.x >> 5)) ? s_part[lane_id()] : (T)0;
        r = warp_sum(r);
    }
    return r;  // valid in thread 0
}

// Count of `key` in the ascending run keys[lo, hi) (a sorted bucket): the first
// position >= key and the first position > key, by binary search.
template <typename K>
__device__ __forceinline__ uint32_t sorted_count(const K* keys, uint32_t lo, uint32_t hi, K key) {
    uint32_t a = lo, b = hi;
    while (a < b) {
        const uint32_t m = (a + b) >> 1;
        if (keys[m] < key) a = m + 1; else b = m;
    }
    uint32_t c = a, d = hi;
    while (c < d) {
        const uint32_t m = (c + d) >> 1;
        if (keys[m] <= key) c = m + 1; else d = m;
    }
    return c - a;
}

// One lane's group of up to VEC query slots; all 32 lanes of the warp call it together.
template <typename K, int OUT, bool GATHER>
__device__ __forceinline__ void probe_group(const uint64_t (&slot)[KeyVec<K>::N], const bool (&valid)[KeyVec<K>::N],
                                            const K (&qk)[KeyVec<K>::N], const K* __restrict__ keys,
                                            const uint32_t* __restrict__ vals, const uint32_t* __restrict__ offs,
                                            const Hasher& H, uint32_t n_keys, void* counts, const LongSink& L,
                                            const uint64_t* __restrict__ out_offs, uint32_t* out_vals,
                                            uint64_t& acc, uint32_t sorted_max, const LongSummary& S) {
    constexpr int VEC = KeyVec<K>::N;
    const unsigned lane = lane_id();
    uint32_t lo[VEC], hi[VEC], cnt[VEC];
    uint8_t cls[VEC];
#pragma unroll
    for (int j = 0; j < VEC; ++j) {
        lo[j] = hi[j] = 0;
        if (valid[j]) {
            const uint32_t b = bucket_of(qk[j], H);
            lo[j] = __ldg(offs + b);
            hi[j] = __ldg(offs + b + 1);
            // offsets of a completed build satisfy lo <= hi <= n; clamp so that a
            // damaged table can never send a walk outside the keys array
            hi[j] = min(hi[j], n_keys);
            lo[j] = min(lo[j], hi[j]);
        }
    }
#pragma unroll
    for (int j = 0; j < VEC; ++j) {
        const uint32_t len = hi[j] - lo[j];
        cls[j] = !valid[j] ? CLS_NONE : len <= WALK_LANE ? CLS_LANE : len <= WALK_WARP ? CLS_WARP : CLS_LONG;
        cnt[j] = 0;
    }
    if (!GATHER) {
#pragma unroll
        for (int j = 0; j < VEC; ++j) {
            if (cls[j] == CLS_LANE) cnt[j] = lane_count(keys, lo[j], hi[j], qk[j]);
            // sorted buckets (HG_SORTED_BUCKETS) of more keys: two binary searches
            if (cls[j] > CLS_LANE && hi[j] - lo[j] <= sorted_max) {
                cnt[j] = sorted_count(keys, lo[j], hi[j], qk[j]);
                cls[j] = CLS_NONE;
            }
            // summarised long buckets (HG_LONG_SUMMARY): a binary search of their distinct keys
            if (cls[j] == CLS_LONG && S.map) {
                uint32_t c = 0;
                if (summary_count(S, bucket_of(qk[j], H), qk[j], c)) {
                    cnt[j] = c;
                    cls[j] = CLS_NONE;
                }
            }
        }
        // long buckets: append to the work list (warp-aggregated); on overflow the warp walks it
#pragma unroll
        for (int j = 0; j < VEC; ++j) {
            const unsigned lm = __ballot_sync(FULL_MASK, cls[j] == CLS_LONG);
            if (lm) {
                const int leader = __ffs(lm) - 1;
                uint32_t base = 0;
                if ((int)lane == leader) base = atomicAdd(L.n, (uint32_t)__popc(lm));
                base = __shfl_sync(FULL_MASK, base, leader);
                if (cls[j] == CLS_LONG) {
                    const uint32_t pos = base + __popc(lm & lanemask_lt());
                    if (pos < L.cap) L.slot[pos] = (uint32_t)slot[j];
                    else cls[j] = CLS_WARP;
                }
            }
        }
    } else {
#pragma unroll
        for (int j = 0; j < VEC; ++j) {
            if (cls[j] == CLS_LANE) {
                uint64_t w = out_offs[slot[j]];
                for (uint32_t p = lo[j]; p < hi[j]; ++p)
                    if (__ldg(keys + p) == qk[j]) out_vals[w++] = __ldg(vals + p);
            }
        }
    }
    // medium buckets: the warp walks each one together
#pragma unroll
    for (int j = 0; j < VEC; ++j) {
        unsigned mm = __ballot_sync(FULL_MASK, cls[j] == CLS_WARP);
        while (mm) {
            const int src = __ffs(mm) - 1;
            mm &= mm - 1;
            const uint32_t l = __shfl_sync(FULL_MASK, lo[j], src);
            const uint32_t h = __shfl_sync(FULL_MASK, hi[j], src);
            const K key = __shfl_sync(FULL_MASK, qk[j], src);
            if (!GATHER) {
                const uint32_t c = warp_count(keys, l, h, key);
                if ((int)lane == src) cnt[j] = c;
            } else {
                const uint64_t s = __shfl_sync(FULL_MASK, slot[j], src);
                warp_write_matches(keys, vals, l, h, key, out_vals + out_offs[s]);
            }
        }
    }
    if (!GATHER) {
#pragma unroll
        for (int j = 0; j < VEC; ++j) {
            if (!valid[j]) continue;
            if (OUT == OUT_U32) static_cast<uint32_t*>(counts)[slot[j]] = cnt[j];
            if (OUT == OUT_U64) static_cast<uint64_t*>(counts)[slot[j]] = cnt[j];
            acc += cnt[j];
        }
    }
}

// Every query slot of qs[0, q): count (OUT_U32 / OUT_U64 into `counts`, the sum
// into *total when TOTAL) or, when GATHER, write matching values for the
// non-long slots.  Persistent grid; each lane takes a 16-byte group of slots.
template <typename K, int OUT, bool TOTAL, bool GATHER>
__global__ void __launch_bounds__(PROBE_THREADS)
k_probe(const K* __restrict__ qs, uint64_t q, uint64_t head, uint64_t nvec, const K* __restrict__ keys,
        const uint32_t* __restrict__ vals, const uint32_t* __restrict__ offs, Hasher H, uint32_t n_keys, void* counts,
        uint64_t* total, LongSink L, const uint64_t* __restrict__ out_offs, uint32_t* out_vals,
        uint32_t sorted_max, LongSummary S) {
    constexpr int VEC = KeyVec<K>::N;
    const unsigned lane = lane_id();
    const uint64_t gw = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint64_t nw = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    uint64_t acc = 0;
    uint64_t slot[VEC];
    bool valid[VEC];
    K qk[VEC];
    for (uint64_t b0 = gw * 32; b0 < nvec; b0 += nw * 32) {
        const uint64_t v = b0 + lane;
        const bool ok = v < nvec;
        KeyVec<K> kv;
        if (ok) kv = load_keys16(qs + head + v * VEC);
#pragma unroll
        for (int j = 0; j < VEC; ++j) {
            slot[j] = head + v * VEC + j;
            valid[j] = ok;
            qk[j] = ok ? kv.k[j] : (K)0;
        }
        probe_group<K, OUT, GATHER>(slot, valid, qk, keys, vals, offs, H, n_keys, counts, L, out_offs, out_vals, acc,
                                    sorted_max, S);
    }
    if (gw == 0) {
        const uint64_t tail0 = head + nvec * VEC;
        const uint64_t nrem = head + (q - tail0);
#pragma unroll
        for (int j = 0; j < VEC; ++j) {
            valid[j] = (j == 0) && lane < nrem;
            slot[j] = lane < head ? lane : tail0 + (lane - head);
            qk[j] = valid[j] ? qs[slot[j]] : (K)0;
        }
        probe_group<K, OUT, GATHER>(slot, valid, qk, keys, vals, offs, H, n_keys, counts, L, out_offs, out_vals, acc,
                                    sorted_max, S);
    }
    if (TOTAL) {
        const uint64_t s = block_sum(acc);
        if (threadIdx.x == 0 && s) atomicAdd(reinterpret_cast<unsigned long long*>(total), (unsigned long long)s);
    }
}

// One block.  With DEDUP (32-bit keys), entries whose query keys are equal
// (hence in the same bucket, with the same count) are grouped through a
// shared-memory hash table: only the first of each group is walked, and the
// others copy its count afterwards (the list intersection of Sec. 3.3 matches
// each distinct query key of a bucket once).  Then
// chunk_start[u] = sum of ceil(len / LONG_CHUNK) over walked entries before u.
template <typename K, bool DEDUP>
__global__ void __launch_bounds__(1024)
k_long_prep(const K* __restrict__ qs, const uint32_t* __restrict__ offs, Hasher H, uint32_t n_keys, LongList L) {
    extern __shared__ unsigned long long s_ht[];  // DEDUP: (entry << 32 | key), all ones = empty
    __shared__ uint64_t s_warp[32];
    __shared__ uint64_t s_total;
    __shared__ uint32_t s_wu[32], s_tu;
    const uint32_t n = min(*L.n, L.cap);
    const unsigned lane = lane_id();
    const int w = threadIdx.x >> 5;
    if (DEDUP) {
        for (uint32_t i = threadIdx.x; i < DEDUP_SLOTS; i += blockDim.x) s_ht[i] = ~0ull;
        __syncthreads();
        for (uint32_t e = threadIdx.x; e < n; e += blockDim.x) {
            const uint32_t key = (uint32_t)query_key(qs[L.slot[e]], L.qunhash);
            uint32_t h = fmix32(key ^ 0x9e3779b9u) & (DEDUP_SLOTS - 1);
            uint32_t r = e;
            for (uint32_t probe = 0; probe < DEDUP_SLOTS; ++probe) {
                unsigned long long wv = s_ht[h];
                if (wv == ~0ull) {
                    wv = atomicCAS(&s_ht[h], ~0ull, ((unsigned long long)e << 32) | key);
                    if (wv == ~0ull) break;  // this entry heads its group
                }
                if ((uint32_t)wv == key) {
                    r = (uint32_t)(wv >> 32);
                    break;
                }
                h = (h + 1) & (DEDUP_SLOTS - 1);
            }
            L.rep[e] = r;  // a full table leaves r = e: the entry is walked on its own
        }
        __syncthreads();
        for (uint32_t e = threadIdx.x; e < n; e += blockDim.x)
            if (L.rep[e] == e) L.mult[e] = 1;
        __syncthreads();
        for (uint32_t e = threadIdx.x; e < n; e += blockDim.x)
            if (L.rep[e] != e) atomicAdd(L.mult + L.rep[e], 1u);
    }
    // list of walked entries (block-wide compaction, input order)
    uint32_t nu = 0;
    for (uint32_t base = 0; base < n; base += blockDim.x) {
        const uint32_t e = base + threadIdx.x;
        const uint32_t u = (e < n && (!DEDUP || L.rep[e] == e)) ? 1u : 0u;
        const uint32_t incl = warp_inclusive_scan(u);
        if (lane == 31) s_wu[w] = incl;
        __syncthreads();
        if (w == 0) {
            const uint32_t wv = lane < (blockDim.x >> 5) ? s_wu[lane] : 0;
            const uint32_t wi = warp_inclusive_scan(wv);
            if (lane < (blockDim.x >> 5)) s_wu[lane] = wi - wv;
            if (lane == 31) s_tu = wi;
        }
        __syncthreads();
        if (u) {
            L.uniq[nu + s_wu[w] + incl - u] = e;
            if (!DEDUP) {
                L.rep[e] = e;
                L.mult[e] = 1;
            }
        }
        nu += s_tu;
        __syncthreads();
    }
    uint64_t running = 0;
    for (uint32_t base = 0; base < nu; base += blockDim.x) {
        const uint32_t u = base + threadIdx.x;
        uint64_t ch = 0;
        if (u < nu) {
            const uint32_t b = bucket_of(query_key(qs[L.slot[L.uniq[u]]], L.qunhash), H);
            const uint32_t hi = min(offs[b + 1], n_keys);
            const uint32_t lo = min(offs[b], hi);
            ch = (hi - lo + LONG_CHUNK - 1) / LONG_CHUNK;
        }
        const uint64_t incl = warp_inclusive_scan(ch);
        if (lane == 31) s_warp[w] = incl;
        __syncthreads();
        if (w == 0) {
            const uint64_t wv = lane < (blockDim.x >> 5) ? s_warp[lane] : 0;
            const uint64_t wi = warp_inclusive_scan(wv);
            if (lane < (blockDim.x >> 5)) s_warp[lane] = wi - wv;
            if (lane == 31) s_total = wi;
        }
        __syncthreads();
        if (u < nu) L.chunk_start[u] = running + s_warp[w] + incl - ch;
        running += s_total;
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        *L.total_chunks = running;
        *L.n_uniq = nu;
    }
}

// Long buckets, one LONG_CHUNK-key chunk per warp iteration, over the walked entries.
template <typename K, int OUT, bool TOTAL, bool GATHER>
__global__ void __launch_bounds__(PROBE_THREADS)
k_long(const K* __restrict__ qs, const K* __restrict__ keys, const uint32_t* __restrict__ vals,
       const uint32_t* __restrict__ offs, Hasher H, uint32_t n_keys, LongList L, void* counts, uint64_t* total,
       const uint64_t* __restrict__ out_offs, uint32_t* out_vals) {
    const unsigned lane = lane_id();
    const uint64_t gw = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint64_t nw = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    const uint64_t nchunks = *L.total_chunks;
    const uint32_t nu = *L.n_uniq;
    uint64_t acc = 0;
    for (uint64_t c = gw; c < nchunks; c += nw) {
        // walked entry u: the last with chunk_start[u] <= c
        uint32_t lo = 0, hi = nu;
        while (hi - lo > 1) {
            const uint32_t mid = (lo + hi) >> 1;
            if (L.chunk_start[mid] <= c) lo = mid; else hi = mid;
        }
        const uint32_t u = lo;
        const uint32_t e = L.uniq[u];
        const uint32_t s = L.slot[e];
        const K key = query_key(qs[s], L.qunhash);
        const uint32_t b = bucket_of(key, H);
        const uint64_t l1 = min(offs[b + 1], n_keys);
        const uint64_t l0 = min((uint64_t)offs[b], l1);
        const uint64_t p0 = l0 + (c - L.chunk_start[u]) * LONG_CHUNK;
        const uint64_t p1 = min(l1, p0 + LONG_CHUNK);
        const uint32_t cnt = warp_count(keys, p0, p1, key);
        if (!GATHER) {
            if (lane == 0 && cnt) {
                if (OUT == OUT_U32) atomicAdd(static_cast<uint32_t*>(counts) + s, cnt);
                if (OUT == OUT_U64)
                    atomicAdd(reinterpret_cast<unsigned long long*>(counts) + s, (unsigned long long)cnt);
                acc += (uint64_t)cnt * L.mult[e];
            }
        } else if (cnt) {
            uint32_t base = 0;
            if (lane == 0) base = atomicAdd(L.cursor + e, cnt);
            base = __shfl_sync(FULL_MASK, base, 0);
            warp_write_matches(keys, vals, p0, p1, key, out_vals + out_offs[s] + base);
        }
    }
    if (TOTAL) {
        const uint64_t sum = block_sum(acc);
        if (threadIdx.x == 0 && sum) atomicAdd(reinterpret_cast<unsigned long long*>(total), (unsigned long long)sum);
    }
}

// Entries answered by another entry's walk copy its (now final) count.
template <int OUT>
__global__ void __launch_bounds__(PROBE_THREADS)
k_long_copy(LongList L, void* counts) {
    const uint32_t n = min(*L.n, L.cap);
    for (uint32_t e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += gridDim.x * blockDim.x) {
        const uint32_t r = L.rep[e];
        if (r == e) continue;
        if (OUT == OUT_U32) static_cast<uint32_t*>(counts)[L.slot[e]] = static_cast<uint32_t*>(counts)[L.slot[r]];
        if (OUT == OUT_U64) static_cast<uint64_t*>(counts)[L.slot[e]] = static_cast<uint64_t*>(counts)[L.slot[r]];
    }
}

template <typename Kern>
unsigned persistent_grid(Kern kern) {
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, PROBE_THREADS, 0) != cudaSuccess || per_sm < 1)
        per_sm = 1;
    return (unsigned)(num_sms() * per_sm);
}

// Scratch layout of a long-bucket list with `cap` entries (16-byte header, then arrays).
void map_list(void* mem, uint32_t cap, bool with_cursor, LongList* L) {
    char* p = static_cast<char*>(mem);
    L->n = reinterpret_cast<uint32_t*>(p);
    L->n_uniq = reinterpret_cast<uint32_t*>(p + 4);
    L->total_chunks = reinterpret_cast<uint64_t*>(p + 8);
    L->chunk_start = reinterpret_cast<uint64_t*>(p + 16);
    L->slot = reinterpret_cast<uint32_t*>(p + 16 + (size_t)cap * 8);
    L->uniq = L->slot + cap;
    L->rep = L->uniq + cap;
    L->mult = L->rep + cap;
    L->cursor = with_cursor ? L->mult + cap : nullptr;
    L->cap = cap;
}

cudaError_t alloc_list(uint32_t cap, bool with_cursor, cudaStream_t s, void** mem, LongList* L) {
    const size_t bytes = 16 + (size_t)cap * (8 + 16 + (with_cursor ? 4 : 0)) + 16;
    cudaError_t e = dev_alloc(mem, bytes, s);
    if (e != cudaSuccess) return e;
    map_list(*mem, cap, with_cursor, L);
    e = cudaMemsetAsync(*mem, 0, 16, s);
    if (e == cudaSuccess && with_cursor) e = cudaMemsetAsync(L->cursor, 0, (size_t)cap * 4, s);
    return e;
}

// Prepares the long-bucket walk (deduplicated when allowed, for 32-bit keys).
template <typename K, bool ALLOW_DEDUP>
cudaError_t launch_long_prep(const Table& t, const K* qs, const LongList& L, cudaStream_t s) {
    constexpr bool DEDUP = sizeof(K) == 4 && ALLOW_DEDUP;
    auto kern = k_long_prep<K, DEDUP>;
    const size_t smem = DEDUP ? DEDUP_SLOTS * sizeof(unsigned long long) : 0;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    launch_begin("long_prep", s);
    kern<<<1, 1024, smem, s>>>(qs, t.offsets, t.H, (uint32_t)t.n, L);
    launch_end("long_prep", s);
    return cudaGetLastError();
}

template <int OUT>
cudaError_t launch_long_copy(const LongList& L, void* counts, cudaStream_t s) {
    if (OUT == OUT_NONE) return cudaSuccess;
    launch_begin("long", s);
    k_long_copy<OUT><<<num_sms() * 2, PROBE_THREADS, 0, s>>>(L, counts);
    launch_end("long", s);
    return cudaGetLastError();
}

template <typename K>
void split_vec(const K* qs, uint64_t q, uint64_t* head, uint64_t* nvec) {
    constexpr int VEC = KeyVec<K>::N;
    uint64_t h = ((16 - (reinterpret_cast<uintptr_t>(qs) & 15)) & 15) / sizeof(K);
    if (h > q) h = q;
    *head = h;
    *nvec = (q - h) / VEC;
}

template <typename K, int OUT, bool TOTAL, bool GATHER>
cudaError_t run_probe(const Table& t, const K* qs, uint64_t q, void* counts, uint64_t* total, const LongList& L,
                      const uint64_t* out_offs, uint32_t* out_vals, cudaStream_t s) {
    uint64_t head, nvec;
    split_vec(qs, q, &head, &nvec);
    const K* keys = static_cast<const K*>(t.keys);
    {
        auto kern = k_probe<K, OUT, TOTAL, GATHER>;
        unsigned g = persistent_grid(kern);
        const uint64_t need = (nvec + PROBE_THREADS) / PROBE_THREADS;
        if (need < g) g = (unsigned)(need < 1 ? 1 : need);
        launch_begin(GATHER ? "gather" : "probe", s);
        kern<<<g, PROBE_THREADS, 0, s>>>(qs, q, head, nvec, keys, t.values, t.offsets, t.H, (uint32_t)t.n, counts,
                                         total, sink_of(L), out_offs, out_vals,
                                         // a gather's two phases must agree on the long slots: both walk
                                         (GATHER || OUT == OUT_U64) ? 0u : sorted_limit(t),
                                         (GATHER || OUT == OUT_U64) ? LongSummary{} : t.sum);
        launch_end(GATHER ? "gather" : "probe", s);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    if (!GATHER) {
        // counts feeding a gather (OUT_U64) keep one walk per entry: the gather's
        // second phase walks every entry itself
        cudaError_t e = launch_long_prep<K, OUT != OUT_U64>(t, qs, L, s);
        if (e != cudaSuccess) return e;
    }
    auto kern = k_long<K, OUT, TOTAL, GATHER>;
    launch_begin(GATHER ? "long_gather" : "long", s);
    kern<<<persistent_grid(kern), PROBE_THREADS, 0, s>>>(qs, keys, t.values, t.offsets, t.H, (uint32_t)t.n, L,
                                                       counts, total, out_offs, out_vals);
    launch_end(GATHER ? "long_gather" : "long", s);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess || GATHER || OUT == OUT_U64) return e;
    return launch_long_copy<OUT>(L, counts, s);
}

// Byte-model helper: stats[0] += sum of walked bucket lengths, stats[1] += the
// part in buckets longer than WALK_WARP, stats[2] += number of such slots;
// 32-byte sectors touched by the walks outside long buckets (stats[4]) and by
// the offset pairs (stats[5]).
template <typename K>
__global__ void __launch_bounds__(PROBE_THREADS)
k_walk_stats(const K* __restrict__ qs, uint64_t q, const uint32_t* __restrict__ offs, Hasher H, uint64_t* stats) {
    uint64_t w = 0, wl = 0, nl = 0, ks = 0, os = 0;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < q; i += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t b = bucket_of(qs[i], H);
        const uint32_t lo = offs[b], len = offs[b + 1] - lo;
        w += len;
        if (len > WALK_WARP) {
            wl += len;
            nl += 1;
        } else if (len) {
            const uint64_t a = (uint64_t)lo * sizeof(K), e = (uint64_t)(lo + len) * sizeof(K);
            ks += (e + 31) / 32 - a / 32;
        }
        os += ((uint64_t)b * 4 + 7) / 32 - ((uint64_t)b * 4) / 32 + 1;  // offsets b and b + 1
    }
    const uint64_t a = block_sum(w);
    __syncthreads();
    const uint64_t c = block_sum(wl);
    __syncthreads();
    const uint64_t d = block_sum(nl);
    __syncthreads();
    const uint64_t f = block_sum(ks);
    __syncthreads();
    const uint64_t g = block_sum(os);
    if (threadIdx.x == 0) {
        atomicAdd(reinterpret_cast<unsigned long long*>(stats), (unsigned long long)a);
        atomicAdd(reinterpret_cast<unsigned long long*>(stats + 1), (unsigned long long)c);
        atomicAdd(reinterpret_cast<unsigned long long*>(stats + 2), (unsigned long long)d);
        atomicAdd(reinterpret_cast<unsigned long long*>(stats + 4), (unsigned long long)f);
        atomicAdd(reinterpret_cast<unsigned long long*>(stats + 5), (unsigned long long)g);
    }
}

// One table bin per CTA work item (the paper's per-bucket intersection,
// Sec. 3.3, done a bin of 8192 buckets at a time).  The bin's offsets and
// (when they fit) keys are brought into shared memory by bulk copies (TMA);
// each CTA holds one bin at a time and two CTAs share an SM, so one CTA's
// copies overlap the other's queries (this measured faster than one CTA of
// 1024 threads double-buffering two bins).  Buckets longer than WALK_WARP keys go to the
// long-bucket list as in the direct probe; a bin whose keys do not fit is
// walked in global memory.  Equal query keys share a bucket, hence a bin: for
// 32-bit keys, the count of every warp-walked bucket is kept in a small
// per-bin shared-memory table, so a key queried again in the same bin is
// answered without walking (the per-bucket list intersection of Sec. 3.3
// matches each distinct query key once).  Every wait on a copy is bounded.
constexpr uint32_t BIN_KEY_BYTES = 72 * 1024;                                  // per buffer
constexpr uint32_t BIN_OFF_BYTES = ((BIN_BUCKETS + 1) * 4 + 15) / 16 * 16;     // 8193 offsets, rounded to 16 B
constexpr uint32_t BIN_BUF_BYTES = BIN_OFF_BYTES + BIN_KEY_BYTES;
constexpr int BIN_PROBE_THREADS = 512;
constexpr int BIN_PROBE_CTAS_PER_SM = 2;
constexpr int BIN_BUFFERS = 1;  // bins in flight per CTA (2 = double buffering within the CTA)
constexpr uint32_t COPY_WAIT_LIMIT = 1u << 26;  // polls of a copy's barrier (far beyond any real copy)
constexpr uint32_t CACHE_SLOTS = 512;           // per-bin (key, count) table; linear probing
constexpr uint32_t CACHE_PROBES = 8;
constexpr unsigned long long CACHE_EMPTY = ~0ull;  // a count never reaches 2^32 - 1 here

template <typename K, int OUT, bool TOTAL>
__global__ void __launch_bounds__(BIN_PROBE_THREADS, BIN_PROBE_CTAS_PER_SM)
k_probe_bins(const K* __restrict__ qs, const uint32_t* __restrict__ qbin_start, BinWork W,
             const K* __restrict__ keys, const uint32_t* __restrict__ offs, Hasher H, uint32_t n_keys, void* counts,
             uint64_t* total, LongSink L, uint32_t* work_ctr, uint32_t* err, uint32_t sorted_max, LongSummary S,
             const uint32_t* __restrict__ list, const uint32_t* __restrict__ n_list) {
    constexpr uint32_t KVEC = 16 / sizeof(K);
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ __align__(8) uint64_t s_bar[2];
    __shared__ uint32_t s_bin[2], s_k0[2], s_klo[2], s_staged[2], s_q0[2], s_q1[2];
    static_assert(BIN_BUFFERS == 1 || BIN_BUFFERS == 2, "one or two bin buffers");
    constexpr bool CACHE = sizeof(K) == 4;
    __shared__ unsigned long long s_cache[CACHE ? CACHE_SLOTS : 1];  // (count << 32 | key)
    const unsigned lane = lane_id();
    const uint32_t warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    const uint64_t B = H.B;
    uint64_t acc = 0;
    const uint32_t n_huge = *W.n_huge, huge_items = *W.huge_chunks;
    const uint32_t n_items = huge_items + *W.n_work;

    if (threadIdx.x == 0) {
        mbar_init(&s_bar[0], 1);
        mbar_init(&s_bar[1], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    // thread 0: claim the next work item (a slice of a huge bin's queries, or a
    // whole bin) and start the copies of its bin into buffer b
    // (with a list: only the listed items)
    auto issue = [&](int b) {
        uint32_t item = atomicAdd(work_ctr, 1u);
        if (list) {
            if (item >= *n_list) {
                s_bin[b] = ~0u;
                return;
            }
            item = list[item];
        }
        if (item >= n_items) {
            s_bin[b] = ~0u;
            return;
        }
        uint32_t p;
        if (item < huge_items) {
            uint32_t lo = 0, hi = n_huge;  // last huge bin e with huge_chunk_start[e] <= item
            while (hi - lo > 1) {
                const uint32_t mid = (lo + hi) >> 1;
                if (W.huge_chunk_start[mid] <= item) lo = mid; else hi = mid;
            }
            p = W.huge_bin[lo];
            const uint32_t c0 = qbin_start[p] + (item - W.huge_chunk_start[lo]) * W.huge_chunk;
            s_q0[b] = c0;
            s_q1[b] = min(qbin_start[p + 1], c0 + W.huge_chunk);
        } else {
            p = W.work[item - huge_items];
            s_q0[b] = qbin_start[p];
            s_q1[b] = qbin_start[p + 1];
        }
        s_bin[b] = p;
        const uint64_t b0 = (uint64_t)p * BIN_BUCKETS;
        const uint32_t nb = (uint32_t)min((uint64_t)BIN_BUCKETS, B - b0);
        const uint32_t k0 = min(__ldg(offs + b0), n_keys);
        const uint32_t k1 = max(k0, min(__ldg(offs + b0 + nb), n_keys));
        const uint32_t klo = k0 & ~(KVEC - 1);
        const uint32_t off_bytes = ((nb + 1) * 4 + 15) & ~15u;
        const uint32_t key_bytes = (uint32_t)((((uint64_t)(k1 - klo)) * sizeof(K) + 15) & ~15ull);
        const bool staged = (uint64_t)(k1 - klo) * sizeof(K) <= BIN_KEY_BYTES;
        s_k0[b] = k0;
        s_klo[b] = klo;
        s_staged[b] = staged;
        unsigned char* buf = smem + (size_t)b * BIN_BUF_BYTES;
        fence_proxy_async_smem();
        mbar_arrive_expect_tx(&s_bar[b], off_bytes + (staged ? key_bytes : 0u));
        bulk_load(buf, offs + b0, off_bytes, &s_bar[b]);
        if (staged && key_bytes) bulk_load(buf + BIN_OFF_BYTES, keys + klo, key_bytes, &s_bar[b]);
    };
    if (BIN_BUFFERS == 2 && threadIdx.x == 0) issue(0);
    uint32_t phase0 = 0, phase1 = 0;
    int cur = 0;
    bool failed = false;
    while (true) {
        // the buffer's previous user finished at the last barrier: with two buffers
        // the next bin's copies start now, with one the current bin's
        if (threadIdx.x == 0) issue(BIN_BUFFERS == 2 ? (cur ^ 1) : 0);
        if (CACHE)
            for (uint32_t t = threadIdx.x; t < CACHE_SLOTS; t += blockDim.x) s_cache[t] = CACHE_EMPTY;
        __syncthreads();
        const uint32_t p = s_bin[cur];
        if (p == ~0u) break;
        {
            const uint32_t ph = cur ? phase1 : phase0;
            uint32_t polls = 0;
            while (!mbar_test_parity(&s_bar[cur], ph) && ++polls < COPY_WAIT_LIMIT) {
            }
            failed = polls >= COPY_WAIT_LIMIT;
            if (cur) phase1 ^= 1; else phase0 ^= 1;
        }
        failed = __syncthreads_or(failed) != 0;  // the same in every thread
        if (failed) break;
        const uint32_t* s_off = reinterpret_cast<const uint32_t*>(smem + (size_t)cur * BIN_BUF_BYTES);
        const uint32_t k0 = s_k0[cur];
        const bool staged = s_staged[cur] != 0;
        const K* kb = staged ? reinterpret_cast<const K*>(smem + (size_t)cur * BIN_BUF_BYTES + BIN_OFF_BYTES) +
                                   (k0 - s_klo[cur])
                             : keys + k0;  // keys of the bin, indexed from k0
        const uint32_t q0 = s_q0[cur], q1 = s_q1[cur];
        const uint64_t b0 = (uint64_t)p * BIN_BUCKETS;
        const uint32_t nb = (uint32_t)min((uint64_t)BIN_BUCKETS, B - b0);
        // each warp answers 32 queries at a time; the next 32 are loaded meanwhile
        // (raw words: a grouped query becomes its key where it is used, so the load stays in flight)
        K key_next = (q0 + warp * 32 + lane < q1) ? __ldg(qs + q0 + warp * 32 + lane) : (K)0;
        for (uint32_t i0 = q0 + warp * 32; i0 < q1; i0 += nwarps * 32) {
            const uint32_t i = i0 + lane;
            const bool ok = i < q1;
            const K key = query_key(key_next, W.qunhash);
            {
                const uint32_t inext = i + nwarps * 32;
                key_next = inext < q1 ? __ldg(qs + inext) : (K)0;
            }
            uint32_t lo = 0, hi = 0, j = 0;
            if (ok) {
                j = bucket_of(key, H) - (uint32_t)b0;
                if (j >= nb) j = nb - 1;  // queries of this bin hash into it by construction
                lo = min(s_off[j], n_keys) - k0;
                hi = max(min(s_off[j + 1], n_keys) - k0, lo);
            }
            const uint32_t len = hi - lo;
            uint8_t cls = !ok ? CLS_NONE : len <= WALK_LANE ? CLS_LANE : len <= WALK_WARP ? CLS_WARP : CLS_LONG;
            uint32_t cnt = 0;
            if (cls > CLS_LANE && len <= sorted_max) {  // a sorted bucket (HG_SORTED_BUCKETS)
                cnt = sorted_count(kb, lo, hi, key);
                cls = CLS_NONE;
            }
            if (cls == CLS_LANE)
                for (uint32_t x = lo; x < hi; ++x) cnt += (kb[x] == key);
            // a key already counted in this bin takes its count from the table
            if (CACHE && cls >= CLS_WARP) {
                uint32_t sl = j & (CACHE_SLOTS - 1);
                for (uint32_t t = 0; t < CACHE_PROBES; ++t) {
                    const unsigned long long w = s_cache[sl];
                    if (w == CACHE_EMPTY) break;
                    if ((uint32_t)w == (uint32_t)key) {
                        cnt = (uint32_t)(w >> 32);
                        cls = CLS_NONE;
                        break;
                    }
                    sl = (sl + 1) & (CACHE_SLOTS - 1);
                }
            }
            // summarised long buckets (HG_LONG_SUMMARY): a binary search of their distinct keys
            bool summarised = false;
            if (cls == CLS_LONG && S.map) {
                summarised = summary_count(S, (uint32_t)b0 + j, key, cnt);
                if (summarised) cls = CLS_NONE;
            }
            // other long buckets to the list (warp-aggregated); on overflow the warp walks them
            const unsigned lm = __ballot_sync(FULL_MASK, cls == CLS_LONG);
            if (lm) {
                const int leader = __ffs(lm) - 1;
                uint32_t base = 0;
                if ((int)lane == leader) base = atomicAdd(L.n, (uint32_t)__popc(lm));
                base = __shfl_sync(FULL_MASK, base, leader);
                if (cls == CLS_LONG) {
                    const uint32_t pos = base + __popc(lm & lanemask_lt());
                    if (pos < L.cap) L.slot[pos] = i;
                    else cls = CLS_WARP;
                }
            }
            unsigned mm = __ballot_sync(FULL_MASK, cls == CLS_WARP);
            const bool walked = cls == CLS_WARP;
            while (mm) {
                const int src = __ffs(mm) - 1;
                mm &= mm - 1;
                const uint32_t l = __shfl_sync(FULL_MASK, lo, src);
                const uint32_t h = __shfl_sync(FULL_MASK, hi, src);
                const K kk = __shfl_sync(FULL_MASK, key, src);
                uint32_t c = 0;
                for (uint32_t x = l + lane; x < h; x += 32) c += (kb[x] == kk);
                c = __reduce_add_sync(FULL_MASK, c);
                if ((int)lane == src) cnt = c;
            }
            if (CACHE && (walked || summarised)) {  // record the count (a full neighbourhood just skips it)
                const unsigned long long w = ((unsigned long long)cnt << 32) | (uint32_t)key;
                uint32_t sl = j & (CACHE_SLOTS - 1);
                for (uint32_t t = 0; t < CACHE_PROBES; ++t) {
                    const unsigned long long old = atomicCAS(&s_cache[sl], CACHE_EMPTY, w);
                    if (old == CACHE_EMPTY || (uint32_t)old == (uint32_t)key) break;
                    sl = (sl + 1) & (CACHE_SLOTS - 1);
                }
            }
            if (ok) {
                if (OUT == OUT_U32) static_cast<uint32_t*>(counts)[i] = cnt;
                if (OUT == OUT_U64) static_cast<uint64_t*>(counts)[i] = cnt;
                acc += cnt;
            }
        }
        __syncthreads();
        if (BIN_BUFFERS == 2) cur ^= 1;
    }
    if (failed) {
        // a copy never completed (not expected): record it, give the other buffer's
        // copy a bounded chance to land, and leave
        if (threadIdx.x == 0) {
            atomicOr(err, DEVERR_TIMEOUT);
            const int other = cur ^ 1;
            if (BIN_BUFFERS == 2 && s_bin[other] != ~0u) {
                const uint32_t ph = other ? phase1 : phase0;
                uint32_t polls = 0;
                while (!mbar_test_parity(&s_bar[other], ph) && ++polls < COPY_WAIT_LIMIT) {
                }
            }
        }
        return;
    }
    if (TOTAL) {
        const uint64_t sum = block_sum(acc);
        if (threadIdx.x == 0 && sum) atomicAdd(reinterpret_cast<unsigned long long*>(total), (unsigned long long)sum);
    }
}

// Grouped probe by hash join (32-bit keys): the paper's per-bucket list
// intersection done a bin at a time through a table of the bin's distinct keys.
// A CTA takes one work item (a bin's queries, or a slice of them for a bin with
// very many), brings the bin's keys into shared memory by a bulk copy, counts
// them into a shared-memory
// open-addressing table of (count << 32 | key) words (zero = empty: a present
// key has a count of at least one; double hashing, so probe sequences do not
// cluster and a warp's 32 lookups end together) -- each warp reads 32
// consecutive keys, and only the first lane of each run of equal keys inserts,
// with the run's length -- and answers every query with one table lookup: the
// count of a key in its bin is its count in its bucket.  A bin whose keys do
// not fit ("hot": it holds some of the longest buckets) is still taken when the
// table has long-bucket summaries (HG_LONG_SUMMARY): the CTA finds the bin's
// buckets of more than SUM_MIN_LEN keys from its offsets, copies only the keys
// between them, and counts each long bucket from its summary instead.  Items
// this kernel does not take go to a list for k_probe_bins: bins that do not fit
// even so (or with more than HJ_MAX_LONG long buckets), and bins with more
// distinct keys than the table holds (if most bins are like that, the rest are
// not tried).
constexpr uint32_t HJ_SLOTS = 4096;                   // table words (32 KiB)
constexpr uint32_t HJ_MAX_FILL = HJ_SLOTS * 3 / 4;    // distinct keys before the bin falls back
constexpr uint32_t HJ_OVF = 512;                      // bucket-indexed table: overflow words (4 KiB)
constexpr uint32_t HJ_OVF_MAX = HJ_OVF * 3 / 4;       // overflow keys before the bin falls back
constexpr uint32_t HJ_TABLE_BYTES = BIN_BUCKETS * 4 + HJ_OVF * 8;  // either table (36 KiB)
constexpr uint32_t HJ_KEY_BYTES = 76 * 1024;          // staged keys (two CTAs per SM)
static_assert(HJ_SLOTS * 8 <= HJ_TABLE_BYTES, "the hashed table fits the table region");
constexpr int HJ_THREADS = 768;                       // two CTAs (48 warps) per SM: 512 took 1.29 ms, 768 1.14
constexpr uint32_t HJ_TRY_LIMIT = 64;                 // fallbacks before the try-rate test applies
constexpr int HJ_QUNROLL = 4;                         // query loads in flight per thread
constexpr uint32_t HJ_MAX_LONG = 8;                   // long buckets of a hot bin (segments: one more)
static_assert(HJ_KEY_BYTES % 16 == 0, "bulk copies move whole 16-byte units");

// First slot and probe step (odd, so the sequence visits every slot of the
// power-of-two table) of a key's hash h.  h is already well mixed, but the keys
// of one bin share the bits that name the bin, so the slot is taken from the
// top bits of h times 2^32 / golden ratio (Knuth's multiplicative hashing,
// TAOCP vol. 3, Sec. 6.4), which depend on every bit of h.
__device__ __forceinline__ void hj_probe_seq(uint32_t h, uint32_t& slot, uint32_t& step) {
    const uint32_t x = h * 0x9e3779b1u;
    slot = x >> (32 - 12);
    step = (x >> 7) | 1u;
}
static_assert(HJ_SLOTS == 4096, "hj_probe_seq returns 12-bit slots");
// The same for the bucket-indexed table's overflow words.
__device__ __forceinline__ void hj_ovf_seq(uint32_t h, uint32_t& slot, uint32_t& step) {
    const uint32_t x = h * 0x9e3779b1u;
    slot = x >> (32 - 9);
    step = (x >> 7) | 1u;
}
static_assert(HJ_OVF == 512, "hj_ovf_seq returns 9-bit slots");

//
// DM (B = 2^lb with lb >= 16, so a bucket's place in its bin is the low 13 bits
// of the hash, and its keys differ only in the lb..31 bits): the table is
// indexed by bucket instead, a 32-bit word per bucket of the bin holding
// (overflow flag << 31 | tag << (lb - 1) | count), tag = h >> lb, so a query
// is one shared-memory load and compare.  A bucket's second and later distinct
// keys (and a hot bin's summary entries, whose counts need 32 bits) go to a
// small double-hashed table of (count << 32 | h) words, which the bucket's flag
// sends a query to.  A bin whose overflow exceeds HJ_OVF_MAX keys falls back.
// Counts in a bucket's word stay below 2^(lb-1) >= 2^15: it counts staged keys.
template <int OUT, bool TOTAL, bool DM>
__global__ void __launch_bounds__(HJ_THREADS, 2)
k_probe_hash(const uint32_t* __restrict__ qs, const uint32_t* __restrict__ qbin_start, BinWork W,
             const uint32_t* __restrict__ keys, const uint32_t* __restrict__ offs, uint64_t B, uint32_t n_keys,
             void* counts, uint64_t* total, uint32_t* work_ctr, uint32_t* fb_list, uint32_t* fb_n, uint32_t* tries,
             uint32_t* err, LongSummary S, uint32_t hseed, uint32_t lb) {
    static_assert(HJ_KEY_BYTES + HJ_TABLE_BYTES <= 112 * 1024, "two CTAs per SM");
    const bool qhashed = (W.qunhash >> 32) != 0;
    extern __shared__ __align__(128) unsigned char smem[];
    unsigned long long* s_ht = reinterpret_cast<unsigned long long*>(smem);   // !DM
    uint32_t* const s_tab = reinterpret_cast<uint32_t*>(smem);                 // DM: a word per bucket
    unsigned long long* const s_ovf = reinterpret_cast<unsigned long long*>(smem + BIN_BUCKETS * 4);
    const uint32_t cbits = lb - 1, cmask = (1u << cbits) - 1u;
    unsigned char* const s_buf = smem + HJ_TABLE_BYTES;
    const uint32_t* s_keys = reinterpret_cast<const uint32_t*>(s_buf);
    __shared__ __align__(8) uint64_t s_bar;
    __shared__ uint32_t s_p, s_bin, s_k0, s_k1, s_q0, s_q1, s_fill, s_abort, s_hot, s_skip;
    // the keys to count: segment i is s_keys[s_seg_a[i], + s_seg_n[i]); a hot bin's
    // long buckets (source range, summary index)
    __shared__ uint32_t s_nseg, s_seg_a[HJ_MAX_LONG + 1], s_seg_n[HJ_MAX_LONG + 1];
    __shared__ uint32_t s_nlong, s_long_lo[HJ_MAX_LONG], s_long_hi[HJ_MAX_LONG], s_long_l[HJ_MAX_LONG];
    const unsigned lane = lane_id();
    const uint32_t warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    const uint32_t huge_items = *W.huge_chunks;
    const uint32_t n_items = huge_items + *W.n_work;
    uint64_t acc = 0;
    uint32_t phase = 0;
    bool failed = false;
    // thread 0: claim items until one is taken here (the others go to the
    // fallback list) and start the copy of its keys; s_p = ~0u when none is left
    auto claim = [&]() {
        s_p = ~0u;
        while (true) {
            const uint32_t item = atomicAdd(work_ctr, 1u);
            if (item >= n_items) return;
            uint32_t p, q0, q1;
            if (item < huge_items) {  // a slice of a bin with very many queries
                uint32_t lo = 0, hi = *W.n_huge;
                while (hi - lo > 1) {
                    const uint32_t mid = (lo + hi) >> 1;
                    if (W.huge_chunk_start[mid] <= item) lo = mid; else hi = mid;
                }
                p = W.huge_bin[lo];
                q0 = qbin_start[p] + (item - W.huge_chunk_start[lo]) * W.huge_chunk;
                q1 = min(qbin_start[p + 1], q0 + W.huge_chunk);
            } else {
                p = W.work[item - huge_items];
                q0 = qbin_start[p];
                q1 = qbin_start[p + 1];
            }
            if (q0 == q1) continue;  // no queries in this bin
            const uint64_t b0 = (uint64_t)p * BIN_BUCKETS;
            const uint64_t b1 = min(B, b0 + BIN_BUCKETS);
            const uint32_t k0 = min(__ldg(offs + b0), n_keys);
            const uint32_t k1 = max(k0, min(__ldg(offs + b1), n_keys));
            const volatile uint32_t* vt = tries;
            const bool give_up = vt[1] >= HJ_TRY_LIMIT && 2 * vt[1] >= vt[0];
            const uint32_t klo = k0 & ~3u;
            const bool fits = (uint64_t)(k1 - klo) * 4 <= HJ_KEY_BYTES;
            if (give_up || (!fits && !S.map)) {
                fb_list[atomicAdd(fb_n, 1u)] = item;
                continue;
            }
            atomicAdd(tries, 1u);
            s_p = item;
            s_bin = p;
            s_k0 = k0;
            s_k1 = k1;
            s_q0 = q0;
            s_q1 = q1;
            s_hot = fits ? 0u : 1u;
            s_skip = 0;
            s_nlong = 0;
            if (fits) {  // one segment, copied now (overlapping the current item's queries)
                const uint32_t bytes = ((k1 - klo) * 4 + 15) & ~15u;
                s_nseg = 1;
                s_seg_a[0] = k0 - klo;
                s_seg_n[0] = k1 - k0;
                fence_proxy_async_smem();  // the key buffer's earlier reads come before the copy's writes
                mbar_arrive_expect_tx(&s_bar, bytes);
                if (bytes) bulk_load(s_buf, keys + klo, bytes, &s_bar);
            }
            return;
        }
    };
    if (threadIdx.x == 0) {
        mbar_init(&s_bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        claim();
        s_fill = 0;
        s_abort = 0;
    }
    for (uint32_t t = threadIdx.x; t < HJ_TABLE_BYTES / 16; t += blockDim.x)
        reinterpret_cast<uint4*>(smem)[t] = make_uint4(0, 0, 0, 0);
    __syncthreads();
    while (true) {
        // here: the table is empty, and the copy of item s_p's keys is in flight
        const uint32_t item = s_p;
        if (item == ~0u) break;
        const bool hot = s_hot != 0;
        if (hot) {
            // a bin too large to copy whole: list its long buckets from its offsets
            const uint32_t p = s_bin;
            const uint64_t b0 = (uint64_t)p * BIN_BUCKETS;
            const uint32_t nb = (uint32_t)min((uint64_t)BIN_BUCKETS, B - b0);
            for (uint32_t j = threadIdx.x; j < nb; j += blockDim.x) {
                const uint32_t hi = min(__ldg(offs + b0 + j + 1), n_keys);
                const uint32_t lo = min(__ldg(offs + b0 + j), hi);
                if (hi - lo > SUM_MIN_LEN) {
                    const uint32_t x = atomicAdd(&s_nlong, 1u);
                    if (x < HJ_MAX_LONG) {
                        s_long_lo[x] = lo;
                        s_long_hi[x] = hi;
                        s_long_l[x] = (uint32_t)(b0 + j);  // bucket id, then its summary index
                    }
                }
            }
            __syncthreads();
            if (threadIdx.x == 0) {
                const uint32_t nl = s_nlong;
                bool ok = nl <= HJ_MAX_LONG;
                if (ok) {
                    for (uint32_t a = 1; a < nl; ++a) {  // by position (a few entries)
                        const uint32_t lo = s_long_lo[a], hi = s_long_hi[a], l = s_long_l[a];
                        int c = (int)a - 1;
                        while (c >= 0 && s_long_lo[c] > lo) {
                            s_long_lo[c + 1] = s_long_lo[c];
                            s_long_hi[c + 1] = s_long_hi[c];
                            s_long_l[c + 1] = s_long_l[c];
                            --c;
                        }
                        s_long_lo[c + 1] = lo;
                        s_long_hi[c + 1] = hi;
                        s_long_l[c + 1] = l;
                    }
                    for (uint32_t a = 0; a < nl && ok; ++a) {
                        const uint32_t l = summary_index(S, s_long_l[a]);
                        ok = l != SUM_OVERFLOW;
                        s_long_l[a] = l;
                    }
                }
                // the keys between the long buckets, each segment copied to a
                // 16-byte-aligned place in the buffer
                uint32_t nseg = 0, dst = 0, total = 0, cur = s_k0;
                for (uint32_t a = 0; a <= nl && ok; ++a) {
                    const uint32_t e = a < nl ? s_long_lo[a] : s_k1;
                    if (e > cur) {
                        const uint32_t al = cur & ~3u;
                        const uint32_t bytes = ((e - al) * 4 + 15) & ~15u;
                        ok = dst * 4 + bytes <= HJ_KEY_BYTES;
                        s_seg_a[nseg] = dst + (cur - al);
                        s_seg_n[nseg] = e - cur;
                        ++nseg;
                        dst += bytes / 4;
                        total += bytes;
                    }
                    if (a < nl) cur = s_long_hi[a];
                }
                if (ok) {
                    s_nseg = nseg;
                    fence_proxy_async_smem();
                    mbar_arrive_expect_tx(&s_bar, total);
                    cur = s_k0;
                    dst = 0;
                    for (uint32_t a = 0; a <= nl; ++a) {
                        const uint32_t e = a < nl ? s_long_lo[a] : s_k1;
                        if (e > cur) {
                            const uint32_t al = cur & ~3u;
                            const uint32_t bytes = ((e - al) * 4 + 15) & ~15u;
                            bulk_load(s_buf + dst * 4, keys + al, bytes, &s_bar);
                            dst += bytes / 4;
                        }
                        if (a < nl) cur = s_long_hi[a];
                    }
                } else {
                    s_skip = 1;
                    fb_list[atomicAdd(fb_n, 1u)] = item;
                }
            }
            __syncthreads();
            if (s_skip) {  // left to the walking probe: take the next item
                __syncthreads();
                if (threadIdx.x == 0) {
                    claim();
                    s_fill = 0;
                    s_abort = 0;
                }
                __syncthreads();
                continue;
            }
        }
        {
            uint32_t polls = 0;
            while (!mbar_test_parity(&s_bar, phase) && ++polls < COPY_WAIT_LIMIT) {
            }
            failed = polls >= COPY_WAIT_LIMIT;
            phase ^= 1;
        }
        failed = __syncthreads_or(failed) != 0;  // the same in every thread
        if (failed) break;
        const uint32_t q0 = s_q0, q1 = s_q1;
        // the bin's first queries are loaded now: their latency overlaps the table's build
        uint32_t kq[HJ_QUNROLL];
#pragma unroll
        for (int u = 0; u < HJ_QUNROLL; ++u) {
            const uint32_t i = q0 + u * blockDim.x + threadIdx.x;
            kq[u] = i < q1 ? __ldg(qs + i) : 0u;  // raw words, made keys where they are used
        }
        // count the bin's keys: runs of equal keys inside each 32-key step, one
        // insert per run; two steps per iteration for independent loads
        // the table holds each key's hash h = fmix32(k ^ seed) (a bijection, so
        // equal hashes are equal keys), the form in which the grouped queries come
        // DM: (count << 32 | h) into the overflow words
        auto ovf_insert = [&](uint32_t h, uint32_t len) {
            const unsigned long long add = (unsigned long long)len << 32;
            uint32_t sl, stp;
            hj_ovf_seq(h, sl, stp);
            for (uint32_t t = 0; t < HJ_OVF; ++t) {
                unsigned long long w = *static_cast<volatile unsigned long long*>(&s_ovf[sl]);
                if (w == 0ull) {
                    w = atomicCAS(&s_ovf[sl], 0ull, add | h);
                    if (w == 0ull) {
                        if (atomicAdd(&s_fill, 1u) + 1 > HJ_OVF_MAX) s_abort = 1;
                        return;
                    }
                }
                if ((uint32_t)w == h) {
                    atomicAdd(&s_ovf[sl], add);
                    return;
                }
                sl = (sl + stp) & (HJ_OVF - 1);
            }
            s_abort = 1;  // (full: the fill limit stops the bin first)
        };
        // DM: the key with hash h, len times; to_ovf: straight to the overflow words
        auto dm_insert = [&](uint32_t h, uint32_t len, bool to_ovf) {
            uint32_t* const slot = s_tab + (h & (BIN_BUCKETS - 1));
            const uint32_t tag = h >> lb;
            uint32_t w = *static_cast<volatile uint32_t*>(slot);
            while (!to_ovf) {
                if ((w & cmask) == 0u) {  // no key in this bucket yet (its flag may be set)
                    const uint32_t old = atomicCAS(slot, w, w | (tag << cbits) | len);
                    if (old == w) return;
                    w = old;
                } else if (((w & 0x7fffffffu) >> cbits) == tag) {
                    atomicAdd(slot, len);
                    return;
                } else {
                    break;  // another key holds the bucket's word
                }
            }
            if (!(w >> 31)) atomicOr(slot, 0x80000000u);
            ovf_insert(h, len);
        };
        auto insert = [&](uint32_t key, uint32_t len) {
            const uint32_t k = fmix32(key ^ hseed);
            if (DM) {
                dm_insert(k, len, false);
                return;
            }
            const unsigned long long add = (unsigned long long)len << 32;
            uint32_t sl, stp;
            hj_probe_seq(k, sl, stp);
            for (uint32_t t = 0; t < HJ_SLOTS; ++t) {
                unsigned long long w = *static_cast<volatile unsigned long long*>(&s_ht[sl]);
                if (w == 0ull) {
                    w = atomicCAS(&s_ht[sl], 0ull, add | k);
                    if (w == 0ull) {
                        if (atomicAdd(&s_fill, 1u) + 1 > HJ_MAX_FILL) s_abort = 1;
                        return;
                    }
                }
                if ((uint32_t)w == k) {
                    atomicAdd(&s_ht[sl], add);
                    return;
                }
                sl = (sl + stp) & (HJ_SLOTS - 1);
            }
        };
        // run heads of a 32-key step: (key, run length) for the lanes that start a run
        auto runs = [&](uint32_t nv, uint32_t k, uint32_t& len) {
            const uint32_t prev = __shfl_up_sync(FULL_MASK, k, 1);
            const bool head = lane < nv && (lane == 0 || k != prev);
            const unsigned hm = __ballot_sync(FULL_MASK, head);
            // the next head above this lane (none: __ffs gives 0, and the run ends at nv)
            const unsigned above = hm & (0xfffffffeu << lane);
            len = min((uint32_t)__ffs(above) - 1u, nv) - lane;
            return head;
        };
        const uint32_t nseg = s_nseg;
        for (uint32_t sg = 0; sg < nseg; ++sg) {
            const uint32_t kofs = s_seg_a[sg], nk = s_seg_n[sg];
            for (uint32_t base = warp * 32; base < nk; base += 2 * nwarps * 32) {
                if (*static_cast<volatile uint32_t*>(&s_abort)) break;
                const uint32_t base2 = base + nwarps * 32;
                const uint32_t nv1 = min(32u, nk - base);
                const uint32_t nv2 = base2 < nk ? min(32u, nk - base2) : 0u;
                const uint32_t ka = lane < nv1 ? s_keys[kofs + base + lane] : 0u;
                const uint32_t kb = lane < nv2 ? s_keys[kofs + base2 + lane] : 0u;
                uint32_t la, lb;
                const bool ha = runs(nv1, ka, la);
                const bool hb = runs(nv2, kb, lb);
                if (ha) insert(ka, la);
                if (hb) insert(kb, lb);
            }
        }
        if (hot && warp < s_nlong) {  // a long bucket's distinct keys with their counts
            const uint32_t l = s_long_l[warp];
            const uint32_t n = __ldg(S.len + l);
            const uint32_t* sk = static_cast<const uint32_t*>(S.keys) + (size_t)l * SUM_SLOTS;
            for (uint32_t e = lane; e < n; e += 32) {
                const uint32_t key = __ldg(sk + e), c = __ldg(S.cnt + (size_t)l * SUM_SLOTS + e);
                if (DM) dm_insert(fmix32(key ^ hseed), c, true);
                else insert(key, c);
            }
        }
        __syncthreads();
        const bool abort = s_abort != 0;
        __syncthreads();  // every thread has read this item's shared state
        if (threadIdx.x == 0) {
            if (abort) {
                fb_list[atomicAdd(fb_n, 1u)] = item;
                atomicAdd(tries + 1, 1u);
            }
            // the keys are counted: the next item's copy overlaps this item's queries
            claim();
            s_fill = 0;
            s_abort = 0;
        }
        if (!abort) {
            // answer the bin's queries: one lookup each; the next HJ_QUNROLL query
            // loads per thread are in flight while the current ones are answered
            for (uint32_t g0 = q0; g0 < q1; g0 += blockDim.x * HJ_QUNROLL) {
                uint32_t kn[HJ_QUNROLL];
#pragma unroll
                for (int u = 0; u < HJ_QUNROLL; ++u) {
                    const uint32_t i = g0 + (HJ_QUNROLL + u) * blockDim.x + threadIdx.x;
                    kn[u] = i < q1 ? __ldg(qs + i) : 0u;
                }
#pragma unroll
                for (int u = 0; u < HJ_QUNROLL; ++u) {
                    const uint32_t i = g0 + u * blockDim.x + threadIdx.x;
                    if (i < q1) {
                        // the query's hash (grouped 32-bit queries already are hashes)
                        const uint32_t qk = qhashed ? kq[u] : fmix32(kq[u] ^ hseed);
                        uint32_t sl, stp, cnt = 0;
                        if (DM) {
                            const uint32_t w = s_tab[qk & (BIN_BUCKETS - 1)];
                            if (((w & 0x7fffffffu) >> cbits) == (qk >> lb)) cnt = w & cmask;
                            if (cnt == 0u && (w >> 31)) {
                                hj_ovf_seq(qk, sl, stp);
                                for (uint32_t t = 0; t < HJ_OVF; ++t) {
                                    const unsigned long long x = s_ovf[sl];
                                    if (x == 0ull) break;
                                    if ((uint32_t)x == qk) {
                                        cnt = (uint32_t)(x >> 32);
                                        break;
                                    }
                                    sl = (sl + stp) & (HJ_OVF - 1);
                                }
                            }
                        } else {
                            hj_probe_seq(qk, sl, stp);
                            for (uint32_t t = 0; t < HJ_SLOTS; ++t) {
                                const unsigned long long w = s_ht[sl];
                                if (w == 0ull) break;
                                if ((uint32_t)w == qk) {
                                    cnt = (uint32_t)(w >> 32);
                                    break;
                                }
                                sl = (sl + stp) & (HJ_SLOTS - 1);
                            }
                        }
                        if (OUT == OUT_U32) static_cast<uint32_t*>(counts)[i] = cnt;
                        acc += cnt;
                    }
                }
#pragma unroll
                for (int u = 0; u < HJ_QUNROLL; ++u) kq[u] = kn[u];
            }
        }
        __syncthreads();  // the table's last reader is done
        for (uint32_t t = threadIdx.x; t < HJ_TABLE_BYTES / 16; t += blockDim.x)
            reinterpret_cast<uint4*>(smem)[t] = make_uint4(0, 0, 0, 0);
        __syncthreads();
    }
    if (failed) {
        if (threadIdx.x == 0) atomicOr(err, DEVERR_TIMEOUT);
        return;
    }
    if (TOTAL) {
        const uint64_t sum = block_sum(acc);
        if (threadIdx.x == 0 && sum) atomicAdd(reinterpret_cast<unsigned long long*>(total), (unsigned long long)sum);
    }
}

template <typename K, int OUT, bool TOTAL>
cudaError_t run_probe_bins(const Table& t, const GroupedQueries& g, void* counts, uint64_t* total,
                           const LongList& L, uint32_t* ctrs, uint32_t* fb_list, cudaStream_t s) {
    const K* keys = static_cast<const K*>(t.keys);
    const K* qs = static_cast<const K*>(g.q_grouped);
    // ctrs (zeroed): [0] hash-join work counter, [1] k_probe_bins work counter,
    // [2] fallback list length, [3..4] bins tried / given up by the hash join
    const uint32_t* list = nullptr;
    if constexpr (sizeof(K) == 4) {
        // the bucket-indexed table when B = 2^lb, lb >= 16
        uint32_t lb = 0;
        while (lb < 63 && (1ull << lb) < t.B) ++lb;
        const bool dm = t.H.mode == MODE_POW2 && (1ull << lb) == t.B && lb >= 16 && lb <= 31;
        auto kern = dm ? k_probe_hash<OUT, TOTAL, true> : k_probe_hash<OUT, TOTAL, false>;
        const size_t smem = (size_t)HJ_TABLE_BYTES + HJ_KEY_BYTES;
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        int per_sm = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, HJ_THREADS, smem) != cudaSuccess || per_sm < 1)
            per_sm = 1;
        launch_begin("probe_hash", s);
        kern<<<num_sms() * per_sm, HJ_THREADS, smem, s>>>(qs, g.bin_start, g.items, keys, t.offsets, t.B, (uint32_t)t.n,
                                                          counts, total, ctrs, fb_list, ctrs + 2, ctrs + 3, t.err, t.sum,
                                                          (uint32_t)t.H.seed, dm ? lb : 16u);
        launch_end("probe_hash", s);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        list = fb_list;
    }
    {
        auto kern = k_probe_bins<K, OUT, TOTAL>;
        const size_t smem = BIN_BUFFERS * (size_t)BIN_BUF_BYTES;
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        int per_sm = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, BIN_PROBE_THREADS, smem) != cudaSuccess ||
            per_sm < 1)
            per_sm = 1;
        launch_begin("probe", s);
        kern<<<num_sms() * per_sm, BIN_PROBE_THREADS, smem, s>>>(qs, g.bin_start, g.items, keys, t.offsets, t.H,
                                                                 (uint32_t)t.n, counts, total, sink_of(L), ctrs + 1, t.err,
                                                                 sorted_limit(t), t.sum, list, list ? ctrs + 2 : nullptr);
        launch_end("probe", s);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    cudaError_t e = launch_long_prep<K, true>(t, qs, L, s);
    if (e != cudaSuccess) return e;
    auto kern = k_long<K, OUT, TOTAL, false>;
    launch_begin("long", s);
    kern<<<persistent_grid(kern), PROBE_THREADS, 0, s>>>(qs, keys, t.values, t.offsets, t.H, (uint32_t)t.n, L, counts,
                                                       total, nullptr, nullptr);
    launch_end("long", s);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return launch_long_copy<OUT>(L, counts, s);
}

// Counts of queries already grouped by the table's bins (see group_queries).
template <typename K>
cudaError_t count_grouped(const Table& t, const GroupedQueries& g, uint64_t q, uint32_t* counts, uint64_t* total,
                          cudaStream_t s) {
    void* mem = nullptr;
    LongList L{};
    const uint32_t cap = (uint32_t)(q < COUNT_LONG_CAP ? q : COUNT_LONG_CAP);
    cudaError_t e = alloc_list(cap, false, s, &mem, &L);
    if (e != cudaSuccess) return e;
    L.qunhash = g.items.qunhash;
    void* cmem = nullptr;
    const size_t cbytes = ((q + 4) * 4 + 255) & ~size_t(255);
    // the hash join's fallback list: at most one entry per work item
    const size_t fb_bytes = ((size_t)g.nbins + q / g.items.huge_chunk + 1024) * 4;
    e = dev_alloc(&cmem, 256 + fb_bytes + (counts ? 2 * cbytes : 0), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(cmem, 0, 256, s);
    if (e == cudaSuccess) {
        uint32_t* ctrs = static_cast<uint32_t*>(cmem);
        uint32_t* fb_list = reinterpret_cast<uint32_t*>(static_cast<char*>(cmem) + 256);
        uint32_t* cs = counts ? reinterpret_cast<uint32_t*>(static_cast<char*>(cmem) + 256 + fb_bytes) : nullptr;
        uint32_t* tmp = counts ? cs + cbytes / 4 : nullptr;
        if (counts && total) e = run_probe_bins<K, OUT_U32, true>(t, g, cs, total, L, ctrs, fb_list, s);
        else if (counts) e = run_probe_bins<K, OUT_U32, false>(t, g, cs, nullptr, L, ctrs, fb_list, s);
        else e = run_probe_bins<K, OUT_NONE, true>(t, g, nullptr, total, L, ctrs, fb_list, s);
        if (e == cudaSuccess && counts) e = ungroup_counts(t, &g, cs, tmp, counts, s);
    }
    if (cmem) dev_free(cmem, s);
    dev_free(mem, s);
    return e;
}

// Counts by walking each query's bucket where it lies in HBM (or L2).
template <typename K>
cudaError_t count_direct(const Table& t, const K* qs, uint64_t q, uint32_t* counts, uint64_t* total,
                         cudaStream_t s) {
    void* mem = nullptr;
    LongList L{};
    const uint32_t cap = (uint32_t)(q < COUNT_LONG_CAP ? q : COUNT_LONG_CAP);
    cudaError_t e = alloc_list(cap, false, s, &mem, &L);
    if (e != cudaSuccess) return e;
    if (counts && total) e = run_probe<K, OUT_U32, true, false>(t, qs, q, counts, total, L, nullptr, nullptr, s);
    else if (counts) e = run_probe<K, OUT_U32, false, false>(t, qs, q, counts, nullptr, L, nullptr, nullptr, s);
    else e = run_probe<K, OUT_NONE, true, false>(t, qs, q, nullptr, total, L, nullptr, nullptr, s);
    dev_free(mem, s);
    return e;
}

template <typename K>
cudaError_t count_impl(const Table& t, const K* qs, uint64_t q, uint32_t* counts, uint64_t* total, cudaStream_t s) {
    // Large query sets against a table larger than L2: build the query-side
    // grouping of the paper's query method (Sec. 3.3: queries bucketed like the
    // table, each group answered against its own slice of the table), probe
    // group by group while the slice sits in shared memory, then put counts
    // back in slot order.
    if (probe_grouping_pays(t, q)) {
        GroupedQueries g;
        cudaError_t e = group_queries(t, qs, q, &g, s);
        if (e == cudaSuccess) e = count_grouped<K>(t, g, q, counts, total, s);
        group_release(&g, s);
        return e;
    }
    return count_direct<K>(t, qs, q, counts, total, s);
}

__global__ void k_merge_err(const uint32_t* __restrict__ from, uint32_t* to) {
    if (*from) atomicOr(to, *from);
}

// counts[slot[j]] = src[j]: per-slot counts from counts in HG(Q) order.
__global__ void __launch_bounds__(256) k_scatter_counts(const uint32_t* __restrict__ src,
                                                        const uint32_t* __restrict__ slot, uint64_t q,
                                                        uint32_t* __restrict__ dst) {
    for (uint64_t j = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; j < q; j += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t sl = slot[j];
        if (sl < q) dst[sl] = src[j];
    }
}

// The paper's query form (Sec. 3.3): build HG(Q) over the queries with the
// table's bucket count and seed, each query carrying its slot as its value;
// then intersect bucket i of HG(A) with bucket i of HG(Q) for every i -- here
// by walking, for each query of HG(Q) in bucket order, its bucket of the
// table, so the table is read in bucket order -- and finally put the counts
// back in slot order.
template <typename K>
cudaError_t intersect_impl(const Table& t, const K* qs, uint64_t q, uint32_t* counts, uint64_t* total,
                           cudaStream_t s) {
    Table qt;
    qt.key_bytes = t.key_bytes;
    qt.has_values = 1;
    qt.flags = HG_INDEX_VALUES;
    qt.device = t.device;
    qt.n = q;
    qt.B = t.B;
    qt.seed = t.seed;
    qt.H = t.H;
    qt.err = t.err;
    void* mem = nullptr;
    LongList L{};
    uint32_t* tmp = nullptr;
    cudaError_t e = dev_alloc(reinterpret_cast<void**>(&qt.offsets), (qt.B + 1) * sizeof(uint32_t) + 16, s);
    if (e == cudaSuccess) e = dev_alloc(&qt.keys, q * sizeof(K) + 16, s);
    if (e == cudaSuccess) e = dev_alloc(reinterpret_cast<void**>(&qt.values), q * 4, s);
    if (e == cudaSuccess && counts) e = dev_alloc(reinterpret_cast<void**>(&tmp), q * 4 + 16, s);
    if (e == cudaSuccess) {
        const uint32_t cap = (uint32_t)(q < COUNT_LONG_CAP ? q : COUNT_LONG_CAP);
        e = alloc_list(cap, false, s, &mem, &L);
    }
    if (e == cudaSuccess) e = build_table(qt, qs, nullptr, s);
    const K* grouped = static_cast<const K*>(qt.keys);
    if (e == cudaSuccess) {
        if (counts && total) e = run_probe<K, OUT_U32, true, false>(t, grouped, q, tmp, total, L, nullptr, nullptr, s);
        else if (counts) e = run_probe<K, OUT_U32, false, false>(t, grouped, q, tmp, nullptr, L, nullptr, nullptr, s);
        else e = run_probe<K, OUT_NONE, true, false>(t, grouped, q, nullptr, total, L, nullptr, nullptr, s);
    }
    if (e == cudaSuccess && counts) {
        launch_begin("scatter_counts", s);
        k_scatter_counts<<<num_sms() * 8, 256, 0, s>>>(tmp, qt.values, q, counts);
        launch_end("scatter_counts", s);
        e = cudaGetLastError();
    }
    if (mem) dev_free(mem, s);
    if (tmp) dev_free(tmp, s);
    if (qt.values) dev_free(qt.values, s);
    if (qt.keys) dev_free(qt.keys, s);
    if (qt.offsets) dev_free(qt.offsets, s);
    return e;
}

}  // namespace

cudaError_t count_by_intersection(const Table& t, const void* d_q, uint64_t q, uint32_t* counts, uint64_t* total,
                                  cudaStream_t s) {
    if (total) {
        cudaError_t e = cudaMemsetAsync(total, 0, sizeof(uint64_t), s);
        if (e != cudaSuccess) return e;
    }
    if (q == 0) return cudaSuccess;
    if (t.key_bytes == 4) return intersect_impl<uint32_t>(t, static_cast<const uint32_t*>(d_q), q, counts, total, s);
    return intersect_impl<uint64_t>(t, static_cast<const uint64_t*>(d_q), q, counts, total, s);
}

cudaError_t plan_queries(const Table& t, const void* d_q, uint64_t q, QueryPlan* p, cudaStream_t s) {
    p->queries = d_q;
    p->q = q;
    p->B = t.B;
    p->seed = t.seed;
    p->n = t.n;
    p->key_bytes = t.key_bytes;
    p->grouped = q > 0 && probe_grouping_pays(t, q);
    cudaError_t e = dev_alloc(reinterpret_cast<void**>(&p->err), 16, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(p->err, 0, 16, s);
    if (e != cudaSuccess || !p->grouped) return e;
    p->g.err = p->err;
    return group_queries(t, d_q, q, &p->g, s);
}

cudaError_t count_planned(const Table& t, const QueryPlan& p, uint32_t* counts, uint64_t* total, cudaStream_t s) {
    if (total) {
        cudaError_t e = cudaMemsetAsync(total, 0, sizeof(uint64_t), s);
        if (e != cudaSuccess) return e;
    }
    if (p.q == 0) return cudaSuccess;
    cudaError_t e;
    if (!p.grouped) {
        e = t.key_bytes == 4 ? count_direct<uint32_t>(t, static_cast<const uint32_t*>(p.queries), p.q, counts, total, s)
                             : count_direct<uint64_t>(t, static_cast<const uint64_t*>(p.queries), p.q, counts, total, s);
    } else {
        e = t.key_bytes == 4 ? count_grouped<uint32_t>(t, p.g, p.q, counts, total, s)
                             : count_grouped<uint64_t>(t, p.g, p.q, counts, total, s);
    }
    if (e == cudaSuccess) {  // the plan's kernel-side errors become the table's
        k_merge_err<<<1, 1, 0, s>>>(p.err, t.err);
        e = cudaGetLastError();
    }
    return e;
}

void plan_release(QueryPlan* p, cudaStream_t s) {
    group_release(&p->g, s);
    if (p->err) dev_free(p->err, s);
    p->err = nullptr;
}

cudaError_t probe_count(const Table& t, const void* d_q, uint64_t q, uint32_t* counts, uint64_t* total,
                        cudaStream_t s) {
    if (total) {
        cudaError_t e = cudaMemsetAsync(total, 0, sizeof(uint64_t), s);
        if (e != cudaSuccess) return e;
    }
    if (q == 0) return cudaSuccess;
    if (t.key_bytes == 4) return count_impl<uint32_t>(t, static_cast<const uint32_t*>(d_q), q, counts, total, s);
    return count_impl<uint64_t>(t, static_cast<const uint64_t*>(d_q), q, counts, total, s);
}

// Gather keeps its work list between the two phases: phase 1 (counts into
// out_offsets, then the scan) and phase 2 (the value writes) must agree on
// which slots are long, so the list is sized for every slot and never overflows.

cudaError_t gather_offsets(const Table& t, const void* d_q, uint64_t q, uint64_t* out_offsets, GatherCtx* ctx,
                           cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(out_offsets + q, 0, sizeof(uint64_t), s);
    if (e != cudaSuccess || q == 0) return e;
    LongList L{};
    e = alloc_list((uint32_t)q, true, s, &ctx->scratch, &L);
    if (e != cudaSuccess) return e;
    ctx->slots = q;
    if (t.key_bytes == 4)
        e = run_probe<uint32_t, OUT_U64, false, false>(t, static_cast<const uint32_t*>(d_q), q, out_offsets, nullptr,
                                                       L, nullptr, nullptr, s);
    else
        e = run_probe<uint64_t, OUT_U64, false, false>(t, static_cast<const uint64_t*>(d_q), q, out_offsets, nullptr,
                                                       L, nullptr, nullptr, s);
    if (e != cudaSuccess) return e;
    return scan_exclusive_u64(out_offsets, q + 1, t.err, s);
}

cudaError_t gather_values(const Table& t, const void* d_q, uint64_t q, const uint64_t* out_offsets,
                          uint32_t* out_values, GatherCtx* ctx, cudaStream_t s) {
    if (q == 0) return cudaSuccess;
    // The list view over the same scratch (layout fixed by map_list).
    LongList L{};
    map_list(ctx->scratch, (uint32_t)q, true, &L);
    if (t.key_bytes == 4)
        return run_probe<uint32_t, OUT_NONE, false, true>(t, static_cast<const uint32_t*>(d_q), q, nullptr, nullptr, L,
                                                          out_offsets, out_values, s);
    return run_probe<uint64_t, OUT_NONE, false, true>(t, static_cast<const uint64_t*>(d_q), q, nullptr, nullptr, L,
                                                      out_offsets, out_values, s);
}

void gather_release(GatherCtx* ctx, cudaStream_t s) {
    if (ctx->scratch) dev_free(ctx->scratch, s);
    ctx->scratch = nullptr;
}

}  // namespace hg

namespace hg {

cudaError_t probe_stats(const Table& t, const void* d_q, uint64_t q, uint64_t* stats, cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(stats, 0, 6 * sizeof(uint64_t), s);
    if (e != cudaSuccess) return e;
    const uint64_t lim = WALK_WARP;
    e = cudaMemcpyAsync(stats + 3, &lim, sizeof(lim), cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess || q == 0) return e;
    const unsigned g = (unsigned)(num_sms() * 4);
    launch_begin("walk_stats", s);
    if (t.key_bytes == 4)
        k_walk_stats<uint32_t><<<g, PROBE_THREADS, 0, s>>>(static_cast<const uint32_t*>(d_q), q, t.offsets, t.H, stats);
    else
        k_walk_stats<uint64_t><<<g, PROBE_THREADS, 0, s>>>(static_cast<const uint64_t*>(d_q), q, t.offsets, t.H, stats);
    launch_end("walk_stats", s);
    return cudaGetLastError();
}

}  // namespace hg
