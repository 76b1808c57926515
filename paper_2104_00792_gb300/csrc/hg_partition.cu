// Partitioned HashGraph build: the "efficient HashGraph" of Sec. 3.2, where
// keys are first grouped by ranges of hashed values ("bins") so that the
// per-bucket counting and placing of Algorithm 1 happen in on-chip shared
// memory instead of as random atomics into an offsets array far larger than
// the cache.
//
// Stages (bin = bucket >> BIN_SHIFT, so a bin is a range of 8192 buckets):
//   1. k_part_count  bin histogram, plus the first pass's digit counts for
//                    every CHUNK-key chunk of the input.
//   2. k_part_plan   one CTA: exclusive scan of the bin counts (bin_start),
//                    the second pass's chunks, the huge bins, the work list.
//   3. MSD partition by bin in one or two passes of radix <= 128, each a
//      reduce-then-scan: per-chunk digit counts -> k_chunk_scan (where each
//      chunk's run of each digit starts) -> the downsweep, where one CTA walks
//      its chunk tile by tile, ranks keys per digit in shared memory, stages
//      them in digit order and writes each digit's run contiguously.  No CTA
//      ever waits for another.  32-bit keys move as their hashes (k_pass32;
//      fmix32 is a bijection, so later stages read buckets straight from the
//      words and recover keys with fmix32_inv); 64-bit keys move as keys
//      (k_pass_down).
//   4. Per-bin counting sort by bucket (Algorithm 1 inside one bin):
//      32-bit keys without values: bins of at most SB_CAP keys by k_bin_small
//      (one bulk copy per bin into shared memory, keys held in registers),
//      larger bins cut into SB_CAP-key chunks: k_big_count (chunk bucket
//      histograms) -> k_huge_scan (offsets and per-bucket cursors) ->
//      k_big_place (one global atomic per nonempty bucket per chunk).
//      Otherwise k_bin_local (staged in shared memory; when a bin does not
//      fit, its largest buckets go straight to global memory), with bins
//      above HUGE_T_BUILD keys split over many CTAs: k_huge_count ->
//      k_huge_scan -> chunk placement through per-bucket cursors.
// The result equals the direct build's (offsets bit-exact; the order inside
// a bucket differs, which Algorithm 1 leaves free).
#include <cstdint>
#include <type_traits>

#include "hg_device.cuh"

namespace hg {

namespace {

constexpr int BIN_SHIFT = 13;
constexpr uint32_t BPB = 1u << BIN_SHIFT;   // buckets per bin
constexpr uint32_t RADIX = 128;             // digits per partition pass
constexpr uint32_t MAX_BINS = RADIX * RADIX;
constexpr int PASS_THREADS = 512;
constexpr int LOCAL_THREADS = 512;
constexpr uint32_t CHUNK = 1u << 16;        // keys per reduce-then-scan chunk
constexpr uint32_t TILES_PER_CHUNK = CHUNK / 2048;  // upper bound for either key width
constexpr uint32_t MAX_HOT = 256;           // buckets per bin that may bypass the staging buffer
constexpr size_t LOCAL_STAGE_BYTES = 72 * 1024;
constexpr uint32_t HUGE_T = 1u << 18;       // query bins with more queries are cut into work items
constexpr uint32_t HUGE_T_BUILD = 1u << 16; // build bins with more keys are split over many CTAs
constexpr uint32_t HUGE_CHUNK = 1u << 16;   // keys per CTA work item of a huge bin
constexpr uint32_t MAX_HUGE = 512;          // huge bins with their own counter/cursor slice
constexpr int NTHR = 5;                     // candidate hot-bucket thresholds

template <typename K>
struct PassCfg {
    static constexpr int IPT = sizeof(K) == 4 ? 8 : 4;  // elements per thread per tile
    static constexpr int TILE = PASS_THREADS * IPT;
};

// Rank-returning shared-memory increment.  A warp whose active lanes all hit
// one counter (a heavily duplicated key) takes a single atomic; the check is a
// shuffle and a vote, far cheaper than the MATCH instruction.
__device__ __forceinline__ uint32_t smem_inc(uint32_t* c, uint32_t idx, unsigned mask) {
    const unsigned lane = lane_id();
    const int leader = __ffs(mask) - 1;
    const uint32_t first = __shfl_sync(mask, idx, leader);
    if (__all_sync(mask, idx == first)) {
        uint32_t base = 0;
        if ((int)lane == leader) base = atomicAdd(c + idx, (uint32_t)__popc(mask));
        base = __shfl_sync(mask, base, leader);
        return base + __popc(mask & lanemask_lt());
    }
    return atomicAdd(c + idx, 1u);
}

__device__ __forceinline__ void smem_add1(uint32_t* c, uint32_t idx, unsigned mask) {
    const unsigned lane = lane_id();
    const int leader = __ffs(mask) - 1;
    const uint32_t first = __shfl_sync(mask, idx, leader);
    if (__all_sync(mask, idx == first)) {
        if ((int)lane == leader) atomicAdd(c + idx, (uint32_t)__popc(mask));
    } else {
        atomicAdd(c + idx, 1u);
    }
}

template <typename K>
__device__ __forceinline__ uint32_t bin_of(K k, const Hasher& H) {
    return bucket_of(k, H) >> BIN_SHIFT;
}

// Calls f(i, key, value, mask) for every i in [s0, s1): the 16-byte aligned body
// U vectors per thread at a time, the few elements around it by warp 0.
// `mask` = lanes of the warp calling f together.  HV: also load in_v[i].
// KEEP: the keys are read again soon (an L2 evict_last hint on their loads).
template <typename K, bool HV, int U = 2, bool KEEP = false, typename F>
__device__ __forceinline__ void block_for_range(const K* __restrict__ in, const uint32_t* __restrict__ in_v,
                                                uint64_t s0, uint64_t s1, F&& f) {
    constexpr int VEC = KeyVec<K>::N;
    const unsigned lane = lane_id();
    const uint32_t nt = blockDim.x;
    const uint64_t mis = (reinterpret_cast<uintptr_t>(in + s0) & 15) / sizeof(K);
    const uint64_t hend = mis ? min(s1, s0 + (VEC - mis)) : s0;
    const uint64_t nv = s1 > hend ? (s1 - hend) / VEC : 0;
    const uint64_t tail0 = hend + nv * VEC;
    for (uint64_t g0 = (threadIdx.x & ~31u) * U; g0 < nv; g0 += (uint64_t)U * nt) {
        KeyVec<K> kv[U];
        uint32_t vv[U][VEC];
        bool ok[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const uint64_t g = g0 + u * 32 + lane;
            ok[u] = g < nv;
            if (ok[u]) {
                if (KEEP) *reinterpret_cast<uint4*>(&kv[u]) = ld_keep16(in + hend + g * VEC);
                else kv[u] = load_keys16(in + hend + g * VEC);
                if (HV) {
                    if (VEC == 4) {
                        const uint4 x = ld_stream16(in_v + hend + g * VEC);
                        vv[u][0] = x.x; vv[u][1] = x.y; vv[u][2 % VEC] = x.z; vv[u][3 % VEC] = x.w;
                    } else {
                        const uint2 x = *reinterpret_cast<const uint2*>(in_v + hend + g * VEC);
                        vv[u][0] = x.x; vv[u][1 % VEC] = x.y;
                    }
                }
            }
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const unsigned m = __ballot_sync(FULL_MASK, ok[u]);
            if (ok[u]) {
                const uint64_t e = hend + (g0 + u * 32 + lane) * VEC;
#pragma unroll
                for (int j = 0; j < VEC; ++j) f(e + j, kv[u].k[j], HV ? vv[u][j] : 0u, m);
            }
        }
    }
    if (threadIdx.x < 32) {
        const uint64_t nh = hend - s0, nrem = nh + (s1 - tail0);  // < 2 * VEC
        const bool ok = lane < nrem;
        const unsigned m = __ballot_sync(FULL_MASK, ok);
        if (ok) {
            const uint64_t i = lane < nh ? s0 + lane : tail0 + (lane - nh);
            f(i, in[i], HV ? in_v[i] : 0u, m);
        }
    }
}


// ------------------------------------------------------------- chunking --
struct Plan {
    uint32_t chunks_b;     // chunks of the second pass
    uint32_t n_huge;       // bins split over many CTAs (at most the plan's max_huge)
    uint32_t huge_chunks;  // their huge_chunk-key work items
    uint32_t n_work;       // bins handled whole by one CTA
    uint32_t n_big;        // the first n_big of them hold more than the plan's big_t keys
    uint32_t huge_chunk;   // keys per work item of a huge bin
};

// Chunk c of a pass: keys [lo, hi) of segment `seg`.  Single-segment passes
// cut [0, n) into CHUNK-key pieces; segmented passes cut each segment
// [bin_start[s * P2], bin_start[(s + 1) * P2]) separately (ChunkMap).

__device__ __forceinline__ void chunk_range(const ChunkMap& cm, uint32_t c, uint32_t& seg, uint32_t& first,
                                            uint64_t& lo, uint64_t& hi) {
    if (!cm.segmented) {
        seg = 0;
        first = 0;
        lo = (uint64_t)c * CHUNK;
        hi = min(cm.n, lo + CHUNK);
        return;
    }
    uint32_t a = 0, b = cm.nseg;  // last segment with seg_chunk_start[s] <= c
    while (b - a > 1) {
        const uint32_t mid = (a + b) >> 1;
        if (cm.seg_chunk_start[mid] <= c) a = mid; else b = mid;
    }
    seg = a;
    first = cm.seg_chunk_start[a];
    const uint64_t s_lo = cm.bin_start[a * cm.P2];
    const uint64_t s_hi = cm.bin_start[min((a + 1) * cm.P2, cm.P)];
    lo = s_lo + (uint64_t)(c - first) * CHUNK;
    hi = min(s_hi, lo + CHUNK);
}

// ---------------------------------------------------------------- count --
// Bin histogram (shared memory per CTA, flushed once; BINS only) and, per
// chunk of the input, the counts of the first pass's digit (bin >> dig_shift);
// digit totals are also added into digit_total when it is given.
template <typename K, bool BINS>
__global__ void __launch_bounds__(PASS_THREADS)
k_part_count(const K* __restrict__ keys, uint64_t n, Hasher H, uint32_t P, uint32_t dig_shift, uint32_t R,
             uint32_t nch, uint32_t* bin_count, uint32_t* chunk_cnt, uint32_t* digit_total) {
    extern __shared__ uint32_t s_hist[];
    __shared__ uint32_t s_dig[RADIX];
    if (BINS)
        for (uint32_t i = threadIdx.x; i < P; i += blockDim.x) s_hist[i] = 0;
    for (uint32_t c = blockIdx.x; c < nch; c += gridDim.x) {
        for (uint32_t i = threadIdx.x; i < RADIX; i += blockDim.x) s_dig[i] = 0;
        __syncthreads();
        const uint64_t lo = (uint64_t)c * CHUNK, hi = min(n, lo + CHUNK);
        block_for_range<K, false, 4>(keys, nullptr, lo, hi, [&](uint64_t, K k, uint32_t, unsigned) {
            const uint32_t b = bin_of(k, H);
            if (BINS) atomicAdd(s_hist + b, 1u);
            atomicAdd(s_dig + ((b >> dig_shift) & (RADIX - 1)), 1u);
        });
        __syncthreads();
        for (uint32_t d = threadIdx.x; d < R; d += blockDim.x) {
            chunk_cnt[(uint64_t)c * RADIX + d] = s_dig[d];
            if (digit_total && s_dig[d]) atomicAdd(digit_total + d, s_dig[d]);
        }
    }
    if (BINS) {
        __syncthreads();
        for (uint32_t i = threadIdx.x; i < P; i += blockDim.x)
            if (s_hist[i]) atomicAdd(bin_count + i, s_hist[i]);
    }
}

// Second-pass chunk counts: digit = bin & (RADIX - 1) inside each chunk's segment.
template <typename K, bool HIN = false>
__global__ void __launch_bounds__(PASS_THREADS)
k_chunk_count(const K* __restrict__ in, Hasher H, ChunkMap cm, const Plan* __restrict__ plan, uint32_t* chunk_cnt) {
    __shared__ uint32_t s_dig[RADIX];
    const uint32_t c = blockIdx.x;
    if (c >= plan->chunks_b) return;
    uint32_t seg, first;
    uint64_t lo, hi;
    chunk_range(cm, c, seg, first, lo, hi);
    for (uint32_t i = threadIdx.x; i < RADIX; i += blockDim.x) s_dig[i] = 0;
    __syncthreads();
    block_for_range<K, false, 4>(in, nullptr, lo, hi, [&](uint64_t, K k, uint32_t, unsigned) {
        const uint32_t bin = HIN ? bucket_of_hash((uint32_t)k, H) >> BIN_SHIFT : bin_of(k, H);
        atomicAdd(s_dig + (bin & (RADIX - 1)), 1u);
    });
    __syncthreads();
    for (uint32_t d = threadIdx.x; d < RADIX; d += blockDim.x) chunk_cnt[(uint64_t)c * RADIX + d] = s_dig[d];
}

// ----------------------------------------------------------------- plan --
template <typename T>
__device__ __forceinline__ T block_exclusive_scan(T v, T* s_warp, T* total) {
    const unsigned lane = lane_id();
    const int w = threadIdx.x >> 5;
    const int nw = blockDim.x >> 5;
    const T incl = warp_inclusive_scan(v);
    if (lane == 31) s_warp[w] = incl;
    __syncthreads();
    if (w == 0) {
        const T x = (int)lane < nw ? s_warp[lane] : (T)0;
        const T xi = warp_inclusive_scan(x);
        if ((int)lane < nw) s_warp[lane] = xi - x;
        if (lane == 31) s_warp[32] = xi;
    }
    __syncthreads();
    const T r = s_warp[w] + incl - v;
    *total = s_warp[32];
    __syncthreads();
    return r;
}

// One CTA.  Writes bin_start[P+1]; seg_chunk_start[P1+1] (chunks of each
// coarse segment in the second pass); offsets[B] = n; the huge bins (more
// than huge_t keys; the first max_huge of them) with the prefix of their
// chunk counts; and the work list of the other bins, bins above big_t keys first.
// Thread t holds the counts of bins [16t, 16t + 16) in registers, so every
// list comes from one block-wide scan of per-thread totals.
constexpr int PLAN_THREADS = 1024;
constexpr int PLAN_PB = MAX_BINS / PLAN_THREADS;  // bins per thread
__global__ void __launch_bounds__(PLAN_THREADS)
k_part_plan(const uint32_t* __restrict__ bin_count, uint32_t P, uint32_t P1, uint32_t P2, uint64_t n,
            uint32_t big_t, uint32_t huge_t, uint32_t huge_chunk, uint32_t max_huge, uint32_t* bin_start,
            uint32_t* seg_chunk_start, uint32_t* work, uint32_t* huge_bin, uint32_t* huge_chunk_start, Plan* plan,
            uint32_t* offsets, uint64_t B) {
    __shared__ uint32_t s_warp[33];
    const uint32_t tid = threadIdx.x, p0 = tid * PLAN_PB;
    uint32_t c[PLAN_PB];
    uint32_t sum = 0, nh_loc = 0;
#pragma unroll
    for (int i = 0; i < PLAN_PB; ++i) {
        c[i] = p0 + i < P ? __ldg(bin_count + p0 + i) : 0u;
        sum += c[i];
        nh_loc += (p0 + i < P && c[i] > huge_t) ? 1u : 0u;
    }
    // bin starts
    uint32_t tot;
    uint32_t run = block_exclusive_scan<uint32_t>(sum, s_warp, &tot);
#pragma unroll
    for (int i = 0; i < PLAN_PB; ++i) {
        if (p0 + i < P) bin_start[p0 + i] = run;
        run += c[i];
    }
    if (tid == 0) {
        bin_start[P] = tot;
        if (offsets) offsets[B] = (uint32_t)n;
    }
    // huge bins in index order (the first max_huge are admitted), their chunks,
    // and the other bins by size
    uint32_t nh_tot;
    const uint32_t hx0 = block_exclusive_scan<uint32_t>(nh_loc, s_warp, &nh_tot);
    uint32_t ch_loc = 0, nb_loc = 0, ns_loc = 0;
    {
        uint32_t hx = hx0;
#pragma unroll
        for (int i = 0; i < PLAN_PB; ++i) {
            const bool in = p0 + i < P;
            const bool huge = in && c[i] > huge_t;
            const bool adm = huge && hx < max_huge;
            hx += huge ? 1u : 0u;
            if (adm) ch_loc += (c[i] + huge_chunk - 1) / huge_chunk;
            if (in && !adm) {
                if (c[i] > big_t) ++nb_loc;
                else ++ns_loc;
            }
        }
    }
    uint32_t ch_tot, nb_tot, ns_tot;
    uint32_t cx = block_exclusive_scan<uint32_t>(ch_loc, s_warp, &ch_tot);
    uint32_t bx = block_exclusive_scan<uint32_t>(nb_loc, s_warp, &nb_tot);
    uint32_t sx = block_exclusive_scan<uint32_t>(ns_loc, s_warp, &ns_tot);
    {
        uint32_t hx = hx0;
#pragma unroll
        for (int i = 0; i < PLAN_PB; ++i) {
            const uint32_t p = p0 + i;
            const bool in = p < P;
            const bool huge = in && c[i] > huge_t;
            const bool adm = huge && hx < max_huge;
            if (adm) {
                huge_bin[hx] = p;
                huge_chunk_start[hx] = cx;
                cx += (c[i] + huge_chunk - 1) / huge_chunk;
            }
            hx += huge ? 1u : 0u;
            if (in && !adm) {
                if (c[i] > big_t) work[bx++] = p;
                else work[nb_tot + sx++] = p;
            }
        }
    }
    const uint32_t n_huge = min(nh_tot, max_huge);
    __syncthreads();  // bin_start is complete
    // second-pass chunks per coarse segment (P1 <= RADIX segments)
    uint32_t t = 0;
    if (tid < P1) {
        const uint32_t lo = bin_start[tid * P2];
        const uint32_t hi = bin_start[min((tid + 1) * P2, P)];
        t = (hi - lo + CHUNK - 1) / CHUNK;
    }
    uint32_t crun;
    const uint32_t sc = block_exclusive_scan<uint32_t>(t, s_warp, &crun);
    if (tid < P1) seg_chunk_start[tid] = sc;
    if (tid == 0) {
        seg_chunk_start[P1] = crun;
        huge_chunk_start[n_huge] = ch_tot;
        plan->chunks_b = crun;
        plan->n_huge = n_huge;
        plan->huge_chunks = ch_tot;
        plan->n_work = nb_tot + ns_tot;
        plan->n_big = nb_tot;
        plan->huge_chunk = huge_chunk;
    }
}

// One CTA of 1024 threads per digit d.  On return cnt[c][d] holds the start of
// digit d's run of chunk c: digit_start(seg(c), d) + the number of keys with
// digit d in earlier chunks of the same segment.  digit_start = bin_start[d *
// dig_mul] for a single-segment pass, bin_start[s * P2 + d] for a segmented
// one.  pref (same shape) receives the plain prefix over all chunks.
__global__ void __launch_bounds__(1024)
k_chunk_scan(uint32_t* cnt, uint32_t* pref, ChunkMap cm, uint32_t nch_host, const Plan* __restrict__ plan, uint32_t R,
             uint32_t dig_mul, const uint32_t* __restrict__ digit_total) {
    __shared__ uint32_t s_warp[33];
    __shared__ uint32_t s_scs[RADIX + 1];  // segmented: the segments' first chunks
    const uint32_t nch = cm.segmented ? plan->chunks_b : nch_host;
    const uint32_t d = blockIdx.x;
    if (cm.segmented)
        for (uint32_t i = threadIdx.x; i <= cm.nseg && i <= RADIX; i += blockDim.x) s_scs[i] = cm.seg_chunk_start[i];
    const uint32_t per = (nch + blockDim.x - 1) / blockDim.x;
    const uint32_t c0 = min(nch, threadIdx.x * per), c1 = min(nch, c0 + per);
    uint32_t sum = 0;
    for (uint32_t c = c0; c < c1; ++c) sum += cnt[(uint64_t)c * RADIX + d];
    uint32_t tot;
    uint32_t run = block_exclusive_scan<uint32_t>(sum, s_warp, &tot);
    for (uint32_t c = c0; c < c1; ++c) {
        pref[(uint64_t)c * RADIX + d] = run;
        run += cnt[(uint64_t)c * RADIX + d];
    }
    __syncthreads();
    // subtract the prefix at the segment's first chunk, add the digit's start
    // (a thread's chunks are consecutive: the segment is looked up in shared
    // memory, and the start read again only when the segment changes)
    uint32_t seg = ~0u, first = 0, start = 0, pfirst = 0;
    for (uint32_t c = c0; c < c1; ++c) {
        uint32_t sg = 0;
        if (cm.segmented) {  // last segment with s_scs[s] <= c
            uint32_t lo = 0, hi = min(cm.nseg, RADIX);
            while (hi - lo > 1) {
                const uint32_t mid = (lo + hi) >> 1;
                if (s_scs[mid] <= c) lo = mid; else hi = mid;
            }
            sg = lo;
        }
        if (sg != seg) {
            seg = sg;
            first = cm.segmented ? s_scs[sg] : 0u;
            start = 0;
            if (d < R) {
                if (digit_total) {
                    for (uint32_t q = 0; q < d; ++q) start += digit_total[q];
                } else {
                    const uint32_t bin = cm.segmented ? seg * cm.P2 + d : d * dig_mul;
                    start = cm.bin_start[min(bin, cm.P)];
                }
            }
            pfirst = pref[(uint64_t)first * RADIX + d];
        }
        cnt[(uint64_t)c * RADIX + d] = start + pref[(uint64_t)c * RADIX + d] - pfirst;
    }
}

// ------------------------------------------------------------ downsweep --
// One CTA per chunk: tiles in order; run[d] = where the chunk's next key with
// digit d goes.  Element li of a tile is held by thread (li / 4) % 256, slot
// (li / 1024) * 4 + li % 4, so each thread's four consecutive keys come from one
// 16-byte load when the chunk is aligned.  The next tile's keys are loaded
// while the current one is ranked, staged and written.
// Shared memory: keys[TILE] | payload[TILE] | destination[TILE].
template <typename K, int PM>
__device__ __forceinline__ void load_tile(const K* __restrict__ in, const uint32_t* __restrict__ in_v, uint64_t t0,
                                          uint32_t cnt_tile, bool vec, K (&k)[PassCfg<K>::IPT],
                                          uint32_t (&v)[PassCfg<K>::IPT]) {
    constexpr int IPT = PassCfg<K>::IPT;
    constexpr int G = 16 / sizeof(K);  // keys per 16-byte group
#pragma unroll
    for (int jj = 0; jj < IPT / G; ++jj) {
        const uint32_t li0 = (threadIdx.x + jj * PASS_THREADS) * G;
        if (vec && li0 + G <= cnt_tile) {
            const KeyVec<K> kv = load_keys16(in + t0 + li0);
#pragma unroll
            for (int u = 0; u < G; ++u) k[jj * G + u] = kv.k[u];
        } else {
#pragma unroll
            for (int u = 0; u < G; ++u) k[jj * G + u] = li0 + u < cnt_tile ? in[t0 + li0 + u] : (K)0;
        }
#pragma unroll
        for (int u = 0; u < G; ++u) {
            if (PM == 1) v[jj * G + u] = li0 + u < cnt_tile ? in_v[t0 + li0 + u] : 0u;
            if (PM == 2) v[jj * G + u] = (uint32_t)(t0 + li0 + u);
        }
    }
}

// DR: also record, for the reverse pass, each input element's (rank << 8 |
// digit) in dr_out (input order) and each tile's (loc, base) per digit in
// tile_lb[c * TILES_PER_CHUNK + tile][RADIX].
template <typename K, int PM, bool DR = false>
__global__ void __launch_bounds__(PASS_THREADS, 3)
k_pass_down(const K* __restrict__ in, const uint32_t* __restrict__ in_v, uint64_t n, Hasher H, uint32_t dig_shift,
            uint32_t dig_mask, uint32_t R, ChunkMap cm, uint32_t nch_host, const Plan* __restrict__ plan,
            const uint32_t* __restrict__ chunk_base, K* __restrict__ out, uint32_t* __restrict__ out_v,
            uint32_t* err, uint32_t* __restrict__ dr_out, uint2* __restrict__ tile_lb) {
    constexpr int IPT = PassCfg<K>::IPT;
    constexpr int TILE = PassCfg<K>::TILE;
    constexpr int G = 16 / sizeof(K);
    constexpr bool PACK = sizeof(K) == 4;  // (key, destination) staged as one 8-byte word
    extern __shared__ __align__(16) unsigned char smem[];
    uint2* s_kd = reinterpret_cast<uint2*>(smem);                       // PACK: key, destination
    K* s_keys = reinterpret_cast<K*>(smem);                             // !PACK
    uint32_t* s_dst = reinterpret_cast<uint32_t*>(smem + TILE * sizeof(K));
    uint32_t* s_pay = reinterpret_cast<uint32_t*>(smem + (size_t)TILE * 8 + (PACK ? 0 : (size_t)TILE * 4));
    __shared__ uint32_t s_cnt[RADIX], s_run[RADIX], s_warp[4];
    __shared__ uint2 s_lb[RADIX];  // (offset of the digit's run inside the tile, its destination)

    const uint32_t nch = cm.segmented ? plan->chunks_b : nch_host;
    const uint32_t c = blockIdx.x;
    if (c >= nch) return;
    uint32_t seg, first;
    uint64_t lo, hi;
    chunk_range(cm, c, seg, first, lo, hi);
    const bool vec = (reinterpret_cast<uintptr_t>(in + lo) & 15) == 0;
    // every tile starts G records after a multiple of G, so one check covers the chunk
    const bool dr_vec = DR && (reinterpret_cast<uintptr_t>(dr_out + lo) & (G * 4 - 1)) == 0;
    for (uint32_t d = threadIdx.x; d < RADIX; d += blockDim.x) {
        s_cnt[d] = 0;
        s_run[d] = d < R ? chunk_base[(uint64_t)c * RADIX + d] : 0u;
    }
    __syncthreads();

    K k[IPT];
    uint32_t v[IPT];
    if (lo < hi) load_tile<K, PM>(in, in_v, lo, (uint32_t)min((uint64_t)TILE, hi - lo), vec, k, v);
    const uint32_t nn = (uint32_t)min(n, (uint64_t)0xffffffffu);
    for (uint64_t t0 = lo; t0 < hi; t0 += TILE) {
        const uint32_t cnt_tile = (uint32_t)min((uint64_t)TILE, hi - t0);
        uint32_t dr[IPT];  // rank << 8 | digit
#pragma unroll
        for (int j = 0; j < IPT; ++j) {
            const uint32_t li = (threadIdx.x + (j / G) * PASS_THREADS) * G + (j % G);
            // the digit is masked to the radix, so shared-memory indices stay in
            // bounds whatever the key; a consistent plan never needs the mask
            const uint32_t d = (bin_of(k[j], H) >> dig_shift) & dig_mask & (RADIX - 1);
            dr[j] = li < cnt_tile ? ((atomicAdd(s_cnt + d, 1u) << 8) | d) : 0xffffffffu;
        }
        __syncthreads();
        // digit offsets inside the tile (first 4 warps), and where each run goes
        if (threadIdx.x < RADIX) {
            const uint32_t d = threadIdx.x;
            const uint32_t cd = s_cnt[d];
            const uint32_t incl = warp_inclusive_scan(cd);
            if (lane_id() == 31) s_warp[d >> 5] = incl;
            asm volatile("bar.sync 1, 128;");
            uint32_t wp = 0;
            for (uint32_t w = 0; w < (d >> 5); ++w) wp += s_warp[w];
            s_lb[d] = make_uint2(wp + incl - cd, s_run[d]);
            if (DR) tile_lb[((uint64_t)c * TILES_PER_CHUNK + (t0 - lo) / TILE) * RADIX + d] = s_lb[d];
            s_run[d] += cd;
            s_cnt[d] = 0;
        }
        __syncthreads();
        uint32_t* dr_t = DR ? dr_out + t0 : nullptr;
#pragma unroll
        for (int j = 0; j < IPT; ++j) {
            if (dr[j] != 0xffffffffu) {
                const uint32_t r = dr[j] >> 8;
                const uint2 lb = s_lb[dr[j] & 0xffu];
                const uint32_t pos = lb.x + r;
                const uint32_t dst = lb.y + r;
                if (PACK) {
                    s_kd[pos] = make_uint2((uint32_t)k[j], dst);
                } else {
                    s_keys[pos] = k[j];
                    s_dst[pos] = dst;
                }
                if (PM) s_pay[pos] = v[j];
                if (DR && !(dr_vec && cnt_tile == (uint32_t)TILE))
                    dr_t[(threadIdx.x + (j / G) * PASS_THREADS) * G + (j % G)] = dr[j];
            }
        }
        if (DR && dr_vec && cnt_tile == (uint32_t)TILE) {
            // a full tile with aligned records: each thread's G records per group are
            // consecutive, so they go out in one vector store
#pragma unroll
            for (int jj = 0; jj < IPT / G; ++jj) {
                uint32_t* d = dr_t + (threadIdx.x + jj * PASS_THREADS) * G;
                if constexpr (G == 4)
                    *reinterpret_cast<uint4*>(d) = make_uint4(dr[jj * 4], dr[jj * 4 + 1], dr[jj * 4 + 2], dr[jj * 4 + 3]);
                else
                    *reinterpret_cast<uint2*>(d) = make_uint2(dr[jj * 2], dr[jj * 2 + 1]);
            }
        }
        __syncthreads();
        // prefetch the next tile while this one is written out
        const uint64_t t1 = t0 + TILE;
        if (t1 < hi) load_tile<K, PM>(in, in_v, t1, (uint32_t)min((uint64_t)TILE, hi - t1), vec, k, v);
        for (uint32_t i = threadIdx.x; i < cnt_tile; i += PASS_THREADS) {
            K key;
            uint32_t dst;
            if (PACK) {
                const uint2 kd = s_kd[i];
                key = (K)kd.x;
                dst = kd.y;
            } else {
                key = s_keys[i];
                dst = s_dst[i];
            }
            if (dst < nn) {
                out[dst] = key;
                if (PM) out_v[dst] = s_pay[i];
            } else {
                atomicOr(err, DEVERR_BOUNDS);
            }
        }
        __syncthreads();
    }
}

// ------------------------------------------------- downsweep, 32-bit keys --
// k_pass_down for 32-bit keys, with each key's hash as the word that moves:
// the pass reads keys (HIN = false, hashing each once) or hashes (HIN = true)
// and always writes hashes, so the next pass, the bin build and the grouped
// probes take a key's bucket straight from its word (the key itself is
// fmix32_inv(h) ^ seed).  Because of that the staging keeps only the words:
// the write-out recomputes each staged word's digit (a mask and a shift) to
// find its run's destination, instead of staging a destination per word,
// which halves the shared-memory traffic of the scatter.  A tile is 256
// threads x IPT words (8192 without payloads; 4096 with): few threads with
// many words each, so the tile's four barriers and its digit scan are
// amortised over more keys.  Element li of a tile is held by thread
// (li / 4) % 256, slot (li / 1024) * 4 + li % 4.
constexpr int P32_THREADS = 256;
constexpr uint32_t P32_COPIES = 4;  // counters per digit (the code reads them as one uint4)
template <int PM>
struct P32 {
    static constexpr int IPT = PM ? 16 : 32;
    static constexpr int TILE = P32_THREADS * IPT;
};
static_assert(CHUNK + 3 <= TILES_PER_CHUNK * (uint32_t)P32<0>::TILE && CHUNK + 3 <= TILES_PER_CHUNK * (uint32_t)P32<1>::TILE,
              "a chunk's window (the chunk and up to 3 words before it) spans at most TILES_PER_CHUNK tiles");

template <bool HIN, int PM, bool DR, bool POW2>
__global__ void __launch_bounds__(P32_THREADS, 2)
k_pass32(const uint32_t* __restrict__ in, const uint32_t* __restrict__ in_v, uint64_t n, Hasher H,
         uint32_t dig_shift, uint32_t dig_mask, uint32_t R, ChunkMap cm, uint32_t nch_host,
         const Plan* __restrict__ plan, const uint32_t* __restrict__ chunk_base, uint32_t* __restrict__ out,
         uint32_t* __restrict__ out_v, uint32_t* err, uint32_t* __restrict__ dr_out, uint2* __restrict__ tile_lb,
         uint32_t in_padded) {
    constexpr int IPT = P32<PM>::IPT;
    constexpr int TILE = P32<PM>::TILE;
    constexpr int NG = IPT / 4;
    extern __shared__ __align__(16) unsigned char smem[];
    uint32_t* s_h = reinterpret_cast<uint32_t*>(smem);  // staged words [TILE]
    uint32_t* s_pay = s_h + TILE;                       // staged payloads [TILE] (PM)
    // each digit's count is kept in P32_COPIES counters, lane l adding to copy
    // l % P32_COPIES, so the lanes of a warp whose keys share a digit (duplicated
    // keys) wait on at most 32 / P32_COPIES increments of one word; s_sub: where
    // each copy's keys start in the staged tile
    __shared__ __align__(16) uint32_t s_cnt[RADIX * P32_COPIES], s_sub[RADIX * P32_COPIES];
    __shared__ uint32_t s_run[RADIX], s_warp[4];
    __shared__ uint2 s_lb[RADIX];  // (offset of the digit's run inside the tile, its destination)
    const uint32_t tid = threadIdx.x;
    const uint32_t cp = lane_id() & (P32_COPIES - 1);
    const uint32_t nch = cm.segmented ? plan->chunks_b : nch_host;
    const uint32_t c = blockIdx.x;
    if (c >= nch) return;
    uint32_t seg, first;
    uint64_t lo64, hi64;
    chunk_range(cm, c, seg, first, lo64, hi64);
    // Tiles cover the chunk's window, which starts at the 16-byte boundary at or
    // before the chunk: window position x is element lo - a + x, valid for
    // a <= x < end, so every 4-word group is one aligned 16-byte load (the few
    // words around the chunk are read and ignored; in_padded: the input may be
    // read up to 3 words past its end, else the last group is read word by word)
    const uint32_t a = (uint32_t)(lo64 & 3);
    const uint32_t end = a + (uint32_t)(hi64 - lo64);
    const uint32_t* __restrict__ inc = in + (lo64 - a);
    const uint32_t* __restrict__ inc_v = PM == 1 ? in_v + (lo64 - a) : nullptr;
    uint16_t* __restrict__ drc = DR ? reinterpret_cast<uint16_t*>(dr_out) + (lo64 - a) : nullptr;
    uint2* __restrict__ lbc = DR ? tile_lb + (uint64_t)c * TILES_PER_CHUNK * RADIX : nullptr;
    const uint32_t base32 = (uint32_t)(lo64 - a);  // (index payloads: positions fit 32 bits)
    const bool vec = (reinterpret_cast<uintptr_t>(in) & 15) == 0 &&
                     (PM != 1 || (reinterpret_cast<uintptr_t>(in_v) & 15) == 0);
    const uint32_t vend = in_padded ? end + 3 : end;  // groups wholly below vend are read as vectors
    const bool dr_vec = DR && (reinterpret_cast<uintptr_t>(dr_out) & 7) == 0;
    for (uint32_t d = tid; d < RADIX * P32_COPIES; d += P32_THREADS) s_cnt[d] = 0;
    for (uint32_t d = tid; d < RADIX; d += P32_THREADS) s_run[d] = d < R ? chunk_base[(uint64_t)c * RADIX + d] : 0u;
    // the digit is masked to the radix, so shared-memory indices stay in bounds
    // whatever the word; a consistent plan never needs the mask.  POW2: B = 2^k,
    // the bucket is the hash's low k bits
    const uint32_t bmask = (uint32_t)H.mask, dsh = BIN_SHIFT + dig_shift, dmask = dig_mask & (RADIX - 1);
    auto digit = [&](uint32_t h) {
        if (POW2) return ((h & bmask) >> dsh) & dmask;
        return (bucket_of_hash(h, H) >> dsh) & dmask;
    };
    uint32_t w[IPT];
    uint32_t v[PM ? IPT : 1];
    // element li of a tile: thread (li / 4) % 256, slot (li / 1024) * 4 + li % 4
    auto load = [&](uint32_t t0, bool full) {
#pragma unroll
        for (int g = 0; g < NG; ++g) {
            const uint32_t x0 = t0 + (tid + g * P32_THREADS) * 4;
            if (full || (vec && x0 + 4 <= vend)) {
                const uint4 q = ld_stream16(inc + x0);
                w[4 * g] = q.x;
                w[4 * g + 1] = q.y;
                w[4 * g + 2] = q.z;
                w[4 * g + 3] = q.w;
                if (PM == 1) {
                    const uint4 y = ld_stream16(inc_v + x0);
                    v[4 * g] = y.x;
                    v[4 * g + 1] = y.y;
                    v[4 * g + 2] = y.z;
                    v[4 * g + 3] = y.w;
                }
            } else {
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const bool ok = x0 + u >= a && x0 + u < end;
                    w[4 * g + u] = ok ? inc[x0 + u] : 0u;
                    if (PM == 1) v[4 * g + u] = ok ? inc_v[x0 + u] : 0u;
                }
            }
            if (PM == 2) {
#pragma unroll
                for (int u = 0; u < 4; ++u) v[4 * g + u] = base32 + x0 + u;
            }
        }
    };
    auto is_full = [&](uint32_t t0) { return vec && t0 >= a && t0 + (uint32_t)TILE <= end; };
    const uint32_t nn = (uint32_t)min(n, (uint64_t)0xffffffffu);
    uint32_t bad = 0;
    // one tile; FULL: all TILE words valid and loaded with 16-byte loads (no per-word checks)
    auto tile = [&](uint32_t t0, auto full_tag) {
        constexpr bool FULL = decltype(full_tag)::value;
        const uint32_t cnt_tile = FULL ? (uint32_t)TILE : min(end, t0 + (uint32_t)TILE) - max(a, t0);
        uint32_t dr[IPT];  // rank << 8 | digit (all ones: no word)
#pragma unroll
        for (int j = 0; j < IPT; ++j) {
            if (!HIN) w[j] = hash_key32(w[j], H);
            const uint32_t d = digit(w[j]);
            const uint32_t x = t0 + (tid + (j / 4) * P32_THREADS) * 4 + (j % 4);
            const bool ok = FULL || (x >= a && x < end);
            dr[j] = ok ? ((atomicAdd(s_cnt + d * P32_COPIES + cp, 1u) << 8) | d) : 0xffffffffu;
        }
        __syncthreads();
        // digit offsets inside the tile (first 4 warps), and where each run goes
        if (tid < RADIX) {
            const uint32_t d = tid;
            const uint4 c4 = *reinterpret_cast<const uint4*>(s_cnt + d * P32_COPIES);
            const uint32_t cd = c4.x + c4.y + c4.z + c4.w;
            const uint32_t incl = warp_inclusive_scan(cd);
            if (lane_id() == 31) s_warp[d >> 5] = incl;
            asm volatile("bar.sync 1, 128;");
            uint32_t wp = 0;
            for (uint32_t x = 0; x < (d >> 5); ++x) wp += s_warp[x];
            const uint2 lb = make_uint2(wp + incl - cd, s_run[d]);
            s_lb[d] = lb;
            *reinterpret_cast<uint4*>(s_sub + d * P32_COPIES) =
                make_uint4(lb.x, lb.x + c4.x, lb.x + c4.x + c4.y, lb.x + c4.x + c4.y + c4.z);
            if (DR) lbc[(t0 / TILE) * RADIX + d] = lb;
            s_run[d] += cd;
            *reinterpret_cast<uint4*>(s_cnt + d * P32_COPIES) = make_uint4(0, 0, 0, 0);
        }
        __syncthreads();
#pragma unroll
        for (int j = 0; j < IPT; ++j) {
            if (FULL || dr[j] != 0xffffffffu) {
                const uint32_t pos = s_sub[(dr[j] & 0xffu) * P32_COPIES + cp] + (dr[j] >> 8);
                s_h[pos] = w[j];
                if (PM) s_pay[pos] = v[j];
                if (DR) dr[j] = pos;
            }
        }
        // DR: each element's record is its staging position in the tile (16 bits):
        // the reverse pass finds every staged word's source from the tile's runs
        if (DR) {
            if (FULL && dr_vec) {
#pragma unroll
                for (int g = 0; g < NG; ++g)
                    *reinterpret_cast<uint2*>(drc + t0 + (tid + g * P32_THREADS) * 4) =
                        make_uint2(dr[4 * g] | (dr[4 * g + 1] << 16), dr[4 * g + 2] | (dr[4 * g + 3] << 16));
            } else {
#pragma unroll
                for (int j = 0; j < IPT; ++j)
                    if (dr[j] != 0xffffffffu) drc[t0 + (tid + (j / 4) * P32_THREADS) * 4 + (j % 4)] = (uint16_t)dr[j];
            }
        }
        __syncthreads();
        // prefetch the next tile while this one is written out
        const uint32_t t1 = t0 + TILE;
        if (t1 < end) load(t1, is_full(t1));
        auto put = [&](uint32_t i) {
            const uint32_t h = s_h[i];
            const uint2 lb = s_lb[digit(h)];
            const uint32_t dst = lb.y + (i - lb.x);
            if (dst < nn) {
                out[dst] = h;
                if (PM) out_v[dst] = s_pay[i];
            } else {
                bad = 1;
            }
        };
        if (FULL) {
#pragma unroll 8
            for (int r = 0; r < IPT; ++r) put(tid + r * P32_THREADS);
        } else {
            for (uint32_t i = tid; i < cnt_tile; i += P32_THREADS) put(i);
        }
        // no barrier ends the tile: the next tile's ranking touches only s_cnt,
        // and s_lb and s_h are rewritten only after its first barrier, which
        // every thread reaches after this write-out
    };
    __syncthreads();
    if (end > a) load(0, is_full(0));
    for (uint32_t t0 = 0; t0 < end; t0 += TILE) {
        if (is_full(t0)) tile(t0, std::true_type{});
        else tile(t0, std::false_type{});
    }
    if (bad) atomicOr(err, DEVERR_BOUNDS);
}

// ---------------------------------------------------------------- reverse --
// Undo one DR-recording pass for 32-bit values: src is in the pass's output
// order, dst receives the values in its input order.  Each tile reads the runs
// it wrote (contiguous, so the reads coalesce) into shared memory in its
// staging order, then every element takes its value from its recorded
// (rank, digit) and writes it in input order.  The run reads are asynchronous
// copies into shared memory, all of a thread's in flight at once, and the next
// tile's records are requested while they land.
template <typename K>
__global__ void __launch_bounds__(PASS_THREADS, sizeof(K) == 4 ? 2 : 3)
k_pass_reverse(const uint32_t* __restrict__ src, uint32_t* __restrict__ dst, ChunkMap cm, uint32_t nch_host,
               const Plan* __restrict__ plan, const uint32_t* __restrict__ dr_in, const uint2* __restrict__ tile_lb,
               uint32_t* err) {
    // the forward pass's tile: k_pass32 for 32-bit keys, k_pass_down otherwise
    constexpr int TILE = sizeof(K) == 4 ? P32<0>::TILE : PassCfg<K>::TILE;
    constexpr int PER = TILE / PASS_THREADS;
    __shared__ uint32_t s_val[TILE];
    __shared__ uint8_t s_dig[TILE];
    __shared__ uint2 s_lb[RADIX];
    const uint32_t nch = cm.segmented ? plan->chunks_b : nch_host;
    const uint32_t c = blockIdx.x;
    if (c >= nch) return;
    uint32_t seg, first;
    uint64_t lo, hi;
    chunk_range(cm, c, seg, first, lo, hi);
    // tiles as the forward pass cut them: for 32-bit keys from the 16-byte
    // boundary at or before the chunk's start (window position x = element
    // lo - a + x, valid for a <= x < end), for 64-bit keys from the start
    const uint32_t a = sizeof(K) == 4 ? (uint32_t)(lo & 3) : 0u;
    const uint32_t end = a + (uint32_t)(hi - lo);
    const uint32_t* __restrict__ drc = dr_in + (lo - a);
    uint32_t* __restrict__ dstc = dst + (lo - a);
    uint32_t drs[PER];
    uint2 lbr = make_uint2(0, 0);
    auto fetch = [&](uint32_t t0) {
#pragma unroll
        for (int j = 0; j < PER; ++j) {
            const uint32_t x = t0 + threadIdx.x + j * PASS_THREADS;
            drs[j] = (x >= a && x < end) ? __ldg(drc + x) : 0xffffffffu;
        }
        if (threadIdx.x < RADIX)
            lbr = __ldg(tile_lb + ((uint64_t)c * TILES_PER_CHUNK + t0 / TILE) * RADIX + threadIdx.x);
    };
    if (end > a) fetch(0);
    for (uint32_t t0 = 0; t0 < end; t0 += TILE) {
        const uint32_t cnt_tile = min(end, t0 + (uint32_t)TILE) - max(a, t0);  // valid elements
        if (threadIdx.x < RADIX) s_lb[threadIdx.x] = lbr;
        __syncthreads();
        // every element marks its staging position with its digit ...
        static_assert(TILE < 0xffff, "staging positions are kept in 16 bits");
        uint32_t pj[PER / 2];  // two 16-bit staging positions per word, 0xffff = none
#pragma unroll
        for (int j = 0; j < PER; ++j) {
            uint32_t pos = 0xffffu;
            if (drs[j] != 0xffffffffu) {
                const uint32_t p = s_lb[drs[j] & 0xffu].x + (drs[j] >> 8);
                if (p < (uint32_t)TILE) {
                    s_dig[p] = (uint8_t)(drs[j] & 0xffu);
                    pos = p;
                } else {
                    atomicOr(err, DEVERR_BOUNDS);
                }
            }
            if (j & 1) pj[j / 2] |= pos << 16;
            else pj[j / 2] = pos;
        }
        __syncthreads();
        // ... so that the tile's runs are read back contiguously in staging order
        // (asynchronous copies straight into shared memory)
#pragma unroll
        for (int j = 0; j < PER; ++j) {
            const uint32_t i = threadIdx.x + j * PASS_THREADS;
            if (i < cnt_tile) {
                const uint2 lb = s_lb[s_dig[i]];
                cp_async4(s_val + i, src + lb.y + (i - lb.x));
            }
        }
        const uint32_t t1 = t0 + TILE;
        if (t1 < end) fetch(t1);
        cp_async_wait_all();
        __syncthreads();
        // s_lb and s_dig are not read past this point, and s_val is next written
        // after the next tile's second barrier, so no barrier ends the tile
#pragma unroll
        for (int j = 0; j < PER; ++j) {
            const uint32_t x = t0 + threadIdx.x + j * PASS_THREADS;
            const uint32_t pos = (pj[j / 2] >> ((j & 1) * 16)) & 0xffffu;
            if (pos != 0xffffu) dstc[x] = s_val[pos];
        }
    }
}

// k_pass_reverse for the 32-bit passes (k_pass32), whose records are each
// element's 16-bit staging position in its tile.  Every warp copies whole runs
// of the tile (digit d's run: staged positions [loc_d, loc_{d+1}) from
// base_d + ...) into shared memory with asynchronous copies, then each element
// takes its value from its staging position.  256 threads, each holding 32
// elements of a tile as eight 4-element groups (element x of the chunk's window
// in thread (x / 4) % 256, as in the forward pass), so the records come in 8
// bytes and the values go out 16 bytes at a time.
__global__ void __launch_bounds__(P32_THREADS, 3)
k_pass_reverse32(const uint32_t* __restrict__ src, uint32_t* __restrict__ dst, ChunkMap cm, uint32_t nch_host,
                 const Plan* __restrict__ plan, const uint32_t* __restrict__ dr_in, const uint2* __restrict__ tile_lb,
                 uint32_t* err) {
    constexpr int TILE = P32<0>::TILE;
    constexpr int NG = P32<0>::IPT / 4;
    constexpr int PER = P32<0>::IPT;
    __shared__ __align__(16) uint32_t s_val[TILE];
    __shared__ uint2 s_lb[RADIX + 1];
    const uint32_t tid = threadIdx.x, lane = lane_id(), warp = tid >> 5;
    const uint32_t nch = cm.segmented ? plan->chunks_b : nch_host;
    const uint32_t c = blockIdx.x;
    if (c >= nch) return;
    uint32_t seg, first;
    uint64_t lo, hi;
    chunk_range(cm, c, seg, first, lo, hi);
    // the forward pass's tiles over the chunk's window: position x is element
    // lo - a + x, valid for a <= x < end
    const uint32_t a = (uint32_t)(lo & 3);
    const uint32_t end = a + (uint32_t)(hi - lo);
    // (records: an internal array, 8-byte aligned and padded past its end)
    const uint16_t* __restrict__ drc = reinterpret_cast<const uint16_t*>(dr_in) + (lo - a);
    uint32_t* __restrict__ dstc = dst + (lo - a);
    const bool dvec = (reinterpret_cast<uintptr_t>(dst) & 15) == 0;
    const uint2* __restrict__ lbc = tile_lb + (uint64_t)c * TILES_PER_CHUNK * RADIX;
    uint32_t pj[PER / 2];  // two 16-bit staging positions per word, 0xffff = no element
    uint2 lbr = make_uint2(0, 0);
    auto fetch = [&](uint32_t t0) {
#pragma unroll
        for (int g = 0; g < NG; ++g) {
            const uint32_t x0 = t0 + (tid + g * P32_THREADS) * 4;
            uint2 q = make_uint2(0xffffffffu, 0xffffffffu);
            if (x0 < end) {
                q = __ldg(reinterpret_cast<const uint2*>(drc + x0));
                if (x0 < a || x0 + 4 > end) {  // a window edge: mark the elements outside the chunk
                    uint32_t m[4] = {q.x & 0xffffu, q.x >> 16, q.y & 0xffffu, q.y >> 16};
#pragma unroll
                    for (int u = 0; u < 4; ++u)
                        if (x0 + u < a || x0 + u >= end) m[u] = 0xffffu;
                    q = make_uint2(m[0] | (m[1] << 16), m[2] | (m[3] << 16));
                }
            }
            pj[2 * g] = q.x;
            pj[2 * g + 1] = q.y;
        }
        if (tid < RADIX) lbr = __ldg(lbc + (t0 / TILE) * RADIX + tid);
    };
    if (end > a) fetch(0);
    for (uint32_t t0 = 0; t0 < end; t0 += TILE) {
        const uint32_t cnt_tile = min(end, t0 + (uint32_t)TILE) - max(a, t0);  // valid elements
        if (tid < RADIX) s_lb[tid] = lbr;
        if (tid == 0) s_lb[RADIX] = make_uint2(cnt_tile, 0);
        __syncthreads();
        // the tile's runs, a warp per digit (d = warp, warp + 8, ...), copied to
        // their staging positions
        for (uint32_t d = warp; d < RADIX; d += P32_THREADS / 32) {
            const uint2 lb = s_lb[d];
            const uint32_t len = min(s_lb[d + 1].x, (uint32_t)TILE) - min(lb.x, (uint32_t)TILE);
            for (uint32_t k = lane; k < len; k += 32) cp_async4(s_val + lb.x + k, src + lb.y + k);
        }
        uint32_t pos_now[PER / 2];
#pragma unroll
        for (int q = 0; q < PER / 2; ++q) pos_now[q] = pj[q];
        const uint32_t t1 = t0 + TILE;
        if (t1 < end) fetch(t1);
        cp_async_wait_all();
        __syncthreads();
#pragma unroll
        for (int g = 0; g < NG; ++g) {
            const uint32_t x0 = t0 + (tid + g * P32_THREADS) * 4;
            uint32_t pos[4], val[4];
            pos[0] = pos_now[2 * g] & 0xffffu;
            pos[1] = pos_now[2 * g] >> 16;
            pos[2] = pos_now[2 * g + 1] & 0xffffu;
            pos[3] = pos_now[2 * g + 1] >> 16;
            bool bad = false;
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                bad |= pos[u] != 0xffffu && pos[u] >= cnt_tile;
                val[u] = pos[u] < cnt_tile ? s_val[pos[u]] : 0u;
            }
            if (bad) atomicOr(err, DEVERR_BOUNDS);
            if (dvec && pos[0] != 0xffffu && pos[3] != 0xffffu) {
                *reinterpret_cast<uint4*>(dstc + x0) = make_uint4(val[0], val[1], val[2], val[3]);
            } else {
#pragma unroll
                for (int u = 0; u < 4; ++u)
                    if (pos[u] != 0xffffu) dstc[x0 + u] = val[u];
            }
        }
        // no barrier ends the tile: s_val is rewritten by the next tile's copies
        // only after its first barrier, which every thread reaches after this
        // tile's reads (s_lb, rewritten before that barrier, is not read here)
    }
}

// ---------------------------------------------------------------- local --
// Huge bin work item -> (huge index e, bin p, key range [c0, c1)).
__device__ __forceinline__ void huge_item(uint32_t item, uint32_t n_huge, uint32_t chunk, const uint32_t* __restrict__ huge_chunk_start,
                                          const uint32_t* __restrict__ huge_bin,
                                          const uint32_t* __restrict__ bin_start, uint32_t& e, uint32_t& p,
                                          uint64_t& c0, uint64_t& c1) {
    uint32_t lo = 0, hi = n_huge;
    while (hi - lo > 1) {
        const uint32_t mid = (lo + hi) >> 1;
        if (huge_chunk_start[mid] <= item) lo = mid; else hi = mid;
    }
    e = lo;
    p = huge_bin[e];
    c0 = (uint64_t)bin_start[p] + (uint64_t)(item - huge_chunk_start[e]) * chunk;
    c1 = min((uint64_t)bin_start[p + 1], c0 + chunk);
}

// Huge bins, step 1: per-chunk bucket histograms added into huge_count[e][*].
// HIN: the keys are 32-bit hashes (the partition passes' words), the bucket is taken from them.
template <typename K, bool HIN>
__device__ __forceinline__ uint32_t bucket_in(K k, const Hasher& H) {
    if constexpr (HIN) return bucket_of_hash((uint32_t)k, H);
    else return bucket_of(k, H);
}
template <typename K, bool HIN>
__device__ __forceinline__ K key_in(K k, const Hasher& H) {
    if constexpr (HIN) return (K)unhash_key32((uint32_t)k, H);
    else return k;
}

template <typename K, bool HIN>
__global__ void __launch_bounds__(LOCAL_THREADS)
k_huge_count(const K* __restrict__ in, Hasher H, const uint32_t* __restrict__ bin_start,
             const uint32_t* __restrict__ huge_bin, const uint32_t* __restrict__ huge_chunk_start,
             const Plan* __restrict__ plan, uint32_t* huge_count, uint32_t* err) {
    extern __shared__ __align__(16) unsigned char smem[];
    uint32_t* s_cnt = reinterpret_cast<uint32_t*>(smem);
    const uint32_t n_huge = plan->n_huge, total = plan->huge_chunks;
    for (uint32_t item = blockIdx.x; item < total; item += gridDim.x) {
        uint32_t e, p;
        uint64_t c0, c1;
        huge_item(item, n_huge, plan->huge_chunk, huge_chunk_start, huge_bin, bin_start, e, p, c0, c1);
        const uint64_t b0 = (uint64_t)p << BIN_SHIFT;
        const uint32_t nb = (uint32_t)min((uint64_t)BPB, H.B - b0);
        for (uint32_t j = threadIdx.x; j < BPB; j += blockDim.x) s_cnt[j] = 0;
        __syncthreads();
        block_for_range<K, false>(in, nullptr, c0, c1, [&](uint64_t, K k, uint32_t, unsigned m) {
            uint32_t j = (uint32_t)(bucket_in<K, HIN>(k, H) - b0);
            if (j >= nb) {
                atomicOr(err, DEVERR_BOUNDS);
                j = nb - 1;
            }
            smem_add1(s_cnt, j, m);
        });
        __syncthreads();
        for (uint32_t j = threadIdx.x; j < nb; j += blockDim.x)
            if (s_cnt[j]) atomicAdd(huge_count + (uint64_t)e * BPB + j, s_cnt[j]);
        __syncthreads();
    }
}

// The huge bins' work items as (bin slot e, bin p, first key, end key), one CTA per huge bin.
__global__ void __launch_bounds__(256)
k_huge_items(const uint32_t* __restrict__ bin_start, const uint32_t* __restrict__ huge_bin,
             const uint32_t* __restrict__ huge_chunk_start, const Plan* __restrict__ plan, uint4* item_meta) {
    const uint32_t e = blockIdx.x;
    if (e >= plan->n_huge) return;
    const uint32_t p = huge_bin[e];
    const uint32_t chunk = plan->huge_chunk, bs = bin_start[p], be = bin_start[p + 1];
    const uint32_t i0 = huge_chunk_start[e], ni = huge_chunk_start[e + 1] - i0;
    for (uint32_t k = threadIdx.x; k < ni; k += blockDim.x) {
        const uint32_t lo = bs + k * chunk;
        item_meta[i0 + k] = make_uint4(e, p, lo, min(be, lo + chunk));
    }
}

// Huge bins, step 2: one CTA per huge bin scans its counts into offsets and cursors.
__global__ void __launch_bounds__(1024)
k_huge_scan(const uint32_t* __restrict__ bin_start, const uint32_t* __restrict__ huge_bin,
            const Plan* __restrict__ plan, const uint32_t* __restrict__ huge_count, uint32_t* huge_cursor,
            uint32_t* offsets, uint64_t B, LongFinder LF) {
    __shared__ uint32_t s_warp[33];
    const uint32_t e = blockIdx.x;
    if (e >= plan->n_huge) return;
    const uint32_t p = huge_bin[e];
    const uint64_t b0 = (uint64_t)p << BIN_SHIFT;
    const uint32_t nb = (uint32_t)min((uint64_t)BPB, B - b0);
    uint32_t running = bin_start[p], tot;
    for (uint32_t base = 0; base < nb; base += blockDim.x) {
        const uint32_t j = base + threadIdx.x;
        const uint32_t c = j < nb ? huge_count[(uint64_t)e * BPB + j] : 0u;
        const uint32_t ex = block_exclusive_scan<uint32_t>(c, s_warp, &tot);
        if (j < nb) {
            offsets[b0 + j] = running + ex;
            huge_cursor[(uint64_t)e * BPB + j] = running + ex;
            if (LF.map && c > SUM_MIN_LEN) note_long(LF, (uint32_t)(b0 + j));
        }
        running += tot;
    }
}


// Step 3 (all bins): work items [0, huge_chunks) place one chunk of a huge bin
// through its cursors; the following n_work items each take a whole bin.
// Shared memory: cnt[BPB] | hotmask[BPB/32] | hot list (pos, prefix length) | stage keys | stage payload.
template <typename K, bool HV, bool HIN>
__global__ void __launch_bounds__(LOCAL_THREADS, 2)
k_bin_local(const K* __restrict__ in, const uint32_t* __restrict__ in_v, uint64_t n, Hasher H,
            const uint32_t* __restrict__ bin_start, const uint32_t* __restrict__ work,
            const uint32_t* __restrict__ huge_bin, const uint32_t* __restrict__ huge_chunk_start,
            const Plan* __restrict__ plan, uint32_t* huge_cursor, uint32_t* work_ctr, uint32_t* offsets,
            K* __restrict__ out, uint32_t* __restrict__ out_v, uint32_t* err, LongFinder LF, bool big_only) {
    // big_only: k_bin_small takes the small bins and k_big_place the huge bins' chunks
    constexpr uint32_t STAGE_CAP = (uint32_t)(LOCAL_STAGE_BYTES / (sizeof(K) + (HV ? 4 : 0)));
    extern __shared__ __align__(16) unsigned char smem[];
    uint32_t* s_cnt = reinterpret_cast<uint32_t*>(smem);
    uint32_t* s_hot = s_cnt + BPB;                 // bitmask
    uint32_t* s_hot_cpos = s_hot + BPB / 32;       // compacted position of each hot bucket
    uint32_t* s_hot_len = s_hot_cpos + MAX_HOT;    // its length (then inclusive prefix)
    K* s_keys = reinterpret_cast<K*>(s_hot_len + MAX_HOT);
    uint32_t* s_pay = reinterpret_cast<uint32_t*>(s_keys + STAGE_CAP);
    __shared__ uint32_t s_item, s_nhot, s_red[NTHR][LOCAL_THREADS / 32];

    const unsigned lane = lane_id();
    const int w = threadIdx.x >> 5;
    constexpr int NW = LOCAL_THREADS / 32;
    const uint64_t B = H.B;
    const uint32_t n_huge = plan->n_huge, huge_chunks = plan->huge_chunks;
    const uint32_t n_work = big_only ? plan->n_big : plan->n_work;
    const uint32_t first_item = big_only ? huge_chunks : 0u;
    // candidate thresholds: a bucket with at least THR[k] keys bypasses the staging buffer
    const uint32_t THR[NTHR] = {0xffffffffu, 4096u, 1024u, 256u, 64u};

    while (true) {
        if (threadIdx.x == 0) s_item = first_item + atomicAdd(work_ctr, 1u);
        __syncthreads();
        const uint32_t item = s_item;
        if (item >= huge_chunks + n_work) break;

        if (item < huge_chunks) {
            // ---- one chunk of a huge bin: local histogram, reserve runs, place
            uint32_t e, p;
            uint64_t c0, c1;
            huge_item(item, n_huge, plan->huge_chunk, huge_chunk_start, huge_bin, bin_start, e, p, c0, c1);
            const uint64_t b0 = (uint64_t)p << BIN_SHIFT;
            const uint32_t nb = (uint32_t)min((uint64_t)BPB, B - b0);
            for (uint32_t j = threadIdx.x; j < BPB; j += blockDim.x) s_cnt[j] = 0;
            __syncthreads();
            block_for_range<K, false>(in, nullptr, c0, c1, [&](uint64_t, K k, uint32_t, unsigned m) {
                uint32_t j = (uint32_t)(bucket_in<K, HIN>(k, H) - b0);
                if (j >= nb) j = nb - 1;  // flagged by k_huge_count
                smem_add1(s_cnt, j, m);
            });
            __syncthreads();
            for (uint32_t j = threadIdx.x; j < nb; j += blockDim.x) {
                const uint32_t c = s_cnt[j];
                if (c) s_cnt[j] = atomicAdd(huge_cursor + (uint64_t)e * BPB + j, c);
            }
            __syncthreads();
            block_for_range<K, HV>(in, in_v, c0, c1, [&](uint64_t, K k, uint32_t v, unsigned m) {
                uint32_t j = (uint32_t)(bucket_in<K, HIN>(k, H) - b0);
                if (j >= nb) j = nb - 1;
                const uint32_t pos = smem_inc(s_cnt, j, m);
                if (pos < n) {
                    out[pos] = key_in<K, HIN>(k, H);
                    if (HV) out_v[pos] = v;
                } else {
                    atomicOr(err, DEVERR_BOUNDS);
                }
            });
            __syncthreads();
            continue;
        }

        // ---- a whole bin
        const uint32_t p = work[item - huge_chunks];
        const uint64_t s0 = bin_start[p], s1 = bin_start[p + 1];
        const uint64_t b0 = (uint64_t)p << BIN_SHIFT;
        const uint32_t nb = (uint32_t)min((uint64_t)BPB, B - b0);

        for (uint32_t j = threadIdx.x; j < BPB; j += blockDim.x) s_cnt[j] = 0;
        for (uint32_t j = threadIdx.x; j < BPB / 32; j += blockDim.x) s_hot[j] = 0;
        if (threadIdx.x == 0) s_nhot = 0;
        __syncthreads();

        // pass 1: bucket histogram.  Only a bin too large for the staging buffer
        // can hold a heavily duplicated key, so only there do warps check for
        // a shared counter first.
        const bool heavy = s1 - s0 > STAGE_CAP;
        auto hist = [&](auto fast) {
            // (the placement pass reads these keys again: keep them in L2)
            block_for_range<K, false, 2, true>(in, nullptr, s0, s1, [&](uint64_t, K k, uint32_t, unsigned m) {
                uint32_t j = (uint32_t)(bucket_in<K, HIN>(k, H) - b0);
                if (j >= nb) {
                    atomicOr(err, DEVERR_BOUNDS);
                    j = nb - 1;
                }
                if (decltype(fast)::value) smem_add1(s_cnt, j, m);
                else atomicAdd(s_cnt + j, 1u);
            });
        };
        if (heavy) hist(std::true_type{});
        else hist(std::false_type{});
        __syncthreads();

        // Choose the largest threshold whose non-bypassed ("cold") keys fit the
        // staging buffer.  Thread t owns the CPT consecutive buckets from t * CPT
        // (so each warp a contiguous slice) and keeps their counts in registers.
        constexpr int CPT = (int)(BPB / LOCAL_THREADS);
        static_assert(CPT % 4 == 0 && 32 % CPT == 0, "bucket slice per thread");
        const uint32_t jt = threadIdx.x * CPT;
        auto cnt4 = [&](int u0) { return *reinterpret_cast<const uint4*>(s_cnt + jt + u0); };
        {
            uint32_t cold[NTHR] = {0, 0, 0, 0, 0};
#pragma unroll
            for (int u0 = 0; u0 < CPT; u0 += 4) {
                const uint4 x = cnt4(u0);
                const uint32_t cv[4] = {x.x, x.y, x.z, x.w};
#pragma unroll
                for (int u = 0; u < 4; ++u)
#pragma unroll
                    for (int q = 0; q < NTHR; ++q) cold[q] += cv[u] < THR[q] ? cv[u] : 0u;
            }
#pragma unroll
            for (int q = 0; q < NTHR; ++q) {
                const uint32_t wsum = __reduce_add_sync(FULL_MASK, cold[q]);
                if (lane == 0) s_red[q][w] = wsum;
            }
        }
        // buckets of more than SUM_MIN_LEN keys (HG_LONG_SUMMARY), only possible in a bin that large
        if (LF.map && s1 - s0 > SUM_MIN_LEN) {
#pragma unroll
            for (int u0 = 0; u0 < CPT; u0 += 4) {
                const uint4 x = cnt4(u0);
                const uint32_t cv[4] = {x.x, x.y, x.z, x.w};
#pragma unroll
                for (int u = 0; u < 4; ++u)
                    if (cv[u] > SUM_MIN_LEN) note_long(LF, (uint32_t)(b0 + jt + u0 + u));
            }
        }
        __syncthreads();
        int sel = -1;
        uint32_t cold_total = 0;
        for (int q = 0; q < NTHR && sel < 0; ++q) {
            uint32_t t = 0;
            for (int x = 0; x < NW; ++x) t += s_red[q][x];
            if (t <= STAGE_CAP) {
                sel = q;
                cold_total = t;
            }
        }
        const bool stage = sel >= 0;
        const uint32_t thr = stage ? THR[sel] : 0u;
        // per-warp prefixes of all keys (q = 0 is "everything") and of the cold keys,
        // then this thread's, then serially over its buckets
        uint32_t pre_all = 0, pre_cold = 0;
        for (int x = 0; x < w; ++x) {
            pre_all += s_red[0][x];
            if (stage) pre_cold += s_red[sel][x];
        }
        uint32_t t_all = 0, t_cold = 0;
#pragma unroll
        for (int u0 = 0; u0 < CPT; u0 += 4) {
            const uint4 x = cnt4(u0);
            const uint32_t cv[4] = {x.x, x.y, x.z, x.w};
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                t_all += cv[u];
                t_cold += (!stage || cv[u] >= thr) ? 0u : cv[u];
            }
        }
        uint32_t run_all = (uint32_t)s0 + pre_all + warp_inclusive_scan(t_all) - t_all;
        uint32_t run_cold = pre_cold + warp_inclusive_scan(t_cold) - t_cold;
        uint32_t hotbits = 0;
#pragma unroll
        for (int u0 = 0; u0 < CPT; u0 += 4) {  // four buckets at a time: one vector store each
            const uint4 x = cnt4(u0);
            const uint32_t cv[4] = {x.x, x.y, x.z, x.w};
            uint32_t st[4], cur[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const uint32_t cu = cv[u];
                const bool hot = !stage || cu >= thr;
                st[u] = run_all;
                run_all += cu;
                if (!hot) {
                    cur[u] = run_cold;  // staging cursor
                    run_cold += cu;
                } else {
                    cur[u] = st[u];  // global cursor
                    if (stage && cu) {
                        hotbits |= 1u << (u0 + u);
                        const uint32_t h = atomicAdd(&s_nhot, 1u);
                        if (h < MAX_HOT) {
                            s_hot_cpos[h] = run_cold;
                            s_hot_len[h] = cu;
                        }
                    }
                }
            }
            *reinterpret_cast<uint4*>(s_cnt + jt + u0) = make_uint4(cur[0], cur[1], cur[2], cur[3]);
            if (jt + u0 + 4 <= nb) {
                *reinterpret_cast<uint4*>(offsets + b0 + jt + u0) = make_uint4(st[0], st[1], st[2], st[3]);
            } else {
#pragma unroll
                for (int u = 0; u < 4; ++u)
                    if (jt + u0 + u < nb) offsets[b0 + jt + u0 + u] = st[u];
            }
        }
        if (hotbits) atomicOr(&s_hot[jt >> 5], hotbits << (jt & 31));
        __syncthreads();
        const uint32_t nhot = s_nhot;
        const bool staged = stage && nhot <= MAX_HOT;
        if (stage && !staged) {
            // too many bypassing buckets for the map: every bucket is placed directly
            for (uint32_t j = threadIdx.x; j < nb; j += blockDim.x) s_cnt[j] = offsets[b0 + j];
            __syncthreads();
        }
        // hot list sorted by compacted position (one thread; the list is short),
        // lengths turned into inclusive prefix sums
        if (staged && threadIdx.x == 0) {
            for (uint32_t a = 1; a < nhot; ++a) {
                const uint32_t kp = s_hot_cpos[a], kl = s_hot_len[a];
                int bidx = (int)a - 1;
                while (bidx >= 0 && s_hot_cpos[bidx] > kp) {
                    s_hot_cpos[bidx + 1] = s_hot_cpos[bidx];
                    s_hot_len[bidx + 1] = s_hot_len[bidx];
                    --bidx;
                }
                s_hot_cpos[bidx + 1] = kp;
                s_hot_len[bidx + 1] = kl;
            }
            for (uint32_t a = 1; a < nhot; ++a) s_hot_len[a] += s_hot_len[a - 1];
        }
        __syncthreads();

        // pass 2: place (bypassing buckets straight to global memory, the rest staged)
        if (staged && nhot == 0 && !heavy) {
            // the common bin: every key is staged, counters are rarely shared
            block_for_range<K, HV>(in, in_v, s0, s1, [&](uint64_t, K k, uint32_t v, unsigned) {
                uint32_t j = (uint32_t)(bucket_in<K, HIN>(k, H) - b0);
                if (j >= nb) j = nb - 1;  // flagged in pass 1
                const uint32_t pos = atomicAdd(s_cnt + j, 1u);
                if (pos < STAGE_CAP) {
                    s_keys[pos] = key_in<K, HIN>(k, H);
                    if (HV) s_pay[pos] = v;
                } else {
                    atomicOr(err, DEVERR_BOUNDS);
                }
            });
        } else {
            block_for_range<K, HV>(in, in_v, s0, s1, [&](uint64_t, K k, uint32_t v, unsigned m) {
                uint32_t j = (uint32_t)(bucket_in<K, HIN>(k, H) - b0);
                if (j >= nb) j = nb - 1;  // flagged in pass 1
                const uint32_t pos = smem_inc(s_cnt, j, m);
                const bool hot = !staged || ((s_hot[j >> 5] >> (j & 31)) & 1u);
                if (!hot) {
                    if (pos < STAGE_CAP) {
                        s_keys[pos] = key_in<K, HIN>(k, H);
                        if (HV) s_pay[pos] = v;
                    } else {
                        atomicOr(err, DEVERR_BOUNDS);
                    }
                } else if (pos < n) {
                    out[pos] = key_in<K, HIN>(k, H);
                    if (HV) out_v[pos] = v;
                } else {
                    atomicOr(err, DEVERR_BOUNDS);
                }
            });
        }
        __syncthreads();
        // staged keys: compacted position c goes to s0 + c + (lengths of hot buckets at or before c)
        if (staged) {
            for (uint32_t c = threadIdx.x; c < cold_total; c += blockDim.x) {
                uint32_t lo_h = 0, hi_h = nhot;
                while (lo_h < hi_h) {
                    const uint32_t mid = (lo_h + hi_h) >> 1;
                    if (s_hot_cpos[mid] <= c) lo_h = mid + 1; else hi_h = mid;
                }
                const uint32_t shift = lo_h ? s_hot_len[lo_h - 1] : 0u;
                const uint64_t dst = s0 + c + shift;
                if (dst < n) {
                    out[dst] = s_keys[c];
                    if (HV) out_v[dst] = s_pay[c];
                }
            }
        }
        __syncthreads();
    }
}

// Bins of at most SB_CAP 32-bit keys (no values), one at a time per CTA, read
// as the partition passes leave them (each key's hash; the keys written out
// are recovered with fmix32_inv): the bin's words arrive in shared memory by
// one bulk copy (TMA) issued while the
// CTA works on the bin before, so no phase waits on HBM.  Each thread holds up
// to SB_KPT keys in registers with their buckets; the counting sort of
// Algorithm 1 runs in shared memory (histogram -> exclusive scan, which gives
// the bin's offsets -> placement back into the same buffer, the keys being in
// registers by then), and the sorted bin leaves in 16-byte stores.
constexpr int SB_THREADS = 1024;
constexpr int SB_KPT = 20;
// A bin's (or chunk's) words are read from the 16-byte boundary at or before
// its start, so up to 3 words before it share the threads' SB_THREADS * SB_KPT
// slots: SB_CAP keys at most.
constexpr uint32_t SB_CAP = (uint32_t)SB_THREADS * SB_KPT - 4;
constexpr uint32_t SB_BUF_KEYS = SB_CAP + 8;        // room for the copy's 16-byte alignment at both ends
constexpr uint32_t SB_WAIT_LIMIT = 1u << 24;        // polls of a copy's barrier before the CTA gives up
constexpr size_t SB_SMEM = (size_t)BPB * 4 + 2 * (size_t)SB_BUF_KEYS * 4;
static_assert(BPB == 8 * SB_THREADS, "each thread scans eight buckets");

// k_bin_small keeps a counter array per buffer, so that a bin's counters can
// be cleared while the next bin is being counted
constexpr size_t SB_SMEM_SMALL = 2 * (size_t)BPB * 4 + 2 * (size_t)SB_BUF_KEYS * 4;
static_assert(SB_SMEM_SMALL + 1024 <= 227 * 1024, "k_bin_small's shared memory exceeds a CTA's");

template <bool POW2, bool LONGS>
__global__ void __launch_bounds__(SB_THREADS, 1)
k_bin_small(const uint32_t* __restrict__ in, Hasher H, const uint32_t* __restrict__ bin_start,
            const uint32_t* __restrict__ work, const Plan* __restrict__ plan, uint32_t* __restrict__ offsets,
            uint32_t* __restrict__ out, uint32_t* err, LongFinder LF) {
    constexpr int GR = SB_KPT / 4;  // 16-byte groups of keys per thread
    extern __shared__ __align__(16) unsigned char smem[];
    uint32_t* const s_cnt0 = reinterpret_cast<uint32_t*>(smem);  // buffer b's counters at s_cnt0 + b * BPB
    uint32_t* const s_buf0 = s_cnt0 + 2 * BPB;                    // buffer b at s_buf0 + b * SB_BUF_KEYS
    __shared__ __align__(8) uint64_t s_bar[2];
    __shared__ uint32_t s_bin[2], s_lo[2], s_hi[2], s_wsum[SB_THREADS / 32];
    const uint32_t tid = threadIdx.x, lane = lane_id(), w = tid >> 5;
    const uint32_t n_big = plan->n_big, n_small = plan->n_work - n_big;
    const uint32_t G = gridDim.x;

    // Static schedule: this CTA takes small bins blockIdx.x, blockIdx.x + G, ...
    // (they are of similar size); bin i goes to buffer i % 2.  Thread 0 starts
    // the copy of bin (p, s0, s1) into buffer b.  The first two bins are copied
    // before the loop; bin i + 1 is copied into the buffer bin i - 1 used as soon
    // as every thread has passed bin i's first barrier (so none still reads it).
    // The bin's number and range are read one bin ahead, so no phase waits on them.
    auto start_copy = [&](int b, uint32_t p, uint32_t s0, uint32_t s1) {
        s_bin[b] = p;
        s_lo[b] = s0;
        s_hi[b] = s1;
        if (p == ~0u || s1 - s0 > SB_CAP) return;  // none left / inconsistent plan (flagged by the CTA)
        const uint32_t klo = s0 & ~3u, khi = (s1 + 3) & ~3u;
        fence_proxy_async_smem();  // earlier reads and writes of the buffer come before the copy's writes
        mbar_arrive_expect_tx(&s_bar[b], (khi - klo) * 4);
        if (khi > klo) bulk_load(s_buf0 + b * SB_BUF_KEYS, in + klo, (khi - klo) * 4, &s_bar[b]);
    };
    if (tid == 0) {
        mbar_init(&s_bar[0], 1);
        mbar_init(&s_bar[1], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        for (int b = 0; b < 2; ++b) {
            const uint32_t it = blockIdx.x + b * G;
            const uint32_t p = it < n_small ? __ldg(work + n_big + it) : ~0u;
            start_copy(b, p, p != ~0u ? __ldg(bin_start + p) : 0u, p != ~0u ? __ldg(bin_start + p + 1) : 0u);
        }
    }
#pragma unroll
    for (int c = 0; c < 4; ++c) *reinterpret_cast<uint4*>(s_cnt0 + 16 * tid + 4 * c) = make_uint4(0, 0, 0, 0);
    __syncthreads();
    uint32_t parity = 0;  // bit b: the phase buffer b's barrier completes next
    bool failed = false, bad = false;
    int b = 0;
    for (uint32_t it = blockIdx.x; it < n_small; it += G, b ^= 1) {
        const uint32_t p = s_bin[b];
        const uint32_t s0 = s_lo[b], s1 = s_hi[b];
        uint32_t* const s_cnt = s_cnt0 + b * BPB;
        // (thread 0) the next bin but one: its number now, its range after the histogram
        const uint32_t it1 = it + G;
        uint32_t p1 = ~0u, lo1 = 0, hi1 = 0;
        if (tid == 0 && it > blockIdx.x && it1 < n_small) p1 = __ldg(work + n_big + it1);
        const bool ok = s1 - s0 <= SB_CAP;
        bad |= !ok;  // (inconsistent plan: nothing was copied)
        if (ok) {
            uint32_t polls = 0;
            while (!mbar_test_parity(&s_bar[b], (parity >> b) & 1u) && ++polls < SB_WAIT_LIMIT) {
            }
            failed |= polls >= SB_WAIT_LIMIT;
            parity ^= 1u << b;
        }
        const uint32_t nk = ok ? s1 - s0 : 0u;
        const uint32_t klo = s0 & ~3u;
        const uint32_t a = s0 - klo;           // the bin's first key sits at buffer index a
        const uint32_t nv = (a + nk + 3) / 4;  // 16-byte groups holding the bin
        uint32_t* buf = s_buf0 + b * SB_BUF_KEYS;
        const uint32_t b0 = p << BIN_SHIFT;
        const uint32_t nb = POW2 ? BPB : (uint32_t)min((uint64_t)BPB, H.B - b0);
        // histogram.  Thread t reads 16-byte groups t, t + 1024, ...; each key's
        // rank among the bin's keys of its bucket is the value its histogram
        // increment returns, kept in registers for the placement, two per word
        // (16 bits each: ranks are below SB_CAP; 0xffff = not a key of the bin).
        // (groups past the thread's last are skipped by a branch, which is the
        // same for all lanes of a warp but the last one: no predicated-off work.
        // A copy that timed out leaves the buffer's old words, read here in
        // bounds; the CTA then leaves at the barrier below.)
        const uint32_t ng = nv > tid ? (nv - tid + SB_THREADS - 1) / SB_THREADS : 0u;
        uint32_t key[SB_KPT], rk[2 * GR];
#pragma unroll
        for (int g = 0; g < GR; ++g) {
            if ((uint32_t)g >= ng) break;
            const uint32_t v = tid + (uint32_t)g * SB_THREADS;
            {
                const uint4 x = reinterpret_cast<const uint4*>(buf)[v];
                key[4 * g] = x.x;
                key[4 * g + 1] = x.y;
                key[4 * g + 2] = x.z;
                key[4 * g + 3] = x.w;
                uint32_t js[4];
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    const bool in_bin = 4 * v + e - a < nk;
                    // the words are the keys' hashes (the partition passes' output)
                    const uint32_t h = key[4 * g + e];
                    uint32_t j;
                    if (POW2) {  // B = 2^k >= BPB: the bucket's low bits are its place in the bin
                        j = h & (BPB - 1);
                        bad |= in_bin && ((h & (uint32_t)H.mask) >> BIN_SHIFT) != p;
                    } else {
                        j = bucket_of_hash(h, H) - b0;
                        bad |= in_bin && j >= nb;
                        j = min(j, nb - 1);
                    }
                    js[e] = in_bin ? atomicAdd(s_cnt + j, 1u) : 0xffffu;
                }
                rk[2 * g] = js[0] | (js[1] << 16);
                rk[2 * g + 1] = js[2] | (js[3] << 16);
            }
        }
        if (tid == 0 && p1 != ~0u) {
            lo1 = __ldg(bin_start + p1);
            hi1 = __ldg(bin_start + p1 + 1);
        }
        if (__syncthreads_or(failed)) {
            failed = true;
            break;
        }
        // every thread is past the previous bin: its buffer takes the next bin
        if (tid == 0 && it > blockIdx.x) start_copy(b ^ 1, p1, lo1, hi1);
        // exclusive scan of the bin's counts: thread t owns buckets [8t, 8t + 8)
        const uint32_t j0 = 8 * tid;
        const uint4 c0 = *reinterpret_cast<const uint4*>(s_cnt + j0);
        const uint4 c1 = *reinterpret_cast<const uint4*>(s_cnt + j0 + 4);
        const uint32_t cv[8] = {c0.x, c0.y, c0.z, c0.w, c1.x, c1.y, c1.z, c1.w};
        uint32_t tsum = 0;
#pragma unroll
        for (int e = 0; e < 8; ++e) tsum += cv[e];
        const uint32_t winc = warp_inclusive_scan(tsum);
        if (lane == 31) s_wsum[w] = winc;
        __syncthreads();
        // every warp takes its prefix from the 32 warp sums itself (no second barrier)
        const uint32_t xw = s_wsum[lane];
        const uint32_t wpre = __shfl_sync(FULL_MASK, warp_inclusive_scan(xw) - xw, w);
        uint32_t st[8];
        st[0] = wpre + winc - tsum;
#pragma unroll
        for (int e = 1; e < 8; ++e) st[e] = st[e - 1] + cv[e - 1];
        if (ok) {
            if (POW2 || j0 + 8 <= nb) {
                uint4* o = reinterpret_cast<uint4*>(offsets + b0 + j0);
                o[0] = make_uint4(s0 + st[0], s0 + st[1], s0 + st[2], s0 + st[3]);
                o[1] = make_uint4(s0 + st[4], s0 + st[5], s0 + st[6], s0 + st[7]);
            } else {
#pragma unroll
                for (int e = 0; e < 8; ++e)
                    if (j0 + e < nb) offsets[b0 + j0 + e] = s0 + st[e];
            }
        }
        if (LONGS && nk > SUM_MIN_LEN) {
#pragma unroll
            for (int e = 0; e < 8; ++e)
                if (cv[e] > SUM_MIN_LEN) note_long(LF, b0 + j0 + e);
        }
        // bucket starts, as buffer indices
        *reinterpret_cast<uint4*>(s_cnt + j0) = make_uint4(a + st[0], a + st[1], a + st[2], a + st[3]);
        *reinterpret_cast<uint4*>(s_cnt + j0 + 4) = make_uint4(a + st[4], a + st[5], a + st[6], a + st[7]);
        __syncthreads();
        // placement into the same buffer (every word is in registers now): the
        // bucket's start plus the key's rank, no atomics; the bucket comes again
        // from the word (POW2: its low bits)
#pragma unroll
        for (int g = 0; g < GR; ++g) {
            if ((uint32_t)g >= ng) break;
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const uint32_t r = (rk[2 * g + e / 2] >> (16 * (e & 1))) & 0xffffu;
                if (r != 0xffffu) {
                    const uint32_t h = key[4 * g + e];
                    const uint32_t j = POW2 ? h & (BPB - 1) : min((uint32_t)(bucket_of_hash(h, H) - b0), nb - 1);
                    const uint32_t pos = s_cnt[j] + r;
                    bad |= pos - a >= nk;
                    if (pos < SB_BUF_KEYS) buf[pos] = h;
                }
            }
        }
        __syncthreads();
        // the sorted bin out as keys (the words are hashes: fmix32_inv undoes them):
        // 16-byte stores for the aligned body, single keys at the edges.  The
        // counters are cleared for the bin after next; no barrier ends the bin:
        // the next bin's first barrier orders this buffer's reuse
        if (ok) {
            const uint32_t v0 = (s0 + 3) & ~3u, v1 = s1 & ~3u;  // aligned body [v0, v1) (empty if v1 <= v0)
            if (v1 > v0) {
                const uint32_t nvec = (v1 - v0) / 4;
                const uint4* src = reinterpret_cast<const uint4*>(buf + (v0 - klo));
                uint4* dst = reinterpret_cast<uint4*>(out + v0);
                for (uint32_t v = tid; v < nvec; v += SB_THREADS) {
                    const uint4 x = src[v];
                    dst[v] = make_uint4(unhash_key32(x.x, H), unhash_key32(x.y, H), unhash_key32(x.z, H),
                                        unhash_key32(x.w, H));
                }
                if (tid < v0 - s0) out[s0 + tid] = unhash_key32(buf[a + tid], H);
                if (tid < s1 - v1) out[v1 + tid] = unhash_key32(buf[(v1 - klo) + tid], H);
            } else if (tid < nk) {
                out[s0 + tid] = unhash_key32(buf[a + tid], H);
            }
        }
        *reinterpret_cast<uint4*>(s_cnt + j0) = make_uint4(0, 0, 0, 0);
        *reinterpret_cast<uint4*>(s_cnt + j0 + 4) = make_uint4(0, 0, 0, 0);
    }
    if (bad) atomicOr(err, DEVERR_BOUNDS);
    if (failed && tid == 0) {
        atomicOr(err, DEVERR_TIMEOUT);
        // let the copies this CTA started finish (bounded) before it leaves
        for (int c = 0; c < 2; ++c) {
            if (s_bin[c] == ~0u || s_hi[c] - s_lo[c] > SB_CAP) continue;
            uint32_t polls = 0;
            while (!mbar_test_parity(&s_bar[c], (parity >> c) & 1u) && ++polls < SB_WAIT_LIMIT) {
            }
        }
    }
}

// Work items of the bins of more than SB_CAP 32-bit keys (no values): chunks of
// SB_CAP words, their buckets pre-counted (k_huge_count) and turned into
// offsets and per-bucket cursors (k_huge_scan).  Each CTA takes chunks
// blockIdx.x, blockIdx.x + G, ... whose words arrive by bulk copies (TMA) two
// chunks ahead, as in k_bin_small; per chunk: a shared-memory histogram, one
// global atomic per nonempty bucket to reserve the chunk's run in it, and each
// key written at its place.  These bins hold the most duplicated keys: the
// lanes of a warp whose keys fall in the chunk's fullest bucket share one
// atomic, and their keys go out as consecutive words.
constexpr uint32_t MAX_HUGE_SB = 1536;  // bins of more than SB_CAP keys with a counter/cursor slice

// Step 1 for the chunks of k_big_place: each chunk's bucket histogram (shared
// memory), added into its bin's global counts; chunks arrive as in k_big_place.
template <bool POW2>
__global__ void __launch_bounds__(SB_THREADS, 1)
k_big_count(const uint32_t* __restrict__ in, Hasher H, const uint4* __restrict__ item_meta,
            const Plan* __restrict__ plan, uint32_t* __restrict__ huge_count, uint32_t* __restrict__ item_hot,
            uint32_t* err) {
    extern __shared__ __align__(16) unsigned char smem[];
    uint32_t* s_cnt = reinterpret_cast<uint32_t*>(smem);
    uint32_t* const s_buf0 = s_cnt + BPB;  // buffer b at s_buf0 + b * SB_BUF_KEYS
    __shared__ __align__(8) uint64_t s_bar[2];
    __shared__ uint32_t s_e[2], s_p[2], s_lo[2], s_hi[2], s_wmax[SB_THREADS / 32];
    const uint32_t tid = threadIdx.x;
    const uint32_t items = plan->huge_chunks;
    const uint32_t G = gridDim.x;
    auto start_copy = [&](int b, uint4 m) {
        const uint32_t e = m.x, p = m.y, lo = m.z, hi = m.w;
        s_e[b] = e;
        s_p[b] = p;
        s_lo[b] = lo;
        s_hi[b] = hi;
        if (e == ~0u || hi - lo > SB_CAP) return;
        const uint32_t klo = lo & ~3u, khi = (hi + 3) & ~3u;
        fence_proxy_async_smem();
        mbar_arrive_expect_tx(&s_bar[b], (khi - klo) * 4);
        if (khi > klo) bulk_load(s_buf0 + b * SB_BUF_KEYS, in + klo, (khi - klo) * 4, &s_bar[b]);
    };
    if (tid == 0) {
        mbar_init(&s_bar[0], 1);
        mbar_init(&s_bar[1], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        const uint4 none = make_uint4(~0u, 0, 0, 0);
        start_copy(0, blockIdx.x < items ? item_meta[blockIdx.x] : none);
        start_copy(1, blockIdx.x + G < items ? item_meta[blockIdx.x + G] : none);
    }
    *reinterpret_cast<uint4*>(s_cnt + 8 * tid) = make_uint4(0, 0, 0, 0);
    *reinterpret_cast<uint4*>(s_cnt + 8 * tid + 4) = make_uint4(0, 0, 0, 0);
    __syncthreads();
    uint32_t parity = 0;
    bool failed = false, bad = false;
    int b = 0;
    for (uint32_t it = blockIdx.x; it < items; it += G, b ^= 1) {
        const uint32_t e = s_e[b], p = s_p[b], s0 = s_lo[b], s1 = s_hi[b];
        uint4 m2 = make_uint4(~0u, 0, 0, 0);
        if (tid == 0 && it + 2 * G < items) m2 = item_meta[it + 2 * G];
        const bool ok = e != ~0u && s1 - s0 <= SB_CAP;
        bad |= !ok;
        if (ok) {
            uint32_t polls = 0;
            while (!mbar_test_parity(&s_bar[b], (parity >> b) & 1u) && ++polls < SB_WAIT_LIMIT) {
            }
            failed = polls >= SB_WAIT_LIMIT;
            parity ^= 1u << b;
        }
        if (__syncthreads_or(failed)) {
            failed = true;
            break;
        }
        const uint32_t nk = ok ? s1 - s0 : 0u;
        const uint32_t klo = s0 & ~3u, a = s0 - klo, nv = (a + nk + 3) / 4;
        const uint32_t* buf = s_buf0 + b * SB_BUF_KEYS;
        const uint32_t b0 = p << BIN_SHIFT;
        const uint32_t nb = POW2 ? BPB : (uint32_t)min((uint64_t)BPB, H.B - b0);
        for (uint32_t v = tid; v < nv; v += SB_THREADS) {
            const uint4 x = reinterpret_cast<const uint4*>(buf)[v];
            const uint32_t hw[4] = {x.x, x.y, x.z, x.w};
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                if (4 * v + u - a < nk) {
                    uint32_t j;
                    if (POW2) {
                        j = hw[u] & (BPB - 1);
                    } else {
                        j = bucket_of_hash(hw[u], H) - b0;
                        bad |= j >= nb;
                        j = min(j, nb - 1);
                    }
                    atomicAdd(s_cnt + j, 1u);
                }
            }
        }
        __syncthreads();
        // flush: thread t adds its 8 buckets' nonzero counts into the bin's, and
        // clears them; the chunk's fullest bucket is recorded for k_big_place
        const uint32_t j0 = 8 * tid;
        {
            const uint4 c0 = *reinterpret_cast<const uint4*>(s_cnt + j0);
            const uint4 c1 = *reinterpret_cast<const uint4*>(s_cnt + j0 + 4);
            const uint32_t cv[8] = {c0.x, c0.y, c0.z, c0.w, c1.x, c1.y, c1.z, c1.w};
            uint32_t cmax = 0;
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                if (cv[u]) atomicAdd(huge_count + (uint64_t)e * BPB + j0 + u, cv[u]);
                cmax = max(cmax, (cv[u] << BIN_SHIFT) | (j0 + u));
            }
            *reinterpret_cast<uint4*>(s_cnt + j0) = make_uint4(0, 0, 0, 0);
            *reinterpret_cast<uint4*>(s_cnt + j0 + 4) = make_uint4(0, 0, 0, 0);
            cmax = __reduce_max_sync(FULL_MASK, cmax);
            if (lane_id() == 0) s_wmax[tid >> 5] = cmax;
        }
        __syncthreads();
        if (tid < 32) {
            const uint32_t m = __reduce_max_sync(FULL_MASK, s_wmax[tid]);
            if (tid == 0 && ok) item_hot[it] = m & (BPB - 1);
        }
        if (tid == 0) start_copy(b, m2);
    }
    if (bad) atomicOr(err, DEVERR_BOUNDS);
    if (failed && tid == 0) {
        atomicOr(err, DEVERR_TIMEOUT);
        for (int c = 0; c < 2; ++c) {
            if (s_e[c] == ~0u || s_hi[c] - s_lo[c] > SB_CAP) continue;
            uint32_t polls = 0;
            while (!mbar_test_parity(&s_bar[c], (parity >> c) & 1u) && ++polls < SB_WAIT_LIMIT) {
            }
        }
    }
}

template <bool POW2>
__global__ void __launch_bounds__(SB_THREADS, 1)
k_big_place(const uint32_t* __restrict__ in, Hasher H, const uint4* __restrict__ item_meta,
            const uint32_t* __restrict__ item_hot, const Plan* __restrict__ plan, uint32_t* __restrict__ huge_cursor,
            uint64_t n, uint32_t* __restrict__ out, uint32_t* err) {
    constexpr int GR = SB_KPT / 4;
    extern __shared__ __align__(16) unsigned char smem[];
    uint32_t* s_cnt = reinterpret_cast<uint32_t*>(smem);
    uint32_t* const s_buf0 = s_cnt + BPB;  // buffer b at s_buf0 + b * SB_BUF_KEYS
    __shared__ __align__(8) uint64_t s_bar[2];
    __shared__ uint32_t s_e[2], s_p[2], s_lo[2], s_hi[2], s_hot[2];
    const uint32_t tid = threadIdx.x, lane = lane_id(), w = tid >> 5;
    const uint32_t items = plan->huge_chunks;
    const uint32_t G = gridDim.x;
    const uint32_t nn = (uint32_t)min(n, (uint64_t)0xffffffffu);

    // thread 0: chunk (e, p, lo, hi) with its fullest bucket jh into buffer b
    // (e = ~0u: none); its description is read one chunk ahead, so no phase waits on it
    auto start_copy = [&](int b, uint4 m, uint32_t jh) {
        const uint32_t e = m.x, p = m.y, lo = m.z, hi = m.w;
        s_e[b] = e;
        s_p[b] = p;
        s_lo[b] = lo;
        s_hi[b] = hi;
        s_hot[b] = jh;
        if (e == ~0u || hi - lo > SB_CAP) return;  // none left / inconsistent plan (flagged by the CTA)
        const uint32_t klo = lo & ~3u, khi = (hi + 3) & ~3u;
        fence_proxy_async_smem();
        mbar_arrive_expect_tx(&s_bar[b], (khi - klo) * 4);
        if (khi > klo) bulk_load(s_buf0 + b * SB_BUF_KEYS, in + klo, (khi - klo) * 4, &s_bar[b]);
    };
    if (tid == 0) {
        mbar_init(&s_bar[0], 1);
        mbar_init(&s_bar[1], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        const uint4 none = make_uint4(~0u, 0, 0, 0);
        const uint32_t i1 = blockIdx.x + G;
        start_copy(0, blockIdx.x < items ? item_meta[blockIdx.x] : none, blockIdx.x < items ? item_hot[blockIdx.x] : 0u);
        start_copy(1, i1 < items ? item_meta[i1] : none, i1 < items ? item_hot[i1] : 0u);
    }
    *reinterpret_cast<uint4*>(s_cnt + 8 * tid) = make_uint4(0, 0, 0, 0);
    *reinterpret_cast<uint4*>(s_cnt + 8 * tid + 4) = make_uint4(0, 0, 0, 0);
    __syncthreads();
    uint32_t parity = 0;
    bool failed = false, bad = false;
    int b = 0;
    for (uint32_t it = blockIdx.x; it < items; it += G, b ^= 1) {
        const uint32_t e = s_e[b], p = s_p[b], s0 = s_lo[b], s1 = s_hi[b], jh = s_hot[b] & (BPB - 1);
        uint4 m2 = make_uint4(~0u, 0, 0, 0);  // (thread 0) the chunk after next
        uint32_t jh2 = 0;
        if (tid == 0 && it + 2 * G < items) {
            m2 = item_meta[it + 2 * G];
            jh2 = item_hot[it + 2 * G];
        }
        const bool ok = e != ~0u && s1 - s0 <= SB_CAP;
        bad |= !ok;
        if (ok) {
            uint32_t polls = 0;
            while (!mbar_test_parity(&s_bar[b], (parity >> b) & 1u) && ++polls < SB_WAIT_LIMIT) {
            }
            failed = polls >= SB_WAIT_LIMIT;
            parity ^= 1u << b;
        }
        if (__syncthreads_or(failed)) {
            failed = true;
            break;
        }
        const uint32_t nk = ok ? s1 - s0 : 0u;
        const uint32_t klo = s0 & ~3u, a = s0 - klo, nv = (a + nk + 3) / 4;
        const uint32_t* buf = s_buf0 + b * SB_BUF_KEYS;
        const uint32_t b0 = p << BIN_SHIFT;
        const uint32_t nb = POW2 ? BPB : (uint32_t)min((uint64_t)BPB, H.B - b0);
        const uint32_t ng = nv > tid ? (nv - tid + SB_THREADS - 1) / SB_THREADS : 0u;
        uint32_t key[SB_KPT], rk[2 * GR];
        // histogram of the chunk's buckets (the words are the keys' hashes); each
        // key's rank in its bucket is what its increment returns (16 bits per key,
        // 0xffff = not a key of the chunk).  These bins hold the most duplicated
        // keys: the lanes of a warp whose keys fall in the chunk's fullest bucket
        // jh (counted by k_big_count) share one increment.
#pragma unroll
        for (int g = 0; g < GR; ++g) {
            if ((uint32_t)g >= ng) break;
            const uint32_t v = tid + (uint32_t)g * SB_THREADS;
            // the lanes of this warp that hold group g: those with tid + g * SB_THREADS < nv
            const uint32_t first_v = g * SB_THREADS + w * 32;
            const unsigned act = nv - first_v >= 32 ? FULL_MASK : (1u << (nv - first_v)) - 1u;
            const uint4 x = reinterpret_cast<const uint4*>(buf)[v];
            key[4 * g] = x.x;
            key[4 * g + 1] = x.y;
            key[4 * g + 2] = x.z;
            key[4 * g + 3] = x.w;
            uint32_t rs[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const bool in_bin = 4 * v + u - a < nk;
                const uint32_t h = key[4 * g + u];
                uint32_t j;
                if (POW2) {
                    j = h & (BPB - 1);
                    bad |= in_bin && ((h & (uint32_t)H.mask) >> BIN_SHIFT) != p;
                } else {
                    j = bucket_of_hash(h, H) - b0;
                    bad |= in_bin && j >= nb;
                    j = min(j, nb - 1);
                }
                const bool hot = in_bin && j == jh;
                const unsigned hm = __ballot_sync(act, hot);
                uint32_t r = 0xffffu;
                if (hot) {
                    const int leader = __ffs(hm) - 1;
                    uint32_t base = 0;
                    if ((int)lane == leader) base = atomicAdd(s_cnt + jh, (uint32_t)__popc(hm));
                    r = __shfl_sync(hm, base, leader) + __popc(hm & lanemask_lt());
                } else if (in_bin) {
                    r = atomicAdd(s_cnt + j, 1u);
                }
                rs[u] = r;
            }
            rk[2 * g] = rs[0] | (rs[1] << 16);
            rk[2 * g + 1] = rs[2] | (rs[3] << 16);
        }
        __syncthreads();
        // reserve the chunk's run in every bucket it touches; thread t owns buckets [8t, 8t + 8)
        const uint32_t j0 = 8 * tid;
        {
            const uint4 c0 = *reinterpret_cast<const uint4*>(s_cnt + j0);
            const uint4 c1 = *reinterpret_cast<const uint4*>(s_cnt + j0 + 4);
            const uint32_t cv[8] = {c0.x, c0.y, c0.z, c0.w, c1.x, c1.y, c1.z, c1.w};
            uint32_t base[8];
#pragma unroll
            for (int u = 0; u < 8; ++u)
                base[u] = cv[u] ? atomicAdd(huge_cursor + (uint64_t)e * BPB + j0 + u, cv[u]) : 0u;
            *reinterpret_cast<uint4*>(s_cnt + j0) = make_uint4(base[0], base[1], base[2], base[3]);
            *reinterpret_cast<uint4*>(s_cnt + j0 + 4) = make_uint4(base[4], base[5], base[6], base[7]);
        }
        __syncthreads();
        // place every key at its bucket's run plus its rank (keys again from their
        // hashes; the bucket again from the word); a warp's keys of the fullest
        // bucket have consecutive ranks, so they go out as consecutive words
#pragma unroll
        for (int g = 0; g < GR; ++g) {
            if ((uint32_t)g >= ng) break;
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const uint32_t r = (rk[2 * g + u / 2] >> (16 * (u & 1))) & 0xffffu;
                if (r != 0xffffu) {
                    const uint32_t h = key[4 * g + u];
                    const uint32_t j = POW2 ? h & (BPB - 1) : min((uint32_t)(bucket_of_hash(h, H) - b0), nb - 1);
                    const uint32_t pos = s_cnt[j] + r;
                    if (pos < nn) out[pos] = unhash_key32(h, H);
                    else bad = true;
                }
            }
        }
        __syncthreads();
        *reinterpret_cast<uint4*>(s_cnt + j0) = make_uint4(0, 0, 0, 0);
        *reinterpret_cast<uint4*>(s_cnt + j0 + 4) = make_uint4(0, 0, 0, 0);
        __syncthreads();
        if (tid == 0) start_copy(b, m2, jh2);  // the chunk after next, into this buffer
    }
    if (bad) atomicOr(err, DEVERR_BOUNDS);
    if (failed && tid == 0) {
        atomicOr(err, DEVERR_TIMEOUT);
        for (int c = 0; c < 2; ++c) {
            if (s_e[c] == ~0u || s_hi[c] - s_lo[c] > SB_CAP) continue;
            uint32_t polls = 0;
            while (!mbar_test_parity(&s_bar[c], (parity >> c) & 1u) && ++polls < SB_WAIT_LIMIT) {
            }
        }
    }
}

size_t local_smem_bytes(size_t key_bytes, bool hv) {
    const size_t cap = LOCAL_STAGE_BYTES / (key_bytes + (hv ? 4 : 0));
    return (size_t)BPB * 4 + BPB / 8 + 2 * MAX_HOT * 4 + cap * (key_bytes + (hv ? 4 : 0));
}

template <typename K>
size_t pass_smem_bytes(bool payload) {
    constexpr int TILE = PassCfg<K>::TILE;
    // u32 keys: (key, destination) pairs; u64 keys: keys then destinations
    return (size_t)TILE * 8 + (sizeof(K) == 4 ? 0 : (size_t)TILE * 4) + (payload ? (size_t)TILE * 4 : 0);
}

template <typename Kern>
unsigned grid_for(Kern kern, int threads, size_t smem) {
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, smem) != cudaSuccess || per_sm < 1)
        per_sm = 1;
    return (unsigned)(num_sms() * per_sm);
}

// One partition pass.  32-bit keys take k_pass32 (HIN: the input is already
// hashes; the output always is), 64-bit keys k_pass_down.  DR: record what the
// reverse passes need (query grouping).
template <typename K, int PM, bool HIN = false, bool DR = false>
cudaError_t launch_down(const K* in, const uint32_t* in_v, uint64_t n, const Hasher& H, uint32_t dig_shift,
                        uint32_t dig_mask, uint32_t R, const ChunkMap& cm, uint32_t nch_host, uint32_t grid,
                        const Plan* plan, const uint32_t* base, K* out, uint32_t* out_v, uint32_t* err,
                        cudaStream_t s, const char* name = "part_scatter", uint32_t* dr = nullptr,
                        uint2* lb = nullptr, bool in_padded = false) {
    cudaError_t e;
    if constexpr (sizeof(K) == 4) {
        auto kern = H.mode == MODE_POW2 ? k_pass32<HIN, PM, DR, true> : k_pass32<HIN, PM, DR, false>;
        const size_t smem = (size_t)P32<PM>::TILE * (PM ? 8 : 4);
        e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        launch_begin(name, s);
        kern<<<grid, P32_THREADS, smem, s>>>(in, in_v, n, H, dig_shift, dig_mask, R, cm, nch_host, plan, base, out,
                                             out_v, err, dr, lb, in_padded ? 1u : 0u);
        launch_end(name, s);
    } else {
        static_assert(!HIN, "64-bit keys are never passed as hashes");
        auto kern = k_pass_down<K, PM, DR>;
        const size_t smem = pass_smem_bytes<K>(PM != 0);
        e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        launch_begin(name, s);
        kern<<<grid, PASS_THREADS, smem, s>>>(in, in_v, n, H, dig_shift, dig_mask, R, cm, nch_host, plan, base, out,
                                              out_v, err, dr, lb);
        launch_end(name, s);
    }
    return cudaGetLastError();
}

template <typename K>
cudaError_t build_partitioned_impl(Table& t, const K* keys, const uint32_t* vals, cudaStream_t s) {
    const uint64_t n = t.n, B = t.B;
    const uint32_t P = (uint32_t)((B + BPB - 1) / BPB);
    const uint32_t P2 = P <= RADIX ? P : RADIX;
    const uint32_t P1 = (P + P2 - 1) / P2;
    const bool two = P1 > 1;
    const bool hv = t.has_values != 0;
    const uint32_t nch_a = (uint32_t)((n + CHUNK - 1) / CHUNK);
    const uint32_t nch_b_max = nch_a + P1 + 1;
    // first pass digit: bin >> 7 (two passes) or the bin itself (one pass, P <= 128)
    const uint32_t shift1 = two ? 7u : 0u;
    const uint32_t R1 = two ? P1 : P;
    // 32-bit keys without values: bins of at most SB_CAP keys go to k_bin_small,
    // larger ones (up to MAX_HUGE_SB of them) are cut into SB_CAP-key chunks for
    // k_big_place; otherwise bins of more than HUGE_T_BUILD keys (up to MAX_HUGE)
    // are cut into HUGE_CHUNK-key chunks for k_bin_local
    const bool small_path = sizeof(K) == 4 && !hv;
    const uint32_t huge_t = small_path ? SB_CAP : HUGE_T_BUILD;
    const uint32_t huge_chunk = small_path ? SB_CAP : HUGE_CHUNK;
    const uint32_t max_huge = small_path ? MAX_HUGE_SB : MAX_HUGE;
    const size_t max_items = small_path ? (size_t)(n / SB_CAP) + max_huge + 1 : 0;

    // scratch (zeroed part first): bin_count[P] | huge_count | counters
    //   | cnt_a[nch_a][RADIX] | cnt_b[nch_b_max][RADIX] | bin_start[P+1] | work[P]
    //   | seg_chunk_start[P1+1] | huge_bin | huge_chunk_start | plan | huge_cursor
    //   | tmpA keys | tmpA vals | tmpB keys | tmpB vals
    auto al = [](size_t x) { return (x + 255) & ~size_t(255); };
    size_t off = 0;
    const size_t o_cnt = off; off += al((size_t)P * 4);
    const size_t o_hcount = off; off += al((size_t)max_huge * BPB * 4);
    const size_t o_ctr = off; off += al(64);
    const size_t zero_bytes = off;
    const size_t o_ca = off; off += al((size_t)nch_a * RADIX * 4);
    const size_t o_cb = off; off += al(two ? (size_t)nch_b_max * RADIX * 4 : 0);
    const size_t o_pref = off; off += al((size_t)nch_b_max * RADIX * 4);
    const size_t o_start = off; off += al((size_t)(P + 1) * 4);
    const size_t o_work = off; off += al((size_t)P * 4);
    const size_t o_seg = off; off += al((size_t)(P1 + 1) * 4);
    const size_t o_hbin = off; off += al((size_t)max_huge * 4);
    const size_t o_hcs = off; off += al((size_t)(max_huge + 1) * 4);
    const size_t o_plan = off; off += al(sizeof(Plan));
    const size_t o_hcur = off; off += al((size_t)max_huge * BPB * 4);
    const size_t o_items = off; off += al(max_items * sizeof(uint4));
    const size_t o_ihot = off; off += al(max_items * 4);
    const size_t o_ka = off; off += al(two ? n * sizeof(K) : 0);
    const size_t o_va = off; off += al(two && hv ? n * 4 : 0);
    const size_t o_kb = off; off += al(n * sizeof(K));
    const size_t o_vb = off; off += al(hv ? n * 4 : 0);
    void* mem = nullptr;
    cudaError_t e = dev_alloc(&mem, off, s);
    if (e != cudaSuccess) return e;
    char* base = static_cast<char*>(mem);
    uint32_t* bin_count = reinterpret_cast<uint32_t*>(base + o_cnt);
    uint32_t* huge_count = reinterpret_cast<uint32_t*>(base + o_hcount);
    uint32_t* ctr = reinterpret_cast<uint32_t*>(base + o_ctr);  // [0] local-stage work counter
    uint32_t* cnt_a = reinterpret_cast<uint32_t*>(base + o_ca);
    uint32_t* cnt_b = reinterpret_cast<uint32_t*>(base + o_cb);
    uint32_t* pref = reinterpret_cast<uint32_t*>(base + o_pref);
    uint32_t* bin_start = reinterpret_cast<uint32_t*>(base + o_start);
    uint32_t* work = reinterpret_cast<uint32_t*>(base + o_work);
    uint32_t* seg = reinterpret_cast<uint32_t*>(base + o_seg);
    uint32_t* huge_bin = reinterpret_cast<uint32_t*>(base + o_hbin);
    uint32_t* huge_cs = reinterpret_cast<uint32_t*>(base + o_hcs);
    Plan* plan = reinterpret_cast<Plan*>(base + o_plan);
    uint32_t* huge_cursor = reinterpret_cast<uint32_t*>(base + o_hcur);
    uint4* item_meta = reinterpret_cast<uint4*>(base + o_items);
    uint32_t* item_hot = reinterpret_cast<uint32_t*>(base + o_ihot);  // each chunk's fullest bucket
    K* ka = reinterpret_cast<K*>(base + o_ka);
    uint32_t* va = reinterpret_cast<uint32_t*>(base + o_va);
    K* kb = reinterpret_cast<K*>(base + o_kb);
    uint32_t* vb = reinterpret_cast<uint32_t*>(base + o_vb);

    ChunkMap cm_a{false, n, P, P2, 1u, bin_start, nullptr};
    ChunkMap cm_b{true, n, P, P2, P1, bin_start, seg};

    e = cudaMemsetAsync(base, 0, zero_bytes, s);
    // 1. bin histogram + first-pass chunk counts
    if (e == cudaSuccess) {
        auto kern = k_part_count<K, true>;
        const size_t smem = (size_t)P * 4;
        e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e == cudaSuccess) {
            unsigned g = grid_for(kern, PASS_THREADS, smem);
            if (g > nch_a) g = nch_a;
            launch_begin("part_hist", s);
            kern<<<g, PASS_THREADS, smem, s>>>(keys, n, t.H, P, shift1, R1, nch_a, bin_count, cnt_a, nullptr);
            launch_end("part_hist", s);
            e = cudaGetLastError();
        }
    }
    // 32-bit keys move through the passes as their hashes (k_pass32), so every
    // kernel after the first pass reads hashes
    constexpr bool HASHED = sizeof(K) == 4;
    // 2. plan
    if (e == cudaSuccess) {
        const uint32_t big_t = small_path ? SB_CAP : (uint32_t)(LOCAL_STAGE_BYTES / (sizeof(K) + (hv ? 4 : 0)));
        launch_begin("part_plan", s);
        k_part_plan<<<1, 1024, 0, s>>>(bin_count, P, P1, P2, n, big_t, huge_t, huge_chunk, max_huge, bin_start, seg,
                                       work, huge_bin, huge_cs, plan, t.offsets, B);
        launch_end("part_plan", s);
        e = cudaGetLastError();
    }
    // 3a. first pass: chunk bases, then the downsweep
    if (e == cudaSuccess) {
        launch_begin("chunk_scan", s);
        k_chunk_scan<<<RADIX, 1024, 0, s>>>(cnt_a, pref, cm_a, nch_a, plan, R1, two ? P2 : 1u, nullptr);
        launch_end("chunk_scan", s);
        e = cudaGetLastError();
    }
    const int pm_first = vals ? 1 : (hv ? 2 : 0);
    K* out1 = two ? ka : kb;
    uint32_t* out1_v = two ? va : vb;
    if (e == cudaSuccess) {
        const uint32_t mask = 0xffffffffu;
        if (pm_first == 1)
            e = launch_down<K, 1>(keys, vals, n, t.H, shift1, mask, R1, cm_a, nch_a, nch_a, plan, cnt_a, out1, out1_v,
                                  t.err, s);
        else if (pm_first == 2)
            e = launch_down<K, 2>(keys, nullptr, n, t.H, shift1, mask, R1, cm_a, nch_a, nch_a, plan, cnt_a, out1,
                                  out1_v, t.err, s);
        else
            e = launch_down<K, 0>(keys, nullptr, n, t.H, shift1, mask, R1, cm_a, nch_a, nch_a, plan, cnt_a, out1,
                                  nullptr, t.err, s);
    }
    // 3b. second pass (bins inside each coarse segment)
    if (e == cudaSuccess && two) {
        launch_begin("chunk_count", s);
        k_chunk_count<K, HASHED><<<nch_b_max, PASS_THREADS, 0, s>>>(ka, t.H, cm_b, plan, cnt_b);
        launch_end("chunk_count", s);
        e = cudaGetLastError();
        if (e == cudaSuccess) {
            launch_begin("chunk_scan", s);
            k_chunk_scan<<<RADIX, 1024, 0, s>>>(cnt_b, pref, cm_b, 0u, plan, P2, 1u, nullptr);
            launch_end("chunk_scan", s);
            e = cudaGetLastError();
        }
        if (e == cudaSuccess) {
            if (hv)
                e = launch_down<K, 1, HASHED>(ka, va, n, t.H, 0, RADIX - 1, P2, cm_b, 0u, nch_b_max, plan, cnt_b, kb,
                                              vb, t.err, s, "part_scatter2", nullptr, nullptr, true);
            else
                e = launch_down<K, 0, HASHED>(ka, nullptr, n, t.H, 0, RADIX - 1, P2, cm_b, 0u, nch_b_max, plan, cnt_b,
                                              kb, nullptr, t.err, s, "part_scatter2", nullptr, nullptr, true);
        }
    }
    // 4. huge bins: chunk histograms, then their offsets and cursors
    if (e == cudaSuccess && small_path) {
        // the chunks as (bin slot, bin, first key, end key), then their counts by TMA-fed CTAs
        launch_begin("huge_items", s);
        k_huge_items<<<max_huge, 256, 0, s>>>(bin_start, huge_bin, huge_cs, plan, item_meta);
        launch_end("huge_items", s);
        e = cudaGetLastError();
        auto run = [&](auto kern) {
            cudaError_t r = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SB_SMEM);
            if (r != cudaSuccess) return r;
            launch_begin("huge_count", s);
            kern<<<grid_for(kern, SB_THREADS, SB_SMEM), SB_THREADS, SB_SMEM, s>>>(
                reinterpret_cast<const uint32_t*>(kb), t.H, item_meta, plan, huge_count, item_hot, t.err);
            launch_end("huge_count", s);
            return cudaGetLastError();
        };
        if (e == cudaSuccess)
            e = (t.H.mode == MODE_POW2 && t.B >= BPB) ? run(k_big_count<true>) : run(k_big_count<false>);
    } else if (e == cudaSuccess) {
        auto kern = k_huge_count<K, HASHED>;
        const size_t smem = (size_t)BPB * 4;
        e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e == cudaSuccess) {
            launch_begin("huge_count", s);
            kern<<<grid_for(kern, LOCAL_THREADS, smem), LOCAL_THREADS, smem, s>>>(kb, t.H, bin_start, huge_bin,
                                                                                 huge_cs, plan, huge_count, t.err);
            launch_end("huge_count", s);
            e = cudaGetLastError();
        }
    }
    if (e == cudaSuccess) {
        launch_begin("huge_scan", s);
        k_huge_scan<<<max_huge, 1024, 0, s>>>(bin_start, huge_bin, plan, huge_count, huge_cursor, t.offsets, B,
                                              t.finder);
        launch_end("huge_scan", s);
        e = cudaGetLastError();
    }
    // 5. per-bin counting sort (and the huge bins' placement)
    if (e == cudaSuccess) {
        K* kout = static_cast<K*>(t.keys);
        const size_t smem = local_smem_bytes(sizeof(K), hv);
        auto run = [&](auto kern) {
            cudaError_t r = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (r != cudaSuccess) return r;
            launch_begin("bin_build", s);
            kern<<<grid_for(kern, LOCAL_THREADS, smem), LOCAL_THREADS, smem, s>>>(
                kb, hv ? vb : nullptr, n, t.H, bin_start, work, huge_bin, huge_cs, plan, huge_cursor, ctr,
                t.offsets, kout, t.values, t.err, t.finder, small_path);
            launch_end("bin_build", s);
            return cudaGetLastError();
        };
        e = hv ? run(k_bin_local<K, true, HASHED>) : run(k_bin_local<K, false, HASHED>);
    }
    if (e == cudaSuccess && small_path) {
        auto run = [&](auto kern) {
            cudaError_t r = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SB_SMEM_SMALL);
            if (r != cudaSuccess) return r;
            launch_begin("bin_small", s);
            kern<<<grid_for(kern, SB_THREADS, SB_SMEM_SMALL), SB_THREADS, SB_SMEM_SMALL, s>>>(
                reinterpret_cast<const uint32_t*>(kb), t.H, bin_start, work, plan, t.offsets,
                static_cast<uint32_t*>(t.keys), t.err, t.finder);
            launch_end("bin_small", s);
            return cudaGetLastError();
        };
        if (t.H.mode == MODE_POW2 && t.B >= BPB)
            e = t.finder.map ? run(k_bin_small<true, true>) : run(k_bin_small<true, false>);
        else
            e = t.finder.map ? run(k_bin_small<false, true>) : run(k_bin_small<false, false>);
    }
    if (e == cudaSuccess && small_path) {
        auto run = [&](auto kern) {
            cudaError_t r = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SB_SMEM);
            if (r != cudaSuccess) return r;
            launch_begin("bin_big", s);
            kern<<<grid_for(kern, SB_THREADS, SB_SMEM), SB_THREADS, SB_SMEM, s>>>(
                reinterpret_cast<const uint32_t*>(kb), t.H, item_meta, item_hot, plan, huge_cursor, n,
                static_cast<uint32_t*>(t.keys), t.err);
            launch_end("bin_big", s);
            return cudaGetLastError();
        };
        e = (t.H.mode == MODE_POW2 && t.B >= BPB) ? run(k_big_place<true>) : run(k_big_place<false>);
    }
    dev_free(mem, s);
    return e;
}

// Queries grouped by the table's bins (bin = bucket >> BIN_SHIFT) with the
// build's one- or two-pass partition, recording what the reverse passes need.
template <typename K>
cudaError_t group_queries_impl(const Table& t, const K* q, uint64_t nq, GroupedQueries* g, cudaStream_t s) {
    const uint64_t B = t.B;
    const uint32_t P = (uint32_t)((B + BPB - 1) / BPB);
    const uint32_t P2 = P <= RADIX ? P : RADIX;
    const uint32_t P1 = (P + P2 - 1) / P2;
    const bool two = P1 > 1;
    const uint32_t nch_a = (uint32_t)((nq + CHUNK - 1) / CHUNK);
    const uint32_t nch_b_max = nch_a + P1 + 1;
    const uint32_t shift1 = two ? 7u : 0u;
    const uint32_t R1 = two ? P1 : P;
    auto al = [](size_t x) { return (x + 255) & ~size_t(255); };
    size_t off = 0;
    const size_t o_cnt = off; off += al((size_t)P * 4);
    off += al(64);  // (spare, zeroed with the counts)
    const size_t zero_bytes = off;
    const size_t o_ca = off; off += al((size_t)nch_a * RADIX * 4);
    const size_t o_cb = off; off += al(two ? (size_t)nch_b_max * RADIX * 4 : 0);
    const size_t o_pref = off; off += al((size_t)nch_b_max * RADIX * 4);
    const size_t o_start = off; off += al((size_t)(P + 1) * 4);
    const size_t o_work = off; off += al((size_t)P * 4);
    const size_t o_seg = off; off += al((size_t)(P1 + 1) * 4);
    const size_t o_hbin = off; off += al((size_t)MAX_HUGE * 4);
    const size_t o_hcs = off; off += al((size_t)(MAX_HUGE + 1) * 4);
    const size_t o_plan = off; off += al(sizeof(Plan));
    const size_t o_lba = off; off += al((size_t)nch_a * TILES_PER_CHUNK * RADIX * 8);
    const size_t o_lbb = off; off += al(two ? (size_t)nch_b_max * TILES_PER_CHUNK * RADIX * 8 : 0);
    // reverse-pass records: 32-bit queries 16-bit staging positions, else (rank, digit) words
    const size_t rec_bytes = sizeof(K) == 4 ? 2 : 4;
    const size_t o_dra = off; off += al(nq * rec_bytes + 16);
    const size_t o_drb = off; off += al(two ? nq * rec_bytes + 16 : 0);
    const size_t o_qa = off; off += al(two ? nq * sizeof(K) : 0);
    const size_t o_qb = off; off += al((nq + 4) * sizeof(K));
    cudaError_t e = dev_alloc(&g->mem, off, s);
    if (e != cudaSuccess) return e;
    char* base = static_cast<char*>(g->mem);
    uint32_t* bin_count = reinterpret_cast<uint32_t*>(base + o_cnt);
    uint32_t* cnt_a = reinterpret_cast<uint32_t*>(base + o_ca);
    uint32_t* cnt_b = reinterpret_cast<uint32_t*>(base + o_cb);
    uint32_t* pref = reinterpret_cast<uint32_t*>(base + o_pref);
    uint32_t* bin_start = reinterpret_cast<uint32_t*>(base + o_start);
    uint32_t* seg = reinterpret_cast<uint32_t*>(base + o_seg);
    Plan* plan = reinterpret_cast<Plan*>(base + o_plan);
    uint2* lb_a = reinterpret_cast<uint2*>(base + o_lba);
    uint2* lb_b = reinterpret_cast<uint2*>(base + o_lbb);
    uint32_t* dr_a = reinterpret_cast<uint32_t*>(base + o_dra);
    uint32_t* dr_b = reinterpret_cast<uint32_t*>(base + o_drb);
    K* qa = reinterpret_cast<K*>(base + o_qa);
    K* qb = reinterpret_cast<K*>(base + o_qb);
    const ChunkMap cm_a{false, nq, P, P2, 1u, bin_start, nullptr};
    const ChunkMap cm_b{true, nq, P, P2, P1, bin_start, seg};
    g->two = two;

    e = cudaMemsetAsync(base, 0, zero_bytes, s);
    if (e == cudaSuccess) {
        auto kern = k_part_count<K, true>;
        const size_t smem = (size_t)P * 4;
        e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e == cudaSuccess) {
            unsigned gr = grid_for(kern, PASS_THREADS, smem);
            if (gr > nch_a) gr = nch_a;
            launch_begin("q_part_count", s);
            kern<<<gr, PASS_THREADS, smem, s>>>(q, nq, t.H, P, shift1, R1, nch_a, bin_count, cnt_a, nullptr);
            launch_end("q_part_count", s);
            e = cudaGetLastError();
        }
    }
    if (e == cudaSuccess) {
        launch_begin("part_plan", s);
        // bins of many queries first in the probe's work list; the bins with the
        // most (huge bins) are cut into HUGE_CHUNK-query work items
        k_part_plan<<<1, 1024, 0, s>>>(bin_count, P, P1, P2, nq, 1u << 16, HUGE_T, HUGE_CHUNK, MAX_HUGE, bin_start, seg,
                                       reinterpret_cast<uint32_t*>(base + o_work),
                                       reinterpret_cast<uint32_t*>(base + o_hbin),
                                       reinterpret_cast<uint32_t*>(base + o_hcs), plan, nullptr, B);
        launch_end("part_plan", s);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) {
        launch_begin("chunk_scan", s);
        k_chunk_scan<<<RADIX, 1024, 0, s>>>(cnt_a, pref, cm_a, nch_a, plan, R1, two ? P2 : 1u, nullptr);
        launch_end("chunk_scan", s);
        e = cudaGetLastError();
    }
    // 32-bit queries move through the passes as their hashes (k_pass32): the
    // grouped queries are hashes, which the probes undo (items.qunhash)
    constexpr bool HASHED = sizeof(K) == 4;
    uint32_t* gerr = g->err ? g->err : t.err;
    if (e == cudaSuccess)
        e = launch_down<K, 0, false, true>(q, nullptr, nq, t.H, shift1, RADIX - 1, R1, cm_a, nch_a, nch_a, plan, cnt_a,
                                           two ? qa : qb, nullptr, gerr, s, "q_partition", dr_a, lb_a);
    if (e == cudaSuccess && two) {
        launch_begin("chunk_count", s);
        k_chunk_count<K, HASHED><<<nch_b_max, PASS_THREADS, 0, s>>>(qa, t.H, cm_b, plan, cnt_b);
        launch_end("chunk_count", s);
        e = cudaGetLastError();
        if (e == cudaSuccess) {
            launch_begin("chunk_scan", s);
            k_chunk_scan<<<RADIX, 1024, 0, s>>>(cnt_b, pref, cm_b, 0u, plan, P2, 1u, nullptr);
            launch_end("chunk_scan", s);
            e = cudaGetLastError();
        }
        if (e == cudaSuccess)
            e = launch_down<K, 0, HASHED, true>(qa, nullptr, nq, t.H, 0, RADIX - 1, P2, cm_b, 0u, nch_b_max, plan,
                                                cnt_b, qb, nullptr, gerr, s, "q_partition2", dr_b, lb_b, true);
    }
    g->q_grouped = qb;
    g->bin_start = bin_start;
    g->nbins = P;
    // what the reverse passes need
    g->cm_a = cm_a;
    g->cm_b = cm_b;
    g->nch_a = nch_a;
    g->nch_b_max = nch_b_max;
    g->plan = plan;
    g->items.n_huge = &plan->n_huge;
    g->items.huge_chunks = &plan->huge_chunks;
    g->items.n_work = &plan->n_work;
    g->items.huge_bin = reinterpret_cast<const uint32_t*>(base + o_hbin);
    g->items.huge_chunk_start = reinterpret_cast<const uint32_t*>(base + o_hcs);
    g->items.work = reinterpret_cast<const uint32_t*>(base + o_work);
    g->items.huge_chunk = HUGE_CHUNK;
    g->items.qunhash = HASHED ? ((1ull << 32) | (uint32_t)t.H.seed) : 0ull;
    g->dr_a = dr_a;
    g->dr_b = dr_b;
    g->lb_a = lb_a;
    g->lb_b = lb_b;
    return e;
}

template <typename K>
cudaError_t ungroup_counts_impl(const Table& t, const GroupedQueries* g, const uint32_t* cs, uint32_t* tmp,
                                uint32_t* counts, cudaStream_t s) {
    const Plan* plan = static_cast<const Plan*>(g->plan);
    uint32_t* gerr = g->err ? g->err : t.err;
    // 32-bit queries were grouped by k_pass32, whose tiles k_pass_reverse32 undoes
    auto reverse = [&](const uint32_t* from, uint32_t* to, const ChunkMap& cm, uint32_t nch_host, uint32_t grid,
                       const uint32_t* dr, const uint2* lb) {
        launch_begin("q_reverse", s);
        if (sizeof(K) == 4)
            k_pass_reverse32<<<grid, P32_THREADS, 0, s>>>(from, to, cm, nch_host, plan, dr, lb, gerr);
        else
            k_pass_reverse<K><<<grid, PASS_THREADS, 0, s>>>(from, to, cm, nch_host, plan, dr, lb, gerr);
        launch_end("q_reverse", s);
        return cudaGetLastError();
    };
    if (g->two) {
        cudaError_t e = reverse(cs, tmp, g->cm_b, 0u, g->nch_b_max, g->dr_b, g->lb_b);
        if (e != cudaSuccess) return e;
        cs = tmp;
    }
    return reverse(cs, counts, g->cm_a, g->nch_a, g->nch_a, g->dr_a, g->lb_a);
}

}  // namespace

bool partition_supported(uint64_t B) { return (B + BPB - 1) / BPB <= MAX_BINS; }

cudaError_t build_partitioned(Table& t, const void* d_keys, const void* d_values, cudaStream_t s) {
    const uint32_t* vals = static_cast<const uint32_t*>(d_values);
    // k_bin_local and k_huge_scan list the long buckets when t.finder asks for them
    t.long_noted = t.finder.map != nullptr;
    if (t.key_bytes == 4) return build_partitioned_impl<uint32_t>(t, static_cast<const uint32_t*>(d_keys), vals, s);
    return build_partitioned_impl<uint64_t>(t, static_cast<const uint64_t*>(d_keys), vals, s);
}

bool probe_grouping_pays(const Table& t, uint64_t q) {
    const uint64_t P = (t.B + BPB - 1) / BPB;
    // one CTA answers one bin at a time: with fewer than ~4 bins per SM the bins
    // (and the walks inside them) are too few and too large to keep the GPU busy
    if (P < 4ull * (uint64_t)num_sms() || P > MAX_BINS || q < (1u << 20)) return false;
    const uint64_t table_bytes = 4 * (t.B + 1) + (uint64_t)t.key_bytes * t.n;
    return table_bytes > (48ull << 20);  // the table does not stay in L2
}

cudaError_t group_queries(const Table& t, const void* d_q, uint64_t q, GroupedQueries* g, cudaStream_t s) {
    if (t.key_bytes == 4) return group_queries_impl<uint32_t>(t, static_cast<const uint32_t*>(d_q), q, g, s);
    return group_queries_impl<uint64_t>(t, static_cast<const uint64_t*>(d_q), q, g, s);
}

cudaError_t ungroup_counts(const Table& t, const GroupedQueries* g, const uint32_t* cs, uint32_t* tmp,
                           uint32_t* counts, cudaStream_t s) {
    if (t.key_bytes == 4) return ungroup_counts_impl<uint32_t>(t, g, cs, tmp, counts, s);
    return ungroup_counts_impl<uint64_t>(t, g, cs, tmp, counts, s);
}

void group_release(GroupedQueries* g, cudaStream_t s) {
    if (g->mem) dev_free(g->mem, s);
    g->mem = nullptr;
}

}  // namespace hg
