// Partitioned HashGraph build: the "efficient HashGraph" of Sec. 3.2, where
// keys are first grouped by ranges of hashed values ("bins") so that the
// per-bucket counting and placing of Algorithm 1 happen in fast on-chip
// memory instead of as random atomics into an offsets array far larger than
// the cache.
//
// Stages (bin = bucket >> BIN_SHIFT, so a bin is a range of 8192 buckets):
//   1. k_part_count  histogram of bins (shared-memory counters per CTA).
//   2. k_part_plan   one CTA: exclusive scan of the bin counts into bin_start,
//                    tile counts per coarse segment, offsets[B] = n.
//   3. k_part_pass   MSD partition by bin, radix <= 128 per pass, one or two
//                    passes: each tile ranks its keys per digit in shared
//                    memory, finds where its run of each digit goes with a
//                    per-digit decoupled look-back over earlier tiles, stages
//                    the keys in digit order and writes each run contiguously.
//   4. k_bin_local   one CTA per bin: counting sort of the bin's keys by
//                    bucket in shared memory (histogram, exclusive scan ->
//                    the bin's offsets, placement), written out contiguously.
//                    Buckets with many copies of one key are written straight
//                    from registers (their positions are consecutive anyway);
//                    the rest are staged so that every global write is a
//                    coalesced run.
// The result equals the direct build's (offsets bit-exact; the order inside
// a bucket differs, which Algorithm 1 leaves free).
#include <cstdint>

#include "hg_device.cuh"

namespace hg {

namespace {

constexpr int BIN_SHIFT = 13;
constexpr uint32_t BPB = 1u << BIN_SHIFT;  // buckets per bin
constexpr uint32_t RADIX = 128;            // digits per partition pass
constexpr uint32_t MAX_BINS = RADIX * RADIX;
constexpr int PASS_THREADS = 512;
constexpr int LOCAL_THREADS = 1024;
constexpr uint32_t HOT_T = 64;             // bucket size from which keys bypass the staging buffer
constexpr uint32_t MAX_HOT = 256;          // hot buckets per bin the staging map can hold
constexpr size_t LOCAL_STAGE_BYTES = 184 * 1024;
constexpr uint32_t SPIN_LIMIT = 1u << 20;
constexpr int LOOK_WIN = 8;                // status words read per look-back step
constexpr uint32_t HUGE_T = 1u << 18;      // bins with more keys are split over many CTAs
constexpr uint32_t HUGE_CHUNK = 1u << 16;  // keys per CTA work item of a huge bin
constexpr uint32_t MAX_HUGE = 512;         // huge bins with their own counter/cursor slice

constexpr uint64_t FLAG_AGG = 1ull << 62, FLAG_PREFIX = 2ull << 62, VALUE_MASK = (1ull << 62) - 1;

template <typename K>
struct PassCfg {
    static constexpr int IPT = sizeof(K) == 4 ? 16 : 8;  // elements per thread per tile
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

// ---------------------------------------------------------------- count --
template <typename K>
__global__ void __launch_bounds__(PASS_THREADS)
k_part_count(const K* __restrict__ keys, uint64_t n, Hasher H, uint32_t P, uint32_t* bin_count) {
    extern __shared__ uint32_t s_hist[];
    for (uint32_t i = threadIdx.x; i < P; i += blockDim.x) s_hist[i] = 0;
    __syncthreads();
    const unsigned lane = lane_id();
    const uint64_t gw = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint64_t nw = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    const bool vec = (reinterpret_cast<uintptr_t>(keys) & 15) == 0;
    constexpr int VEC = KeyVec<K>::N;
    const uint64_t ngroups = (n + VEC - 1) / VEC;
    for (uint64_t g0 = gw * 32; g0 < ngroups; g0 += nw * 32) {
        const uint64_t g = g0 + lane;
        const uint64_t e0 = g * VEC;
        K k[VEC];
        bool ok[VEC];
        if (vec && e0 + VEC <= n) {
            const KeyVec<K> kv = load_keys16(keys + e0);
#pragma unroll
            for (int j = 0; j < VEC; ++j) { k[j] = kv.k[j]; ok[j] = true; }
        } else {
#pragma unroll
            for (int j = 0; j < VEC; ++j) { ok[j] = e0 + j < n; k[j] = ok[j] ? keys[e0 + j] : (K)0; }
        }
#pragma unroll
        for (int j = 0; j < VEC; ++j) {
            const unsigned m = __ballot_sync(FULL_MASK, ok[j]);
            if (ok[j]) smem_add1(s_hist, bin_of(k[j], H), m);
        }
    }
    __syncthreads();
    for (uint32_t i = threadIdx.x; i < P; i += blockDim.x)
        if (s_hist[i]) atomicAdd(bin_count + i, s_hist[i]);
}

// ----------------------------------------------------------------- plan --
struct Plan {
    uint32_t tiles_b;      // tiles of the segmented pass
    uint32_t n_huge;       // bins split over many CTAs (at most MAX_HUGE)
    uint32_t huge_chunks;  // their HUGE_CHUNK-key work items
    uint32_t n_work;       // bins handled whole by one CTA
};

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

// One CTA.  Writes bin_start[P+1]; seg_tile_start[P1+1] (tiles of each coarse
// segment in the segmented pass); offsets[B] = n; the huge bins (more than
// HUGE_T keys; the first MAX_HUGE of them) with the prefix of their chunk
// counts; and the work list of the other bins, bins above big_t keys first.
__global__ void __launch_bounds__(1024)
k_part_plan(const uint32_t* __restrict__ bin_count, uint32_t P, uint32_t P1, uint32_t P2, uint64_t n, uint32_t tile,
            uint32_t big_t, uint32_t* bin_start, uint32_t* seg_tile_start, uint32_t* work, uint32_t* huge_bin,
            uint32_t* huge_chunk_start, Plan* plan, uint32_t* offsets, uint64_t B) {
    __shared__ uint32_t s_warp[33];
    __shared__ uint32_t s_huge[MAX_BINS / 32];
    uint32_t running = 0, tot;
    for (uint32_t i = threadIdx.x; i < MAX_BINS / 32; i += blockDim.x) s_huge[i] = 0;
    for (uint32_t base = 0; base < P; base += blockDim.x) {
        const uint32_t p = base + threadIdx.x;
        const uint32_t c = p < P ? bin_count[p] : 0u;
        const uint32_t ex = block_exclusive_scan<uint32_t>(c, s_warp, &tot);
        if (p < P) bin_start[p] = running + ex;
        running += tot;
    }
    if (threadIdx.x == 0) {
        bin_start[P] = running;
        offsets[B] = (uint32_t)n;
    }
    __syncthreads();
    // tiles per coarse segment
    uint32_t trun = 0;
    for (uint32_t base = 0; base < P1; base += blockDim.x) {
        const uint32_t sg = base + threadIdx.x;
        uint32_t t = 0;
        if (sg < P1) {
            const uint32_t lo = bin_start[sg * P2];
            const uint32_t hi = bin_start[min((sg + 1) * P2, P)];
            t = (hi - lo + tile - 1) / tile;
        }
        const uint32_t ex = block_exclusive_scan<uint32_t>(t, s_warp, &tot);
        if (sg < P1) seg_tile_start[sg] = trun + ex;
        trun += tot;
    }
    // huge bins (index order, first MAX_HUGE) and their chunk prefix
    uint32_t nh = 0, cr = 0;
    for (uint32_t base = 0; base < P; base += blockDim.x) {
        const uint32_t p = base + threadIdx.x;
        const uint32_t c = p < P ? bin_count[p] : 0u;
        const uint32_t is_huge = c > HUGE_T ? 1u : 0u;
        const uint32_t hx = block_exclusive_scan<uint32_t>(is_huge, s_warp, &tot);
        const bool admit = is_huge && nh + hx < MAX_HUGE;
        const uint32_t ch = admit ? (c + HUGE_CHUNK - 1) / HUGE_CHUNK : 0u;
        uint32_t ctot;
        const uint32_t cx = block_exclusive_scan<uint32_t>(ch, s_warp, &ctot);
        if (admit) {
            huge_bin[nh + hx] = p;
            huge_chunk_start[nh + hx] = cr + cx;
            atomicOr(&s_huge[p >> 5], 1u << (p & 31));
        }
        nh += tot;
        cr += ctot;
    }
    const uint32_t n_huge = min(nh, MAX_HUGE);
    __syncthreads();
    // work list: big bins first, then the rest
    uint32_t nbig = 0;
    for (uint32_t base = 0; base < P; base += blockDim.x) {
        const uint32_t p = base + threadIdx.x;
        const bool hz = p < P && ((s_huge[p >> 5] >> (p & 31)) & 1u);
        const uint32_t big = (p < P && !hz && bin_count[p] > big_t) ? 1u : 0u;
        const uint32_t ex = block_exclusive_scan<uint32_t>(big, s_warp, &tot);
        if (big) work[nbig + ex] = p;
        nbig += tot;
    }
    uint32_t nsmall = 0;
    for (uint32_t base = 0; base < P; base += blockDim.x) {
        const uint32_t p = base + threadIdx.x;
        const bool hz = p < P && ((s_huge[p >> 5] >> (p & 31)) & 1u);
        const uint32_t small = (p < P && !hz && bin_count[p] <= big_t) ? 1u : 0u;
        const uint32_t ex = block_exclusive_scan<uint32_t>(small, s_warp, &tot);
        if (small) work[nbig + nsmall + ex] = p;
        nsmall += tot;
    }
    if (threadIdx.x == 0) {
        seg_tile_start[P1] = trun;
        huge_chunk_start[n_huge] = cr;
        plan->tiles_b = trun;
        plan->n_huge = n_huge;
        plan->huge_chunks = cr;
        plan->n_work = nbig + nsmall;
    }
}

// ----------------------------------------------------------------- pass --
// Stage buffer layout in dynamic shared memory: keys[TILE] | payload[TILE] | digit[TILE] (u8)
// | cnt[RADIX] | loc[RADIX] | base[RADIX] | scratch.
template <typename K, int PM, bool SEG>
__global__ void __launch_bounds__(PASS_THREADS)
k_part_pass(const K* __restrict__ in, const uint32_t* __restrict__ in_v, uint64_t n, Hasher H, uint32_t dig_shift,
            uint32_t dig_mask, uint32_t R, uint32_t P, uint32_t P2, const uint32_t* __restrict__ bin_start,
            const uint32_t* __restrict__ seg_tile_start, uint32_t nseg, const Plan* __restrict__ plan,
            uint32_t* tile_ctr, uint64_t* status, K* __restrict__ out, uint32_t* __restrict__ out_v, uint32_t* err) {
    constexpr int IPT = PassCfg<K>::IPT;
    constexpr int TILE = PassCfg<K>::TILE;
    extern __shared__ __align__(16) unsigned char smem[];
    K* s_keys = reinterpret_cast<K*>(smem);
    uint32_t* s_pay = reinterpret_cast<uint32_t*>(smem + TILE * sizeof(K));
    uint8_t* s_dig = reinterpret_cast<uint8_t*>(smem + TILE * sizeof(K) + (PM ? TILE * 4 : 0));
    uint32_t* s_cnt = reinterpret_cast<uint32_t*>(smem + TILE * sizeof(K) + (PM ? TILE * 4 : 0) + TILE);
    uint32_t* s_loc = s_cnt + RADIX;
    uint32_t* s_base = s_loc + RADIX;
    __shared__ uint32_t s_tile;
    __shared__ uint64_t s_e0, s_e1;
    __shared__ uint32_t s_seg, s_first;
    __shared__ uint32_t s_warp[33];

    const uint32_t ntiles = SEG ? plan->tiles_b : (uint32_t)((n + TILE - 1) / TILE);
    for (uint32_t i = threadIdx.x; i < RADIX; i += blockDim.x) s_cnt[i] = 0;

    while (true) {
        if (threadIdx.x == 0) s_tile = atomicAdd(tile_ctr, 1u);
        __syncthreads();
        const uint32_t t = s_tile;
        if (t >= ntiles) break;
        if (threadIdx.x == 0) {
            if (SEG) {
                uint32_t lo = 0, hi = nseg;  // last segment with seg_tile_start[s] <= t
                while (hi - lo > 1) {
                    const uint32_t mid = (lo + hi) >> 1;
                    if (seg_tile_start[mid] <= t) lo = mid; else hi = mid;
                }
                const uint32_t s = lo;
                const uint64_t a = bin_start[s * P2];
                const uint64_t b = bin_start[min((s + 1) * P2, P)];
                const uint32_t ts = t - seg_tile_start[s];
                s_seg = s;
                s_first = seg_tile_start[s];
                s_e0 = a + (uint64_t)ts * TILE;
                s_e1 = min(b, s_e0 + TILE);
            } else {
                s_seg = 0;
                s_first = 0;
                s_e0 = (uint64_t)t * TILE;
                s_e1 = min(n, s_e0 + TILE);
            }
        }
        __syncthreads();
        const uint64_t e0 = s_e0, e1 = s_e1;
        const uint32_t seg = s_seg;
        const uint32_t first = s_first;
        const uint32_t cnt_tile = (uint32_t)(e1 - e0);

        // load (coalesced), digit, rank within the tile
        K k[IPT];
        uint32_t v[IPT];
        uint32_t d[IPT], r[IPT];
#pragma unroll
        for (int j = 0; j < IPT; ++j) {
            const uint32_t li = threadIdx.x + j * PASS_THREADS;
            const bool ok = li < cnt_tile;
            k[j] = ok ? in[e0 + li] : (K)0;
            if (PM == 1) v[j] = ok ? in_v[e0 + li] : 0u;
            if (PM == 2) v[j] = (uint32_t)(e0 + li);
        }
#pragma unroll
        for (int j = 0; j < IPT; ++j) {
            const uint32_t li = threadIdx.x + j * PASS_THREADS;
            const bool ok = li < cnt_tile;
            const unsigned m = __ballot_sync(FULL_MASK, ok);
            d[j] = 0;
            r[j] = 0;
            if (ok) {
                d[j] = (bin_of(k[j], H) >> dig_shift) & dig_mask;
                if (d[j] >= R) {  // cannot happen for a consistent plan; keep shared memory in bounds
                    atomicOr(err, DEVERR_BOUNDS);
                    d[j] = R - 1;
                }
                r[j] = smem_inc(s_cnt, d[j], m);
            }
        }
        __syncthreads();

        // publish this tile's counts, look back for the runs before it, local digit offsets
        if (threadIdx.x < RADIX) {
            const uint32_t dd = threadIdx.x;
            const uint32_t c = dd < R ? s_cnt[dd] : 0u;
            uint64_t excl = 0;
            if (dd < R) {
                uint64_t* my = status + (uint64_t)t * R + dd;
                if (t == first) {
                    atomicExch(reinterpret_cast<unsigned long long*>(my), (unsigned long long)(FLAG_PREFIX | c));
                } else {
                    atomicExch(reinterpret_cast<unsigned long long*>(my), (unsigned long long)(FLAG_AGG | c));
                    // walk back over earlier tiles of the segment, LOOK_WIN status words per step
                    // (independent loads), until a tile with its inclusive prefix is found
                    int64_t pt = (int64_t)t - 1;
                    uint32_t polls = 0;
                    bool done = false;
                    while (!done && pt >= (int64_t)first) {
                        uint64_t wv[LOOK_WIN];
#pragma unroll
                        for (int q = 0; q < LOOK_WIN; ++q) {
                            const int64_t tt = pt - q;
                            wv[q] = tt >= (int64_t)first
                                        ? *reinterpret_cast<const volatile uint64_t*>(status + (uint64_t)tt * R + dd)
                                        : FLAG_PREFIX;
                        }
#pragma unroll
                        for (int q = 0; q < LOOK_WIN; ++q) {
                            if (!done) {
                                const int64_t tt = pt - q;
                                uint64_t w = wv[q];
                                while ((w & ~VALUE_MASK) == 0 && polls < SPIN_LIMIT) {
                                    ++polls;
                                    __nanosleep(32);
                                    w = *reinterpret_cast<const volatile uint64_t*>(status + (uint64_t)tt * R + dd);
                                }
                                if ((w & ~VALUE_MASK) == 0) {
                                    atomicOr(err, DEVERR_TIMEOUT);
                                    done = true;
                                } else {
                                    excl += (w & VALUE_MASK);
                                    if ((w & ~VALUE_MASK) == FLAG_PREFIX) done = true;
                                }
                            }
                        }
                        pt -= LOOK_WIN;
                    }
                    __threadfence();
                    atomicExch(reinterpret_cast<unsigned long long*>(my), (unsigned long long)(FLAG_PREFIX | (excl + c)));
                }
                const uint32_t bin = SEG ? seg * P2 + dd : dd * P2;
                s_base[dd] = bin_start[min(bin, P)] + (uint32_t)excl;
            }
        }
        // exclusive scan of tile counts over digits (first 128 threads = 4 warps)
        if (threadIdx.x < RADIX) {
            const uint32_t c = threadIdx.x < R ? s_cnt[threadIdx.x] : 0u;
            const uint32_t incl = warp_inclusive_scan(c);
            if (lane_id() == 31) s_warp[threadIdx.x >> 5] = incl;
            asm volatile("bar.sync 1, 128;");
            uint32_t wp = 0;
            for (uint32_t w = 0; w < (threadIdx.x >> 5); ++w) wp += s_warp[w];
            s_loc[threadIdx.x] = wp + incl - c;
        }
        __syncthreads();

        // stage in digit order
#pragma unroll
        for (int j = 0; j < IPT; ++j) {
            const uint32_t li = threadIdx.x + j * PASS_THREADS;
            if (li < cnt_tile) {
                const uint32_t pos = s_loc[d[j]] + r[j];
                s_keys[pos] = k[j];
                if (PM) s_pay[pos] = v[j];
                s_dig[pos] = (uint8_t)d[j];
            }
        }
        __syncthreads();
        // write each digit's run contiguously
        for (uint32_t i = threadIdx.x; i < cnt_tile; i += PASS_THREADS) {
            const uint32_t dd = s_dig[i];
            const uint64_t dst = (uint64_t)s_base[dd] + (i - s_loc[dd]);
            if (dst < n) {
                out[dst] = s_keys[i];
                if (PM) out_v[dst] = s_pay[i];
            } else {
                atomicOr(err, DEVERR_BOUNDS);
            }
        }
        for (uint32_t i = threadIdx.x; i < RADIX; i += blockDim.x) s_cnt[i] = 0;
        __syncthreads();
    }
}

// ---------------------------------------------------------------- local --
// Calls f(i, key, value, mask) for every i in [s0, s1): the 16-byte aligned body
// two vectors per thread at a time, the few elements around it by warp 0.
// `mask` = lanes of the warp calling f together.  HV: also load in_v[i].
template <typename K, bool HV, typename F>
__device__ __forceinline__ void block_for_range(const K* __restrict__ in, const uint32_t* __restrict__ in_v,
                                                uint64_t s0, uint64_t s1, F&& f) {
    constexpr int VEC = KeyVec<K>::N;
    const unsigned lane = lane_id();
    const uint32_t nt = blockDim.x;
    const uint64_t mis = (reinterpret_cast<uintptr_t>(in + s0) & 15) / sizeof(K);
    const uint64_t hend = mis ? min(s1, s0 + (VEC - mis)) : s0;
    const uint64_t nv = s1 > hend ? (s1 - hend) / VEC : 0;
    const uint64_t tail0 = hend + nv * VEC;
    for (uint64_t g0 = (threadIdx.x & ~31u) * 2; g0 < nv; g0 += 2ull * nt) {
        KeyVec<K> kv[2];
        uint32_t vv[2][VEC];
        bool ok[2];
#pragma unroll
        for (int u = 0; u < 2; ++u) {
            const uint64_t g = g0 + u * 32 + lane;
            ok[u] = g < nv;
            if (ok[u]) {
                kv[u] = load_keys16(in + hend + g * VEC);
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
        for (int u = 0; u < 2; ++u) {
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

// Huge bin work item -> (huge index e, bin p, key range [c0, c1)).
__device__ __forceinline__ void huge_item(uint32_t item, uint32_t n_huge, const uint32_t* __restrict__ huge_chunk_start,
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
    c0 = (uint64_t)bin_start[p] + (uint64_t)(item - huge_chunk_start[e]) * HUGE_CHUNK;
    c1 = min((uint64_t)bin_start[p + 1], c0 + HUGE_CHUNK);
}

// Huge bins, step 1: per-chunk bucket histograms added into huge_count[e][*].
template <typename K>
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
        huge_item(item, n_huge, huge_chunk_start, huge_bin, bin_start, e, p, c0, c1);
        const uint64_t b0 = (uint64_t)p << BIN_SHIFT;
        const uint32_t nb = (uint32_t)min((uint64_t)BPB, H.B - b0);
        for (uint32_t j = threadIdx.x; j < BPB; j += blockDim.x) s_cnt[j] = 0;
        __syncthreads();
        block_for_range<K, false>(in, nullptr, c0, c1, [&](uint64_t, K k, uint32_t, unsigned m) {
            uint32_t j = (uint32_t)(bucket_of(k, H) - b0);
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

// Huge bins, step 2: one CTA per huge bin scans its counts into offsets and cursors.
__global__ void __launch_bounds__(1024)
k_huge_scan(const uint32_t* __restrict__ bin_start, const uint32_t* __restrict__ huge_bin,
            const Plan* __restrict__ plan, const uint32_t* __restrict__ huge_count, uint32_t* huge_cursor,
            uint32_t* offsets, uint64_t B) {
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
        }
        running += tot;
    }
}

// Step 3 (all bins): work items [0, huge_chunks) place one chunk of a huge bin
// through its cursors; the following n_work items each take a whole bin.
// Shared memory: cnt[BPB] | hotmask[BPB/32] | hot list (pos, prefix length) | stage keys | stage payload.
template <typename K, bool HV>
__global__ void __launch_bounds__(LOCAL_THREADS)
k_bin_local(const K* __restrict__ in, const uint32_t* __restrict__ in_v, uint64_t n, Hasher H,
            const uint32_t* __restrict__ bin_start, const uint32_t* __restrict__ work,
            const uint32_t* __restrict__ huge_bin, const uint32_t* __restrict__ huge_chunk_start,
            const Plan* __restrict__ plan, uint32_t* huge_cursor, uint32_t* work_ctr, uint32_t* offsets,
            K* __restrict__ out, uint32_t* __restrict__ out_v, uint32_t* err) {
    constexpr uint32_t STAGE_CAP = (uint32_t)(LOCAL_STAGE_BYTES / (sizeof(K) + (HV ? 4 : 0)));
    extern __shared__ __align__(16) unsigned char smem[];
    uint32_t* s_cnt = reinterpret_cast<uint32_t*>(smem);
    uint32_t* s_hot = s_cnt + BPB;                 // bitmask
    uint32_t* s_hot_cpos = s_hot + BPB / 32;       // compacted position of each hot bucket
    uint32_t* s_hot_len = s_hot_cpos + MAX_HOT;    // its length (then inclusive prefix)
    K* s_keys = reinterpret_cast<K*>(s_hot_len + MAX_HOT);
    uint32_t* s_pay = reinterpret_cast<uint32_t*>(s_keys + STAGE_CAP);
    __shared__ uint32_t s_item, s_nhot, s_warp[33];

    const unsigned lane = lane_id();
    const int w = threadIdx.x >> 5;
    const int nw = blockDim.x >> 5;
    const uint64_t B = H.B;
    const uint32_t n_huge = plan->n_huge, huge_chunks = plan->huge_chunks, n_work = plan->n_work;

    while (true) {
        if (threadIdx.x == 0) s_item = atomicAdd(work_ctr, 1u);
        __syncthreads();
        const uint32_t item = s_item;
        if (item >= huge_chunks + n_work) break;

        if (item < huge_chunks) {
            // ---- one chunk of a huge bin: local histogram, reserve runs, place
            uint32_t e, p;
            uint64_t c0, c1;
            huge_item(item, n_huge, huge_chunk_start, huge_bin, bin_start, e, p, c0, c1);
            const uint64_t b0 = (uint64_t)p << BIN_SHIFT;
            const uint32_t nb = (uint32_t)min((uint64_t)BPB, B - b0);
            for (uint32_t j = threadIdx.x; j < BPB; j += blockDim.x) s_cnt[j] = 0;
            __syncthreads();
            block_for_range<K, false>(in, nullptr, c0, c1, [&](uint64_t, K k, uint32_t, unsigned m) {
                uint32_t j = (uint32_t)(bucket_of(k, H) - b0);
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
                uint32_t j = (uint32_t)(bucket_of(k, H) - b0);
                if (j >= nb) j = nb - 1;
                const uint32_t pos = smem_inc(s_cnt, j, m);
                if (pos < n) {
                    out[pos] = k;
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

        // pass 1: bucket histogram
        block_for_range<K, false>(in, nullptr, s0, s1, [&](uint64_t, K k, uint32_t, unsigned m) {
            uint32_t j = (uint32_t)(bucket_of(k, H) - b0);
            if (j >= nb) {
                atomicOr(err, DEVERR_BOUNDS);
                j = nb - 1;
            }
            smem_add1(s_cnt, j, m);
        });
        __syncthreads();

        // scan: offsets of the bin's buckets; hot buckets; compacted staging positions.
        // Each warp scans a contiguous slice of BPB / nw buckets, 32 at a time.
        const uint32_t slice = BPB / nw;
        const uint32_t lo = w * slice;
        uint32_t tot_all = 0, tot_cold = 0;
        for (uint32_t j = lo + lane; j < lo + slice; j += 32) {
            const uint32_t c = s_cnt[j];
            tot_all += c;
            tot_cold += (c >= HOT_T) ? 0u : c;
        }
        tot_all = __reduce_add_sync(FULL_MASK, tot_all);
        tot_cold = __reduce_add_sync(FULL_MASK, tot_cold);
        if (lane == 0) s_warp[w] = tot_all;
        __syncthreads();
        uint32_t pre_all = 0;
        for (int q = 0; q < w; ++q) pre_all += s_warp[q];
        __syncthreads();
        if (lane == 0) s_warp[w] = tot_cold;
        __syncthreads();
        uint32_t pre_cold = 0, cold_total = 0;
        for (int q = 0; q < nw; ++q) {
            if (q < w) pre_cold += s_warp[q];
            cold_total += s_warp[q];
        }
        const bool stage = cold_total <= STAGE_CAP;
        uint32_t run_all = pre_all, run_cold = pre_cold;
        for (uint32_t j0 = lo; j0 < lo + slice; j0 += 32) {
            const uint32_t j = j0 + lane;
            const uint32_t c = s_cnt[j];
            const bool hot = c >= HOT_T;
            const uint32_t ia = warp_inclusive_scan(c);
            const uint32_t cc = hot ? 0u : c;
            const uint32_t ic = warp_inclusive_scan(cc);
            const uint32_t start = (uint32_t)s0 + run_all + ia - c;
            const uint32_t cstart = run_cold + ic - cc;
            if (j < nb) offsets[b0 + j] = start;
            if (stage && !hot) {
                s_cnt[j] = cstart;
            } else {
                s_cnt[j] = start;
                if (stage) {
                    atomicOr(&s_hot[j >> 5], 1u << (j & 31));
                    const uint32_t h = atomicAdd(&s_nhot, 1u);
                    if (h < MAX_HOT) {
                        s_hot_cpos[h] = cstart;
                        s_hot_len[h] = c;
                    }
                }
            }
            run_all += __shfl_sync(FULL_MASK, ia, 31);
            run_cold += __shfl_sync(FULL_MASK, ic, 31);
        }
        __syncthreads();
        const uint32_t nhot = s_nhot;
        const bool staged = stage && nhot <= MAX_HOT;
        if (stage && !staged) {
            // too many hot buckets for the map: every bucket is placed directly
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

        // pass 2: place (hot buckets straight to global memory, the rest staged)
        block_for_range<K, HV>(in, in_v, s0, s1, [&](uint64_t, K k, uint32_t v, unsigned m) {
            uint32_t j = (uint32_t)(bucket_of(k, H) - b0);
            if (j >= nb) j = nb - 1;  // flagged in pass 1
            const uint32_t pos = smem_inc(s_cnt, j, m);
            const bool hot = staged && ((s_hot[j >> 5] >> (j & 31)) & 1u);
            if (staged && !hot) {
                if (pos < STAGE_CAP) {
                    s_keys[pos] = k;
                    if (HV) s_pay[pos] = v;
                } else {
                    atomicOr(err, DEVERR_BOUNDS);
                }
            } else if (pos < n) {
                out[pos] = k;
                if (HV) out_v[pos] = v;
            } else {
                atomicOr(err, DEVERR_BOUNDS);
            }
        });
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

size_t local_smem_bytes(size_t key_bytes, bool hv) {
    const size_t cap = LOCAL_STAGE_BYTES / (key_bytes + (hv ? 4 : 0));
    return (size_t)BPB * 4 + BPB / 8 + 2 * MAX_HOT * 4 + cap * (key_bytes + (hv ? 4 : 0));
}

template <typename K>
size_t pass_smem_bytes(bool payload) {
    constexpr int TILE = PassCfg<K>::TILE;
    return (size_t)TILE * sizeof(K) + (payload ? (size_t)TILE * 4 : 0) + TILE + 3 * RADIX * 4 + 16;
}

template <typename Kern>
unsigned grid_for(Kern kern, int threads, size_t smem) {
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, smem) != cudaSuccess || per_sm < 1)
        per_sm = 1;
    return (unsigned)(num_sms() * per_sm);
}

template <typename K, int PM, bool SEG>
cudaError_t launch_pass(const K* in, const uint32_t* in_v, uint64_t n, const Hasher& H, uint32_t dig_shift,
                        uint32_t dig_mask, uint32_t R, uint32_t P, uint32_t P2, const uint32_t* bin_start,
                        const uint32_t* seg_tile_start, uint32_t nseg, const Plan* plan, uint32_t* tile_ctr,
                        uint64_t* status, K* out, uint32_t* out_v, uint32_t* err, cudaStream_t s) {
    auto kern = k_part_pass<K, PM, SEG>;
    const size_t smem = pass_smem_bytes<K>(PM != 0);
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    launch_begin("part_scatter", s);
    kern<<<grid_for(kern, PASS_THREADS, smem), PASS_THREADS, smem, s>>>(in, in_v, n, H, dig_shift, dig_mask, R, P, P2,
                                                                       bin_start, seg_tile_start, nseg, plan,
                                                                       tile_ctr, status, out, out_v, err);
    launch_end("part_scatter", s);
    return cudaGetLastError();
}

template <typename K>
cudaError_t build_partitioned_impl(Table& t, const K* keys, const uint32_t* vals, cudaStream_t s) {
    constexpr int TILE = PassCfg<K>::TILE;
    const uint64_t n = t.n, B = t.B;
    const uint32_t P = (uint32_t)((B + BPB - 1) / BPB);
    const uint32_t P2 = P <= RADIX ? P : RADIX;
    const uint32_t P1 = (P + P2 - 1) / P2;
    const bool two = P1 > 1;
    const bool hv = t.has_values != 0;
    const uint64_t tiles_a = (n + TILE - 1) / TILE;
    const uint64_t tiles_b_max = tiles_a + P1 + 1;

    // scratch (zeroed part first): counters | bin_count[P] | statusA | statusB | huge_count
    //   | bin_start[P+1] | work[P] | seg_tile_start[P1+1] | huge_bin | huge_chunk_start | plan
    //   | huge_cursor | tmpA keys | tmpA vals | tmpB keys | tmpB vals
    auto al = [](size_t x) { return (x + 255) & ~size_t(255); };
    size_t off = 0;
    const size_t o_ctr = off; off += al(64);
    const size_t o_cnt = off; off += al((size_t)P * 4);
    const size_t o_status_a = off; off += al(two ? (size_t)tiles_a * P1 * 8 : 0);
    const size_t o_status_b = off; off += al((size_t)tiles_b_max * P2 * 8);
    const size_t o_hcount = off; off += al((size_t)MAX_HUGE * BPB * 4);
    const size_t zero_bytes = off;
    const size_t o_start = off; off += al((size_t)(P + 1) * 4);
    const size_t o_work = off; off += al((size_t)P * 4);
    const size_t o_seg = off; off += al((size_t)(P1 + 1) * 4);
    const size_t o_hbin = off; off += al((size_t)MAX_HUGE * 4);
    const size_t o_hcs = off; off += al((size_t)(MAX_HUGE + 1) * 4);
    const size_t o_plan = off; off += al(sizeof(Plan));
    const size_t o_hcur = off; off += al((size_t)MAX_HUGE * BPB * 4);
    const size_t o_ka = off; off += al(two ? n * sizeof(K) : 0);
    const size_t o_va = off; off += al(two && hv ? n * 4 : 0);
    const size_t o_kb = off; off += al(n * sizeof(K));
    const size_t o_vb = off; off += al(hv ? n * 4 : 0);
    void* mem = nullptr;
    cudaError_t e = dev_alloc(&mem, off, s);
    if (e != cudaSuccess) return e;
    char* base = static_cast<char*>(mem);
    uint32_t* ctr = reinterpret_cast<uint32_t*>(base + o_ctr);  // [0] pass A tiles, [1] pass B tiles, [2] local work
    uint32_t* bin_count = reinterpret_cast<uint32_t*>(base + o_cnt);
    uint64_t* status_a = reinterpret_cast<uint64_t*>(base + o_status_a);
    uint64_t* status_b = reinterpret_cast<uint64_t*>(base + o_status_b);
    uint32_t* huge_count = reinterpret_cast<uint32_t*>(base + o_hcount);
    uint32_t* bin_start = reinterpret_cast<uint32_t*>(base + o_start);
    uint32_t* work = reinterpret_cast<uint32_t*>(base + o_work);
    uint32_t* seg = reinterpret_cast<uint32_t*>(base + o_seg);
    uint32_t* huge_bin = reinterpret_cast<uint32_t*>(base + o_hbin);
    uint32_t* huge_cs = reinterpret_cast<uint32_t*>(base + o_hcs);
    Plan* plan = reinterpret_cast<Plan*>(base + o_plan);
    uint32_t* huge_cursor = reinterpret_cast<uint32_t*>(base + o_hcur);
    K* ka = reinterpret_cast<K*>(base + o_ka);
    uint32_t* va = reinterpret_cast<uint32_t*>(base + o_va);
    K* kb = reinterpret_cast<K*>(base + o_kb);
    uint32_t* vb = reinterpret_cast<uint32_t*>(base + o_vb);

    e = cudaMemsetAsync(base, 0, zero_bytes, s);
    // 1. bin histogram
    if (e == cudaSuccess) {
        auto kern = k_part_count<K>;
        const size_t smem = (size_t)P * 4;
        e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e == cudaSuccess) {
            unsigned g = grid_for(kern, PASS_THREADS, smem);
            const unsigned cap = (unsigned)num_sms() * 3;
            if (g > cap) g = cap;
            launch_begin("part_hist", s);
            kern<<<g, PASS_THREADS, smem, s>>>(keys, n, t.H, P, bin_count);
            launch_end("part_hist", s);
            e = cudaGetLastError();
        }
    }
    // 2. plan
    if (e == cudaSuccess) {
        const uint32_t big_t = (uint32_t)(LOCAL_STAGE_BYTES / (sizeof(K) + (hv ? 4 : 0)));
        launch_begin("part_plan", s);
        k_part_plan<<<1, 1024, 0, s>>>(bin_count, P, P1, P2, n, TILE, big_t, bin_start, seg, work, huge_bin, huge_cs,
                                       plan, t.offsets, B);
        launch_end("part_plan", s);
        e = cudaGetLastError();
    }
    // 3. partition passes
    const K* src = keys;
    const uint32_t* src_v = vals;
    const int pm_first = vals ? 1 : (hv ? 2 : 0);
    if (e == cudaSuccess && two) {
        if (pm_first == 1)
            e = launch_pass<K, 1, false>(keys, vals, n, t.H, 7, 0xffffffffu, P1, P, P2, bin_start, seg, P1, plan,
                                         ctr + 0, status_a, ka, va, t.err, s);
        else if (pm_first == 2)
            e = launch_pass<K, 2, false>(keys, nullptr, n, t.H, 7, 0xffffffffu, P1, P, P2, bin_start, seg, P1, plan,
                                         ctr + 0, status_a, ka, va, t.err, s);
        else
            e = launch_pass<K, 0, false>(keys, nullptr, n, t.H, 7, 0xffffffffu, P1, P, P2, bin_start, seg, P1, plan,
                                         ctr + 0, status_a, ka, nullptr, t.err, s);
        src = ka;
        src_v = hv ? va : nullptr;
    }
    if (e == cudaSuccess) {
        const int pm = two ? (hv ? 1 : 0) : pm_first;
        const uint32_t mask = two ? (RADIX - 1) : 0xffffffffu;
        if (pm == 1)
            e = launch_pass<K, 1, true>(src, src_v, n, t.H, 0, mask, P2, P, P2, bin_start, seg, P1, plan, ctr + 1,
                                        status_b, kb, vb, t.err, s);
        else if (pm == 2)
            e = launch_pass<K, 2, true>(src, nullptr, n, t.H, 0, mask, P2, P, P2, bin_start, seg, P1, plan, ctr + 1,
                                        status_b, kb, vb, t.err, s);
        else
            e = launch_pass<K, 0, true>(src, nullptr, n, t.H, 0, mask, P2, P, P2, bin_start, seg, P1, plan, ctr + 1,
                                        status_b, kb, nullptr, t.err, s);
    }
    // 4. huge bins: chunk histograms, then their offsets and cursors
    if (e == cudaSuccess) {
        auto kern = k_huge_count<K>;
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
        k_huge_scan<<<MAX_HUGE, 1024, 0, s>>>(bin_start, huge_bin, plan, huge_count, huge_cursor, t.offsets, B);
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
                kb, hv ? vb : nullptr, n, t.H, bin_start, work, huge_bin, huge_cs, plan, huge_cursor, ctr + 2,
                t.offsets, kout, t.values, t.err);
            launch_end("bin_build", s);
            return cudaGetLastError();
        };
        e = hv ? run(k_bin_local<K, true>) : run(k_bin_local<K, false>);
    }
    dev_free(mem, s);
    return e;
}

}  // namespace

bool partition_supported(uint64_t B) { return (B + BPB - 1) / BPB <= MAX_BINS; }

cudaError_t build_partitioned(Table& t, const void* d_keys, const void* d_values, cudaStream_t s) {
    const uint32_t* vals = static_cast<const uint32_t*>(d_values);
    if (t.key_bytes == 4) return build_partitioned_impl<uint32_t>(t, static_cast<const uint32_t*>(d_keys), vals, s);
    return build_partitioned_impl<uint64_t>(t, static_cast<const uint64_t*>(d_keys), vals, s);
}

}  // namespace hg
