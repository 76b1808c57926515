// Batched HashGraph: many independent tables of uneven size, every one built
// (Algorithm 1) and probed (Sec. 3.3) in a single persistent launch.
//
// One CTA takes a whole table at a time (largest tables first, claimed from
// an atomic counter), so tables need no synchronisation between CTAs and the
// launch is one kernel, captured once in a CUDA graph and replayed.
//
//  * A table with at most 2^bin_shift buckets and at most fuse_keys keys is
//    built entirely in shared memory: histogram, exclusive scan and scatter
//    fused, the CSR arrays written out once, and its queries answered from the
//    shared-memory copy.
//  * A larger table is first partitioned inside the CTA by bin (bucket >>
//    bin_shift, the binning of Sec. 3.2) -- keys and queries both, through
//    shared-memory-staged tiles -- and then each bin is built by a shared-memory
//    counting sort and its queries are answered while the bin is resident
//    (the per-bucket list intersection of Sec. 3.3, a bin at a time).  Counts
//    come back to query order through each query's recorded grouped position.
//
// Results equal the single-table build's: per-table offsets are those of
// Algorithm 1, and the order inside a bucket is free.
#include <algorithm>
#include <cstdio>
#include <new>
#include <vector>

#include "hg_device.cuh"

namespace hg {
namespace {

constexpr uint32_t BATCH_STAGE_KEYS = 16384;  // keys of one bin staged in shared memory (64 KiB)
constexpr uint32_t BATCH_MAX_BINS = 512;      // bins per table
constexpr int BATCH_IPT = 8;                  // elements per thread per partition tile
constexpr uint64_t BATCH_MAX_BUCKETS = (uint64_t)BATCH_MAX_BINS << 12;  // for the smallest bin size

struct BatchTable {
    uint64_t key_begin;  // first key of the table in the concatenated key (and CSR key) arrays
    uint64_t q_begin;    // first query (and count) of the table
    uint64_t off_begin;  // first offset of the table: the sum of (B + 1) over earlier tables
    uint32_t n, q;
    Hasher H;  // H.B = the table's bucket count
};

struct BatchArgs {
    const BatchTable* tabs;
    const uint32_t* order;  // table indices, largest first
    uint32_t n_tables;
    uint32_t fuse_keys;
    const uint32_t* keys;
    const uint32_t* queries;
    uint32_t* keys_out;
    uint32_t* offsets_out;
    uint32_t* counts;
    uint32_t* tmp_keys;  // partitioned tables: keys grouped by bin (same slots as keys)
    uint32_t* tmp_q;     // queries grouped by bin (same slots as queries)
    uint32_t* tmp_pos;   // each query's slot in tmp_q, in query order
    uint32_t* tmp_cnt;   // counts in tmp_q order
    uint32_t* work_ctr;
    uint32_t* err;
};

// In-place exclusive scan of a[0, m) by the block; returns the total.  Ends
// with a barrier, so a[] may be read by any thread afterwards.
template <int T>
__device__ uint32_t cta_scan(uint32_t* a, uint32_t m, uint32_t* s_warp) {
    const unsigned lane = lane_id();
    const int w = threadIdx.x >> 5;
    const uint32_t per = (m + T - 1) / T;
    const uint32_t i0 = min(m, threadIdx.x * per), i1 = min(m, i0 + per);
    uint32_t sum = 0;
    for (uint32_t i = i0; i < i1; ++i) sum += a[i];
    const uint32_t incl = warp_inclusive_scan(sum);
    if (lane == 31) s_warp[w] = incl;
    __syncthreads();
    if (w == 0) {
        const uint32_t x = (int)lane < T / 32 ? s_warp[lane] : 0u;
        const uint32_t xi = warp_inclusive_scan(x);
        if ((int)lane < T / 32) s_warp[lane] = xi - x;
        if (lane == 31) s_warp[32] = xi;
    }
    __syncthreads();
    uint32_t run = s_warp[w] + incl - sum;
    for (uint32_t i = i0; i < i1; ++i) {
        const uint32_t v = a[i];
        a[i] = run;
        run += v;
    }
    const uint32_t total = s_warp[32];
    __syncthreads();
    return total;
}

struct BatchSmem {
    uint32_t* cnt;    // [BPB + 1] bucket counters / cursors of the current bin
    uint32_t* stage;  // [BATCH_STAGE_KEYS] a bin's keys; also a partition tile's (key, slot) pairs
    uint32_t* kb;     // [BATCH_MAX_BINS + 1] key bin starts
    uint32_t* qb;     // [BATCH_MAX_BINS + 1] query bin starts
    uint32_t* cur;    // [BATCH_MAX_BINS] partition cursors
    uint32_t* tc;     // [BATCH_MAX_BINS] tile counts
    uint32_t* tx;     // [BATCH_MAX_BINS] tile-local starts
    uint32_t* ty;     // [BATCH_MAX_BINS] slots of the tile's runs
    uint32_t* warp;   // [33]
};

template <int BSHIFT>
size_t batch_smem_bytes() {
    const size_t cnt = (((size_t)(1u << BSHIFT) + 1) * 4 + 15) / 16 * 16;
    const size_t bins = ((size_t)(BATCH_MAX_BINS + 1) * 4 + 15) / 16 * 16;
    return cnt + (size_t)BATCH_STAGE_KEYS * 4 + 2 * bins + 4 * (size_t)BATCH_MAX_BINS * 4;
}

template <int BSHIFT>
__device__ BatchSmem batch_smem(unsigned char* base, uint32_t* s_warp) {
    BatchSmem S;
    const size_t cnt = (((size_t)(1u << BSHIFT) + 1) * 4 + 15) / 16 * 16;
    const size_t bins = ((size_t)(BATCH_MAX_BINS + 1) * 4 + 15) / 16 * 16;
    S.cnt = reinterpret_cast<uint32_t*>(base);
    S.stage = reinterpret_cast<uint32_t*>(base + cnt);
    unsigned char* p = base + cnt + (size_t)BATCH_STAGE_KEYS * 4;
    S.kb = reinterpret_cast<uint32_t*>(p);
    S.qb = reinterpret_cast<uint32_t*>(p + bins);
    S.cur = reinterpret_cast<uint32_t*>(p + 2 * bins);
    S.tc = S.cur + BATCH_MAX_BINS;
    S.tx = S.tc + BATCH_MAX_BINS;
    S.ty = S.tx + BATCH_MAX_BINS;
    S.warp = s_warp;
    return S;
}

// Keys (or queries) walked in bucket order: count of `key` in src[lo, hi).
__device__ __forceinline__ uint32_t walk_count(const uint32_t* src, uint32_t lo, uint32_t hi, uint32_t key) {
    uint32_t c = 0;
    for (uint32_t x = lo; x < hi; ++x) c += (src[x] == key);
    return c;
}

// The whole table in shared memory: histogram, scan, scatter, write-out, probe.
template <int T, int BSHIFT>
__device__ void fused_table(const BatchArgs& A, const BatchTable& tb, const BatchSmem& S) {
    const uint32_t B = (uint32_t)tb.H.B, n = tb.n, q = tb.q;
    const uint32_t* kin = A.keys + tb.key_begin;
    for (uint32_t j = threadIdx.x; j <= B; j += T) S.cnt[j] = 0;
    __syncthreads();
    for (uint32_t i = threadIdx.x; i < n; i += T) atomicAdd(S.cnt + bucket_of(kin[i], tb.H), 1u);
    __syncthreads();
    cta_scan<T>(S.cnt, B, S.warp);  // cnt[j] = start of bucket j
    uint32_t* offs = A.offsets_out + tb.off_begin;
    for (uint32_t j = threadIdx.x; j < B; j += T) offs[j] = S.cnt[j];
    if (threadIdx.x == 0) offs[B] = n;
    __syncthreads();
    for (uint32_t i = threadIdx.x; i < n; i += T) {
        const uint32_t k = kin[i];
        const uint32_t pos = atomicAdd(S.cnt + bucket_of(k, tb.H), 1u);
        if (pos < BATCH_STAGE_KEYS) S.stage[pos] = k;
        else atomicOr(A.err, DEVERR_BOUNDS);
    }
    __syncthreads();
    uint32_t* kout = A.keys_out + tb.key_begin;
    for (uint32_t i = threadIdx.x; i < n; i += T) kout[i] = S.stage[i];
    // cnt[j] is now the end of bucket j (= the start of bucket j + 1)
    const uint32_t* qin = A.queries + tb.q_begin;
    uint32_t* cout = A.counts + tb.q_begin;
    for (uint32_t i = threadIdx.x; i < q; i += T) {
        const uint32_t k = qin[i];
        const uint32_t j = bucket_of(k, tb.H);
        const uint32_t lo = j ? S.cnt[j - 1] : 0u, hi = S.cnt[j];
        cout[i] = walk_count(S.stage, lo, min(hi, BATCH_STAGE_KEYS), k);
    }
    __syncthreads();
}

// Partition of in[0, n) by bin into out[] (bin d's run starts at starts[d]),
// through shared-memory tiles; pos_out (optional) receives each element's slot.
template <int T, int BSHIFT>
__device__ void part_scatter(const uint32_t* __restrict__ in, uint32_t n, const Hasher& H, uint32_t nb,
                             const uint32_t* starts, uint32_t* __restrict__ out, uint32_t* __restrict__ pos_out,
                             const BatchSmem& S, uint32_t* err) {
    constexpr uint32_t TILE = (uint32_t)T * BATCH_IPT;
    static_assert(TILE * 8 <= BATCH_STAGE_KEYS * 4, "tile staging fits the stage buffer");
    uint2* s_kd = reinterpret_cast<uint2*>(S.stage);
    const unsigned lane = lane_id();
    for (uint32_t d = threadIdx.x; d < nb; d += T) S.cur[d] = starts[d];
    for (uint32_t t0 = 0; t0 < n; t0 += TILE) {
        const uint32_t cnt_tile = min(TILE, n - t0);
        for (uint32_t d = threadIdx.x; d < nb; d += T) S.tc[d] = 0;
        __syncthreads();
        uint32_t e[BATCH_IPT], dg[BATCH_IPT], rk[BATCH_IPT];
#pragma unroll
        for (int j = 0; j < BATCH_IPT; ++j) {
            const uint32_t li = threadIdx.x + j * T;
            dg[j] = 0xffffffffu;
            if (li < cnt_tile) {
                e[j] = in[t0 + li];
                const uint32_t d = min(bucket_of(e[j], H) >> BSHIFT, nb - 1);
                dg[j] = d;
                rk[j] = atomicAdd(S.tc + d, 1u);
            }
        }
        __syncthreads();
        if (threadIdx.x < 32) {  // tile-local starts and the runs' slots (one warp, nb <= 512)
            const uint32_t per = (nb + 31) / 32;
            const uint32_t d0 = min(nb, lane * per), d1 = min(nb, d0 + per);
            uint32_t sum = 0;
            for (uint32_t d = d0; d < d1; ++d) sum += S.tc[d];
            uint32_t run = warp_inclusive_scan(sum) - sum;
            for (uint32_t d = d0; d < d1; ++d) {
                const uint32_t c = S.tc[d];
                S.tx[d] = run;
                S.ty[d] = S.cur[d];
                S.cur[d] += c;
                run += c;
            }
        }
        __syncthreads();
#pragma unroll
        for (int j = 0; j < BATCH_IPT; ++j) {
            if (dg[j] != 0xffffffffu) {
                const uint32_t p = S.tx[dg[j]] + rk[j];
                const uint32_t dst = S.ty[dg[j]] + rk[j];
                if (p < TILE) s_kd[p] = make_uint2(e[j], dst);
                else atomicOr(err, DEVERR_BOUNDS);
                if (pos_out) pos_out[t0 + threadIdx.x + j * T] = dst;
            }
        }
        __syncthreads();
        for (uint32_t i = threadIdx.x; i < cnt_tile; i += T) {
            const uint2 kd = s_kd[i];
            if (kd.y < n) out[kd.y] = kd.x;
            else atomicOr(err, DEVERR_BOUNDS);
        }
        __syncthreads();
    }
}

// A table too large to build in shared memory at once: partition by bin, then
// build and probe each bin while it is resident.
template <int T, int BSHIFT>
__device__ void part_table(const BatchArgs& A, const BatchTable& tb, const BatchSmem& S) {
    constexpr uint32_t BPB = 1u << BSHIFT;
    const uint32_t B = (uint32_t)tb.H.B, n = tb.n, q = tb.q;
    const uint32_t nb = (B + BPB - 1) >> BSHIFT;  // <= BATCH_MAX_BINS (checked on the host)
    const uint32_t* kin = A.keys + tb.key_begin;
    const uint32_t* qin = A.queries + tb.q_begin;
    for (uint32_t d = threadIdx.x; d <= nb; d += T) {
        S.kb[d] = 0;
        S.qb[d] = 0;
    }
    __syncthreads();
    for (uint32_t i = threadIdx.x; i < n; i += T) atomicAdd(S.kb + min(bucket_of(kin[i], tb.H) >> BSHIFT, nb - 1), 1u);
    for (uint32_t i = threadIdx.x; i < q; i += T) atomicAdd(S.qb + min(bucket_of(qin[i], tb.H) >> BSHIFT, nb - 1), 1u);
    __syncthreads();
    cta_scan<T>(S.kb, nb, S.warp);
    cta_scan<T>(S.qb, nb, S.warp);
    if (threadIdx.x == 0) {
        S.kb[nb] = n;
        S.qb[nb] = q;
    }
    __syncthreads();
    uint32_t* tk = A.tmp_keys + tb.key_begin;
    uint32_t* tq = A.tmp_q + tb.q_begin;
    uint32_t* tpos = A.tmp_pos + tb.q_begin;
    uint32_t* tcnt = A.tmp_cnt + tb.q_begin;
    part_scatter<T, BSHIFT>(kin, n, tb.H, nb, S.kb, tk, nullptr, S, A.err);
    part_scatter<T, BSHIFT>(qin, q, tb.H, nb, S.qb, tq, tpos, S, A.err);

    uint32_t* offs = A.offsets_out + tb.off_begin;
    uint32_t* kout_t = A.keys_out + tb.key_begin;
    for (uint32_t b = 0; b < nb; ++b) {
        const uint32_t k0 = S.kb[b], nk = S.kb[b + 1] - k0;
        const uint32_t bb0 = b << BSHIFT, nbk = min(BPB, B - bb0);
        const uint32_t* bk = tk + k0;
        uint32_t* kout = kout_t + k0;
        const bool staged = nk <= BATCH_STAGE_KEYS;
        for (uint32_t j = threadIdx.x; j <= nbk; j += T) S.cnt[j] = 0;
        __syncthreads();
        for (uint32_t i = threadIdx.x; i < nk; i += T)
            atomicAdd(S.cnt + min(bucket_of(bk[i], tb.H) - bb0, nbk - 1), 1u);
        __syncthreads();
        cta_scan<T>(S.cnt, nbk, S.warp);
        for (uint32_t j = threadIdx.x; j < nbk; j += T) offs[bb0 + j] = k0 + S.cnt[j];
        __syncthreads();
        for (uint32_t i = threadIdx.x; i < nk; i += T) {
            const uint32_t k = bk[i];
            const uint32_t pos = atomicAdd(S.cnt + min(bucket_of(k, tb.H) - bb0, nbk - 1), 1u);
            if (pos >= nk) atomicOr(A.err, DEVERR_BOUNDS);
            else if (staged) S.stage[pos] = k;
            else kout[pos] = k;
        }
        __syncthreads();
        if (staged)
            for (uint32_t i = threadIdx.x; i < nk; i += T) kout[i] = S.stage[i];
        // the bin's queries, answered from the resident bin (cnt[j] = end of bucket j)
        const uint32_t q0 = S.qb[b], nq = S.qb[b + 1] - q0;
        const uint32_t* src = staged ? S.stage : kout;
        for (uint32_t i = threadIdx.x; i < nq; i += T) {
            const uint32_t k = tq[q0 + i];
            const uint32_t j = min(bucket_of(k, tb.H) - bb0, nbk - 1);
            const uint32_t lo = j ? S.cnt[j - 1] : 0u, hi = min(S.cnt[j], nk);
            tcnt[q0 + i] = walk_count(src, lo, hi, k);
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) offs[B] = n;
    // counts back to query order
    uint32_t* cout = A.counts + tb.q_begin;
    for (uint32_t i = threadIdx.x; i < q; i += T) {
        const uint32_t p = tpos[i];
        cout[i] = p < q ? tcnt[p] : 0u;
    }
    __syncthreads();
}

template <int T, int BSHIFT>
__global__ void __launch_bounds__(T, 2) k_batch(BatchArgs A) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ uint32_t s_warp[33];
    __shared__ uint32_t s_item;
    const BatchSmem S = batch_smem<BSHIFT>(smem, s_warp);
    while (true) {
        if (threadIdx.x == 0) s_item = atomicAdd(A.work_ctr, 1u);
        __syncthreads();
        const uint32_t it = s_item;
        __syncthreads();  // every thread has read s_item before thread 0 claims again
        if (it >= A.n_tables) break;
        const BatchTable tb = A.tabs[A.order[it]];
        if (tb.H.B <= (1u << BSHIFT) && tb.n <= A.fuse_keys && tb.n <= BATCH_STAGE_KEYS)
            fused_table<T, BSHIFT>(A, tb, S);
        else
            part_table<T, BSHIFT>(A, tb, S);
    }
}

// Byte-model helper: stats[0] += the bucket length of every query (the keys
// its walk visits), from the built tables.  One CTA per table.
__global__ void __launch_bounds__(256) k_batch_walk(const BatchTable* __restrict__ tabs, uint32_t n_tables,
                                                    const uint32_t* __restrict__ offsets_out,
                                                    const uint32_t* __restrict__ queries,
                                                    unsigned long long* stats) {
    uint64_t w = 0;
    for (uint32_t t = blockIdx.x; t < n_tables; t += gridDim.x) {
        const BatchTable tb = tabs[t];
        const uint32_t* offs = offsets_out + tb.off_begin;
        for (uint32_t i = threadIdx.x; i < tb.q; i += blockDim.x) {
            const uint32_t j = bucket_of(queries[tb.q_begin + i], tb.H);
            w += offs[j + 1] - offs[j];
        }
    }
    const uint64_t tot = warp_sum(w);
    if (lane_id() == 0 && tot) atomicAdd(stats, (unsigned long long)tot);
}

}  // namespace
}  // namespace hg

// ------------------------------------------------------------------ host --
using namespace hg;

struct hg_batch {
    int device = 0;
    uint32_t n_tables = 0;
    uint64_t total_keys = 0, total_q = 0, total_off = 0;
    std::vector<BatchTable> h_tabs;
    std::vector<uint32_t> h_order;
    BatchTable* d_tabs = nullptr;
    uint32_t* d_order = nullptr;
    uint32_t* keys_out = nullptr;
    uint32_t* offsets_out = nullptr;
    uint32_t* tmp = nullptr;   // tmp_keys | tmp_q | tmp_pos | tmp_cnt
    uint32_t* ctl = nullptr;   // [0] work counter, [1] error word
    hg_batch_params params{512, 13, BATCH_STAGE_KEYS};
    cudaGraphExec_t graph = nullptr;
    const void* g_keys = nullptr;
    const void* g_q = nullptr;
    void* g_counts = nullptr;
    hg_batch_params g_params{};
};

namespace {

thread_local char g_bmsg[320];

hg_status bfail(hg_status st, const char* msg) {
    set_error_message(msg);
    return st;
}

hg_status bcuda(cudaError_t e, const char* what) {
    cudaGetLastError();
    snprintf(g_bmsg, sizeof(g_bmsg), "%s: %s", what, cudaGetErrorString(e));
    return bfail(e == cudaErrorMemoryAllocation ? HG_ERR_OOM : HG_ERR_CUDA, g_bmsg);
}

bool params_ok(const hg_batch_params& p) {
    return (p.threads == 256 || p.threads == 512) && (p.bin_shift == 12 || p.bin_shift == 13) && p.fuse_keys >= 1;
}

template <int T, int BSHIFT>
cudaError_t launch_batch_kernel(const BatchArgs& A, cudaStream_t s) {
    auto kern = k_batch<T, BSHIFT>;
    const size_t smem = batch_smem_bytes<BSHIFT>();
    int per_sm = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, T, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) per_sm = 1;
    kern<<<num_sms() * per_sm, T, smem, s>>>(A);
    return cudaGetLastError();
}

template <int T, int BSHIFT>
cudaError_t prepare_kernel() {
    return cudaFuncSetAttribute(k_batch<T, BSHIFT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)batch_smem_bytes<BSHIFT>());
}

cudaError_t prepare_all() {
    cudaError_t e = prepare_kernel<256, 12>();
    if (e == cudaSuccess) e = prepare_kernel<256, 13>();
    if (e == cudaSuccess) e = prepare_kernel<512, 12>();
    if (e == cudaSuccess) e = prepare_kernel<512, 13>();
    return e;
}

cudaError_t enqueue_batch(hg_batch* b, const hg_batch_params& p, const uint32_t* keys, const uint32_t* queries,
                          uint32_t* counts, cudaStream_t s) {
    BatchArgs A{};
    A.tabs = b->d_tabs;
    A.order = b->d_order;
    A.n_tables = b->n_tables;
    A.fuse_keys = p.fuse_keys;
    A.keys = keys;
    A.queries = queries;
    A.keys_out = b->keys_out;
    A.offsets_out = b->offsets_out;
    A.counts = counts;
    A.tmp_keys = b->tmp;
    A.tmp_q = b->tmp + b->total_keys;
    A.tmp_pos = A.tmp_q + b->total_q;
    A.tmp_cnt = A.tmp_pos + b->total_q;
    A.work_ctr = b->ctl;
    A.err = b->ctl + 1;
    cudaError_t e = cudaMemsetAsync(b->ctl, 0, sizeof(uint32_t), s);
    if (e != cudaSuccess) return e;
    if (p.threads == 256) return p.bin_shift == 12 ? launch_batch_kernel<256, 12>(A, s) : launch_batch_kernel<256, 13>(A, s);
    return p.bin_shift == 12 ? launch_batch_kernel<512, 12>(A, s) : launch_batch_kernel<512, 13>(A, s);
}

void drop_graph(hg_batch* b) {
    if (b->graph) cudaGraphExecDestroy(b->graph);
    b->graph = nullptr;
}

// One graph per (inputs, outputs, parameters); replayed while they stay the same.
cudaError_t run_graph(hg_batch* b, const uint32_t* keys, const uint32_t* queries, uint32_t* counts, cudaStream_t s) {
    const hg_batch_params& p = b->params;
    const bool same = b->graph && b->g_keys == keys && b->g_q == queries && b->g_counts == counts &&
                      b->g_params.threads == p.threads && b->g_params.bin_shift == p.bin_shift &&
                      b->g_params.fuse_keys == p.fuse_keys;
    if (!same) {
        drop_graph(b);
        cudaError_t e = prepare_all();
        if (e != cudaSuccess) return e;
        // the legacy default stream cannot be captured, and a stream the caller is
        // already capturing takes the launch into the caller's own graph
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        if (s != nullptr && s != cudaStreamLegacy) {
            e = cudaStreamIsCapturing(s, &cs);
            if (e != cudaSuccess) return e;
        }
        if (s == nullptr || s == cudaStreamLegacy || cs != cudaStreamCaptureStatusNone) {
            launch_begin("batch", s);
            e = enqueue_batch(b, p, keys, queries, counts, s);
            launch_end("batch", s);
            return e;
        }
        e = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) return e;
        cudaError_t e2 = enqueue_batch(b, p, keys, queries, counts, s);
        cudaGraph_t g = nullptr;
        e = cudaStreamEndCapture(s, &g);
        if (e2 != cudaSuccess) e = e2;
        if (e == cudaSuccess) e = cudaGraphInstantiate(&b->graph, g, 0);
        if (g) cudaGraphDestroy(g);
        if (e != cudaSuccess) {
            b->graph = nullptr;
            return e;
        }
        b->g_keys = keys;
        b->g_q = queries;
        b->g_counts = counts;
        b->g_params = p;
    }
    launch_begin("batch", s);
    cudaError_t e = cudaGraphLaunch(b->graph, s);
    launch_end("batch", s);
    return e;
}

void free_batch(hg_batch* b, cudaStream_t s) {
    drop_graph(b);
    dev_free(b->d_tabs, s);
    dev_free(b->d_order, s);
    dev_free(b->keys_out, s);
    dev_free(b->offsets_out, s);
    dev_free(b->tmp, s);
    dev_free(b->ctl, s);
    delete b;
}

}  // namespace

extern "C" {

hg_status hg_batch_create(const hg_config* cfg, uint32_t n_tables, const uint64_t* h_key_offsets,
                          const uint64_t* h_num_buckets, const uint64_t* h_query_offsets, hg_stream_t st,
                          hg_batch** out) {
    cudaStream_t s = reinterpret_cast<cudaStream_t>(st);
    if (!out) return bfail(HG_ERR_INVALID_ARG, "hg_batch_create: out is NULL");
    *out = nullptr;
    if (!cfg || !h_key_offsets || !h_num_buckets) return bfail(HG_ERR_INVALID_ARG, "hg_batch_create: NULL argument");
    if (cfg->key_bytes != 4 || cfg->value_bytes != 0)
        return bfail(HG_ERR_INVALID_ARG, "hg_batch_create: batches hold 32-bit keys without values");
    if (n_tables == 0) return bfail(HG_ERR_INVALID_ARG, "hg_batch_create: n_tables is 0");
    if (h_key_offsets[0] != 0 || (h_query_offsets && h_query_offsets[0] != 0))
        return bfail(HG_ERR_INVALID_ARG, "hg_batch_create: offsets must start at 0");
    hg_batch* b = new (std::nothrow) hg_batch;
    if (!b) return bfail(HG_ERR_OOM, "hg_batch_create: host allocation failed");
    cudaGetDevice(&b->device);
    b->n_tables = n_tables;
    b->h_tabs.resize(n_tables);
    uint64_t off = 0;
    for (uint32_t t = 0; t < n_tables; ++t) {
        const uint64_t k0 = h_key_offsets[t], k1 = h_key_offsets[t + 1];
        const uint64_t q0 = h_query_offsets ? h_query_offsets[t] : 0, q1 = h_query_offsets ? h_query_offsets[t + 1] : 0;
        const uint64_t B = h_num_buckets[t];
        if (k1 < k0 || q1 < q0 || k1 - k0 > 0xffffffffull || q1 - q0 > 0xffffffffull || B < 1 ||
            B > BATCH_MAX_BUCKETS) {
            snprintf(g_bmsg, sizeof(g_bmsg),
                     "hg_batch_create: table %u has a bad key/query range or num_buckets = %llu outside [1, %llu]", t,
                     (unsigned long long)B, (unsigned long long)BATCH_MAX_BUCKETS);
            delete b;
            return bfail(HG_ERR_INVALID_ARG, g_bmsg);
        }
        BatchTable& tb = b->h_tabs[t];
        tb.key_begin = k0;
        tb.q_begin = q0;
        tb.off_begin = off;
        tb.n = (uint32_t)(k1 - k0);
        tb.q = (uint32_t)(q1 - q0);
        tb.H = make_hasher(4, B, cfg->seed);
        off += B + 1;
    }
    b->total_keys = h_key_offsets[n_tables];
    b->total_q = h_query_offsets ? h_query_offsets[n_tables] : 0;
    b->total_off = off;
    // largest tables first, so that the last CTAs to finish hold small ones
    b->h_order.resize(n_tables);
    for (uint32_t t = 0; t < n_tables; ++t) b->h_order[t] = t;
    std::stable_sort(b->h_order.begin(), b->h_order.end(), [&](uint32_t x, uint32_t y) {
        return (uint64_t)b->h_tabs[x].n + b->h_tabs[x].q > (uint64_t)b->h_tabs[y].n + b->h_tabs[y].q;
    });
    cudaError_t e = dev_alloc(reinterpret_cast<void**>(&b->d_tabs), sizeof(BatchTable) * n_tables, s);
    if (e == cudaSuccess) e = dev_alloc(reinterpret_cast<void**>(&b->d_order), 4ull * n_tables, s);
    if (e == cudaSuccess) e = dev_alloc(reinterpret_cast<void**>(&b->keys_out), 4 * b->total_keys + 16, s);
    if (e == cudaSuccess) e = dev_alloc(reinterpret_cast<void**>(&b->offsets_out), 4 * b->total_off + 16, s);
    if (e == cudaSuccess) e = dev_alloc(reinterpret_cast<void**>(&b->tmp), 4 * (b->total_keys + 3 * b->total_q) + 16, s);
    if (e == cudaSuccess) e = dev_alloc(reinterpret_cast<void**>(&b->ctl), 16, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(b->ctl, 0, 16, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(b->d_tabs, b->h_tabs.data(), sizeof(BatchTable) * n_tables, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(b->d_order, b->h_order.data(), 4ull * n_tables, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);  // the host descriptor copies are read before return
    if (e != cudaSuccess) {
        hg_status r = bcuda(e, "hg_batch_create");
        free_batch(b, s);
        return r;
    }
    *out = b;
    return HG_OK;
}

hg_status hg_batch_run(hg_batch* b, const uint32_t* d_keys, const uint32_t* d_queries, uint32_t* d_counts,
                       hg_stream_t st) {
    if (!b) return bfail(HG_ERR_INVALID_ARG, "hg_batch_run: batch is NULL");
    if ((b->total_keys && !d_keys) || (b->total_q && (!d_queries || !d_counts)))
        return bfail(HG_ERR_INVALID_ARG, "hg_batch_run: NULL keys, queries or counts");
    cudaError_t e = run_graph(b, d_keys, d_queries, d_counts, reinterpret_cast<cudaStream_t>(st));
    return e == cudaSuccess ? HG_OK : bcuda(e, "hg_batch_run");
}

hg_status hg_batch_set_params(hg_batch* b, const hg_batch_params* p) {
    if (!b || !p || !params_ok(*p))
        return bfail(HG_ERR_INVALID_ARG, "hg_batch_set_params: threads must be 256 or 512, bin_shift 12 or 13");
    b->params = *p;
    return HG_OK;
}

hg_status hg_batch_get_params(const hg_batch* b, hg_batch_params* p) {
    if (!b || !p) return bfail(HG_ERR_INVALID_ARG, "hg_batch_get_params: NULL argument");
    *p = b->params;
    return HG_OK;
}

hg_status hg_batch_tune(hg_batch* b, const uint32_t* d_keys, const uint32_t* d_queries, uint32_t* d_counts,
                        hg_stream_t st, hg_batch_params* chosen) {
    if (!b) return bfail(HG_ERR_INVALID_ARG, "hg_batch_tune: batch is NULL");
    if ((b->total_keys && !d_keys) || (b->total_q && (!d_queries || !d_counts)))
        return bfail(HG_ERR_INVALID_ARG, "hg_batch_tune: NULL keys, queries or counts");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(st);
    cudaError_t e = prepare_all();
    if (e != cudaSuccess) return bcuda(e, "hg_batch_tune");
    std::vector<hg_batch_params> cand;
    for (uint32_t threads : {256u, 512u})
        for (uint32_t shift : {12u, 13u})
            for (uint32_t fuse : {1u << shift, 1u << (shift - 1)}) cand.push_back(hg_batch_params{threads, shift, fuse});
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    float best = 0.f;
    hg_batch_params bestp = b->params;
    for (size_t c = 0; c < cand.size() && e == cudaSuccess; ++c) {
        e = enqueue_batch(b, cand[c], d_keys, d_queries, d_counts, s);  // warm-up
        if (e == cudaSuccess) e = cudaEventRecord(e0, s);
        for (int r = 0; r < 2 && e == cudaSuccess; ++r) e = enqueue_batch(b, cand[c], d_keys, d_queries, d_counts, s);
        if (e == cudaSuccess) e = cudaEventRecord(e1, s);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        float ms = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (e == cudaSuccess && (c == 0 || ms < best)) {
            best = ms;
            bestp = cand[c];
        }
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (e != cudaSuccess) return bcuda(e, "hg_batch_tune");
    b->params = bestp;
    if (chosen) *chosen = bestp;
    return HG_OK;
}

hg_status hg_batch_view(const hg_batch* b, uint32_t table, const void** d_offsets, const void** d_keys, uint64_t* n,
                        uint64_t* num_buckets) {
    if (!b || table >= b->n_tables) return bfail(HG_ERR_INVALID_ARG, "hg_batch_view: bad batch or table index");
    const BatchTable& tb = b->h_tabs[table];
    if (d_offsets) *d_offsets = b->offsets_out + tb.off_begin;
    if (d_keys) *d_keys = b->keys_out + tb.key_begin;
    if (n) *n = tb.n;
    if (num_buckets) *num_buckets = tb.H.B;
    return HG_OK;
}

hg_status hg_batch_sync(const hg_batch* b, hg_stream_t st) {
    if (!b) return bfail(HG_ERR_INVALID_ARG, "hg_batch_sync: batch is NULL");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(st);
    uint32_t err = 0;
    cudaError_t e = cudaMemcpyAsync(&err, b->ctl + 1, sizeof(err), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return bcuda(e, "hg_batch_sync");
    if (err) return bfail(HG_ERR_CUDA, "hg_batch_sync: a batch kernel found an index out of range");
    return HG_OK;
}

hg_status hg_batch_walk_stats(const hg_batch* b, const uint32_t* d_queries, uint64_t* d_stats, hg_stream_t st) {
    if (!b || !d_stats || (b->total_q && !d_queries))
        return bfail(HG_ERR_INVALID_ARG, "hg_batch_walk_stats: NULL argument");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(st);
    cudaError_t e = cudaMemsetAsync(d_stats, 0, sizeof(uint64_t), s);
    if (e == cudaSuccess && b->total_q) {
        const unsigned g = std::min<unsigned>(b->n_tables, (unsigned)num_sms() * 8);
        launch_begin("walk_stats", s);
        k_batch_walk<<<g, 256, 0, s>>>(b->d_tabs, b->n_tables, b->offsets_out, d_queries,
                                       reinterpret_cast<unsigned long long*>(d_stats));
        launch_end("walk_stats", s);
        e = cudaGetLastError();
    }
    return e == cudaSuccess ? HG_OK : bcuda(e, "hg_batch_walk_stats");
}

hg_status hg_batch_free(hg_batch* b, hg_stream_t st) {
    if (b) free_batch(b, reinterpret_cast<cudaStream_t>(st));
    return HG_OK;
}

}  // extern "C"
