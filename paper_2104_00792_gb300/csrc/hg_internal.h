// Internal host-side declarations shared by the library's translation units.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "hashgraph.h"

namespace hg {

// Device-side error bits (the table's error word).
enum : uint32_t {
    DEVERR_TIMEOUT = 1u,   // a decoupled-lookback wait ran out
    DEVERR_BOUNDS = 2u,    // an index derived from the offsets fell outside its array (access skipped)
};

// bucket(k) = hash(k) mod B, with the remainder computed one of three ways
// that all equal the unsigned '%' (checked by the tests):
//   MODE_POW2    B = 2^j: hash & (B - 1)
//   MODE_FAST32  32-bit hash, B < 2^32: Lemire, Kaser and Kurz, "Faster
//                remainder by direct computation" (2019):
//                M = floor((2^64 - 1) / B) + 1, r = mulhi64(M * h, B)
//   MODE_DIV64   64-bit hash, B not a power of two: hardware-emulated '%'
struct Hasher {
    uint64_t seed;
    uint64_t B;
    uint64_t mask;
    uint64_t magic;
    uint32_t mode;
};
enum : uint32_t { MODE_POW2 = 0, MODE_FAST32 = 1, MODE_DIV64 = 2 };

Hasher make_hasher(uint32_t key_bytes, uint64_t B, uint64_t seed);

// Long-bucket summaries (HG_LONG_SUMMARY): every bucket of more than
// SUM_MIN_LEN keys as its distinct keys (ascending) with their multiplicities.
constexpr uint32_t SUM_MIN_LEN = 8192;        // equals the probe's warp-walk limit
constexpr uint32_t SUM_SLOTS = 64;            // entries per bucket summary
constexpr uint32_t SUM_OVERFLOW = 0xFFFFFFFFu;  // summary length of a bucket with more distinct keys
struct LongSummary {
    const unsigned long long* map = nullptr;  // (l << 32 | bucket), all ones = empty; null: no summaries
    uint32_t map_mask = 0;
    const void* keys = nullptr;     // [cap * SUM_SLOTS]: summary l at l * SUM_SLOTS
    const uint32_t* cnt = nullptr;  // [cap * SUM_SLOTS]
    const uint32_t* len = nullptr;  // [cap]: entries, or SUM_OVERFLOW
};

// Where the build lists the buckets of more than SUM_MIN_LEN keys (null map: not wanted).
struct LongFinder {
    uint32_t* n_long = nullptr;
    uint32_t* bucket = nullptr;          // [cap]
    unsigned long long* map = nullptr;   // bucket -> index, see summary_slot
    uint32_t map_mask = 0;
    uint32_t cap = 0;
};

struct Table {
    uint32_t key_bytes = 4;
    uint32_t has_values = 0;  // values array present (user values or input indices)
    uint32_t flags = 0;
    int device = 0;
    uint64_t n = 0;
    uint64_t B = 0;
    uint64_t seed = 0;
    Hasher H{};
    uint32_t* offsets = nullptr;  // B + 1
    void* keys = nullptr;         // n
    uint32_t* values = nullptr;   // n or null
    uint32_t* err = nullptr;      // device error word
    LongSummary sum{};            // HG_LONG_SUMMARY
    LongFinder finder{};          // set before the build when summaries are wanted
    bool long_noted = false;      // the build listed the long buckets itself
    void* sum_mem = nullptr;
    uint32_t sum_cap = 0;
    const uint32_t* sum_n_long = nullptr;
    const uint32_t* sum_bucket = nullptr;
};

// Sets the message hg_last_error() returns on the calling thread.
void set_error_message(const char* msg);

// Stream-ordered allocation from the device's default memory pool.
cudaError_t dev_alloc(void** p, size_t bytes, cudaStream_t s);
void dev_free(void* p, cudaStream_t s);

// Kernel launch bookkeeping (launch counter and optional per-kernel events).
void launch_begin(const char* name, cudaStream_t s);
void launch_end(const char* name, cudaStream_t s);
int num_sms();

// Build (Algorithm 1): fills t.offsets, t.keys, t.values.  Returns a CUDA error.
cudaError_t build_table(Table& t, const void* d_keys, const void* d_values, cudaStream_t s);
// The partitioned build (Sec. 3.2 binning); requires partition_supported(B).
bool partition_supported(uint64_t B);
cudaError_t build_partitioned(Table& t, const void* d_keys, const void* d_values, cudaStream_t s);

// HG_SORTED_BUCKETS: ascending keys inside every bucket of at most
// sorted_bucket_max(key_bytes) keys (values moved along); run after the build.
uint32_t sorted_bucket_max(uint32_t key_bytes);
cudaError_t sort_buckets(Table& t, cudaStream_t s);

// HG_LONG_SUMMARY: summary_prepare (before the build) allocates t.sum_mem and
// sets t.finder, through which the partitioned build lists the long buckets;
// summary_finish (after it) lists them itself if the build did not, and fills t.sum.
cudaError_t summary_prepare(Table& t, cudaStream_t s);
cudaError_t summary_finish(Table& t, cudaStream_t s);

// Queries grouped by the table's bins (ranges of 8192 buckets), so that a
// bin's offsets and keys stay in L1 while its queries are probed (32-bit
// queries are grouped as their hashes, items.qunhash saying so); the counts,
// produced in grouped order, go back to slot order through reverse passes.
// Chunk c of a partition pass: keys [lo, hi) of segment `seg` (see chunk_range).
struct ChunkMap {
    bool segmented;
    uint64_t n;
    uint32_t P, P2, nseg;
    const uint32_t* bin_start;
    const uint32_t* seg_chunk_start;  // [nseg + 1], segmented only
};
// Work items of the grouped probe: items [0, *huge_chunks) are slices of
// huge_chunk queries of the bins with the most queries (huge bin e owns items
// from huge_chunk_start[e]); the next *n_work items are whole bins, work[i].
struct BinWork {
    const uint32_t* n_huge = nullptr;  // device scalars, written by the grouping
    const uint32_t* huge_chunks = nullptr;
    const uint32_t* n_work = nullptr;
    const uint32_t* huge_bin = nullptr;
    const uint32_t* huge_chunk_start = nullptr;
    const uint32_t* work = nullptr;
    uint32_t huge_chunk = 0;
    // 32-bit grouped queries are held as their hashes (see group_queries): then
    // (1 << 32 | seed), and a probe recovers each query as fmix32_inv(h) ^ seed
    uint64_t qunhash = 0;
};
struct GroupedQueries {
    void* mem = nullptr;
    bool two = false;
    void* q_grouped = nullptr;  // queries in bin order (padded to a multiple of 4 elements)
    const uint32_t* bin_start = nullptr;  // [nbins + 1]: bin p's queries are q_grouped[bin_start[p] ..)
    uint32_t nbins = 0;
    BinWork items{};
    // reverse-pass records (opaque to callers)
    ChunkMap cm_a{}, cm_b{};
    uint32_t nch_a = 0, nch_b_max = 0;
    const void* plan = nullptr;
    const uint32_t* dr_a = nullptr;
    const uint32_t* dr_b = nullptr;
    const uint2* lb_a = nullptr;
    const uint2* lb_b = nullptr;
    uint32_t* err = nullptr;  // error word of the grouping and reverse kernels (null: the table's)
};
bool probe_grouping_pays(const Table& t, uint64_t q);
cudaError_t group_queries(const Table& t, const void* d_q, uint64_t q, GroupedQueries* g, cudaStream_t s);
cudaError_t ungroup_counts(const Table& t, const GroupedQueries* g, const uint32_t* cs, uint32_t* tmp,
                           uint32_t* counts, cudaStream_t s);
void group_release(GroupedQueries* g, cudaStream_t s);

// Buckets per bin of the partitioned build and of the query grouping.
constexpr uint32_t BIN_BUCKETS = 8192;

// Probe entry points.  Return a CUDA error.
//   counts: u32 per slot (may be null); total: u64 sum (may be null).
cudaError_t probe_count(const Table& t, const void* d_q, uint64_t q, uint32_t* counts, uint64_t* total,
                        cudaStream_t s);
// Gather, phase 1: per-slot counts into out_offsets and exclusive scan (out_offsets[q] = total).
// Keeps the long-bucket work list in *ctx for phase 2.
struct GatherCtx {
    void* scratch = nullptr;
    uint64_t slots = 0;
};
cudaError_t gather_offsets(const Table& t, const void* d_q, uint64_t q, uint64_t* out_offsets, GatherCtx* ctx,
                           cudaStream_t s);
cudaError_t gather_values(const Table& t, const void* d_q, uint64_t q, const uint64_t* out_offsets,
                          uint32_t* out_values, GatherCtx* ctx, cudaStream_t s);
void gather_release(GatherCtx* ctx, cudaStream_t s);

// Queries prepared for counting against a table: grouped by the table's bins
// when grouping pays (needs only the table's bucket count, seed and size, not
// its arrays, so it may run while the table is being built), else kept as given.
struct QueryPlan {
    const void* queries = nullptr;
    uint64_t q = 0;
    bool grouped = false;
    GroupedQueries g;
    uint32_t* err = nullptr;  // the plan's own device error word
    uint64_t B = 0, seed = 0, n = 0;  // the table it was made for
    uint32_t key_bytes = 0;
};
cudaError_t plan_queries(const Table& t, const void* d_q, uint64_t q, QueryPlan* p, cudaStream_t s);
cudaError_t count_planned(const Table& t, const QueryPlan& p, uint32_t* counts, uint64_t* total, cudaStream_t s);
void plan_release(QueryPlan* p, cudaStream_t s);

// The paper's query form: HG(Q) built with the table's buckets and seed, then
// bucket-by-bucket intersection with the table; per-slot counts as probe_count.
cudaError_t count_by_intersection(const Table& t, const void* d_q, uint64_t q, uint32_t* counts, uint64_t* total,
                                  cudaStream_t s);

// Byte-model helper behind hg_probe_stats.
cudaError_t probe_stats(const Table& t, const void* d_q, uint64_t q, uint64_t* stats, cudaStream_t s);

// Exclusive scan in place over data[0, n) with decoupled look-back; `err` receives DEVERR_TIMEOUT.
cudaError_t scan_exclusive_u32(uint32_t* data, uint64_t n, uint32_t* err, cudaStream_t s);
cudaError_t scan_exclusive_u64(uint64_t* data, uint64_t n, uint32_t* err, cudaStream_t s);

// Runs one scan tile whose predecessor never publishes: its bounded wait runs
// out (about a second) and records DEVERR_TIMEOUT in *err.
cudaError_t scan_wait_limit_selftest(uint32_t* err, cudaStream_t s);

// The same scan with caller-provided scratch (16-byte aligned, at least
// scan_u32_scratch_bytes(data, n) bytes); allocates nothing.
size_t scan_u32_scratch_bytes(const uint32_t* data, uint64_t n);
cudaError_t scan_exclusive_u32_into(uint32_t* data, uint64_t n, void* scratch, size_t scratch_bytes, uint32_t* err,
                                    cudaStream_t s);

// Direct Algorithm 1 build into caller-provided CSR arrays, scan scratch supplied
// by the caller; allocates nothing.  vals may be null; index_values stores input
// positions as values (vals_out required then).
cudaError_t build_direct_into(const Hasher& H, uint32_t key_bytes, const void* keys, const uint32_t* vals,
                              bool index_values, uint64_t n, uint64_t B, uint32_t* offsets, void* keys_out,
                              uint32_t* vals_out, void* scan_scratch, size_t scan_scratch_bytes, uint32_t* err,
                              cudaStream_t s);

}  // namespace hg
