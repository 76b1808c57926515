// C ABI of libhashgraph.so (declared in include/hashgraph.h): argument
// checks, table ownership, stream-ordered allocation, error reporting and the
// launch bookkeeping used for diagnostics.
#include <atomic>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "hg_internal.h"

namespace hg {

namespace {

thread_local std::string g_err;

hg_status fail(hg_status st, const char* fmt, ...) __attribute__((format(printf, 2, 3)));
hg_status fail(hg_status st, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_err = buf;
    return st;
}

hg_status cuda_fail(cudaError_t e, const char* what) {
    if (e == cudaErrorMemoryAllocation) {
        cudaGetLastError();
        return fail(HG_ERR_OOM, "%s: out of device memory", what);
    }
    return fail(HG_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

std::atomic<uint64_t> g_launches{0};

// ---- per-kernel event timing (diagnostics) ----
const char* const kKernelNames[] = {"hist", "scan", "scatter", "probe", "long_prep", "long", "gather",
                                    "long_gather", "walk_stats", "part_hist", "part_plan", "chunk_scan", "chunk_count", "part_scatter", "part_scatter2", "huge_count",
                                    "huge_items", "huge_scan", "bin_build", "bin_small", "bin_big", "q_part_count", "q_partition", "q_partition2", "q_reverse", "batch", "probe_multi", "scatter_counts", "sort_buckets",
                                    "sum_find", "sum_plan", "sum_count", "sum_finish", "probe_hash"};
struct ProfRecord {
    const char* name;
    cudaEvent_t start, stop;
};
std::mutex g_prof_mu;
bool g_prof_on = false;
std::vector<ProfRecord> g_prof_records;
std::vector<cudaEvent_t> g_event_pool;
thread_local cudaEvent_t t_pending_start = nullptr;

cudaEvent_t take_event() {
    if (!g_event_pool.empty()) {
        cudaEvent_t e = g_event_pool.back();
        g_event_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

void prof_clear_locked() {
    for (auto& r : g_prof_records) {
        g_event_pool.push_back(r.start);
        g_event_pool.push_back(r.stop);
    }
    g_prof_records.clear();
}

std::string g_names_csv;

}  // namespace

void set_error_message(const char* msg) { g_err = msg ? msg : ""; }

void launch_begin(const char* name, cudaStream_t s) {
    (void)name;
    if (!g_prof_on) return;
    std::lock_guard<std::mutex> lk(g_prof_mu);
    t_pending_start = take_event();
    cudaEventRecord(t_pending_start, s);
}

void launch_end(const char* name, cudaStream_t s) {
    g_launches.fetch_add(1, std::memory_order_relaxed);
    if (!g_prof_on || !t_pending_start) return;
    std::lock_guard<std::mutex> lk(g_prof_mu);
    cudaEvent_t stop = take_event();
    cudaEventRecord(stop, s);
    g_prof_records.push_back({name, t_pending_start, stop});
    t_pending_start = nullptr;
}

int num_sms() {
    static int cached[64] = {0};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64) dev = 0;
    if (cached[dev] == 0) {
        int v = 0;
        cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
        cached[dev] = v > 0 ? v : 1;
    }
    return cached[dev];
}

// hg_debug_fail_alloc_after: allocations left before injected failures (< 0: off)
std::atomic<int64_t> g_allocs_before_failure{-1};

cudaError_t dev_alloc(void** p, size_t bytes, cudaStream_t s) {
    *p = nullptr;
    for (int64_t k = g_allocs_before_failure.load(); k >= 0;) {
        if (k == 0) return cudaErrorMemoryAllocation;  // injected (host side; nothing runs on the device)
        if (g_allocs_before_failure.compare_exchange_weak(k, k - 1)) break;
    }
    static std::once_flag once[64];
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev >= 0 && dev < 64) {
        // Keep freed blocks in the pool instead of returning them to the driver
        // between calls (affects this process's default pool only).
        std::call_once(once[dev], [dev] {
            cudaMemPool_t pool;
            if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
                uint64_t thr = UINT64_MAX;
                cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
            }
        });
    }
    *p = nullptr;
    if (bytes == 0) bytes = 16;
    return cudaMallocAsync(p, bytes, s);
}

void dev_free(void* p, cudaStream_t s) {
    if (p) cudaFreeAsync(p, s);
}

Hasher make_hasher(uint32_t key_bytes, uint64_t B, uint64_t seed) {
    Hasher H{};
    H.seed = seed;
    H.B = B;
    if ((B & (B - 1)) == 0) {
        H.mode = MODE_POW2;
        H.mask = B - 1;
    } else if (key_bytes == 4) {
        H.mode = MODE_FAST32;
        H.magic = UINT64_MAX / B + 1;
    } else {
        H.mode = MODE_DIV64;
    }
    return H;
}

}  // namespace hg

using namespace hg;

namespace {

bool aligned(const void* p, size_t a) { return (reinterpret_cast<uintptr_t>(p) % a) == 0; }

hg_status check_device(const Table* t) {
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    if (dev != t->device) return fail(HG_ERR_INVALID_ARG, "table lives on device %d, current device is %d", t->device, dev);
    return HG_OK;
}

hg_status check_queries(const Table* t, const void* d_q, uint64_t q) {
    if (q >= (1ull << 32)) return fail(HG_ERR_INVALID_ARG, "q = %llu must be < 2^32", (unsigned long long)q);
    if (q > 0 && !d_q) return fail(HG_ERR_INVALID_ARG, "d_queries is NULL");
    if (q > 0 && !aligned(d_q, t->key_bytes)) return fail(HG_ERR_INVALID_ARG, "d_queries is not %u-byte aligned", t->key_bytes);
    return HG_OK;
}

void free_table(Table* t, cudaStream_t s) {
    dev_free(t->offsets, s);
    dev_free(t->keys, s);
    dev_free(t->values, s);
    dev_free(t->err, s);
    dev_free(t->sum_mem, s);
    delete t;
}

}  // namespace

extern "C" {

const char* hg_last_error(void) { return g_err.c_str(); }

const char* hg_version(void) { return "hashgraph-gb300 0.1 (sm_103a)"; }

hg_status hg_build(const hg_config* cfg, const void* d_keys, const void* d_values, uint64_t n, hg_stream_t s,
                   hg_table** out) {
    if (!out) return fail(HG_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (!cfg) return fail(HG_ERR_INVALID_ARG, "cfg is NULL");
    if (cfg->key_bytes != 4 && cfg->key_bytes != 8)
        return fail(HG_ERR_INVALID_ARG, "key_bytes = %u, must be 4 or 8", cfg->key_bytes);
    if (cfg->value_bytes != 0 && cfg->value_bytes != 4)
        return fail(HG_ERR_INVALID_ARG, "value_bytes = %u, must be 0 or 4", cfg->value_bytes);
    if (cfg->num_buckets < 1 || cfg->num_buckets > (1ull << 31))
        return fail(HG_ERR_INVALID_ARG, "num_buckets = %llu, must be in [1, 2^31]",
                    (unsigned long long)cfg->num_buckets);
    if (n >= (1ull << 32)) return fail(HG_ERR_INVALID_ARG, "n = %llu must be < 2^32", (unsigned long long)n);
    const uint32_t known = HG_INDEX_VALUES | HG_PLAIN_BUILD | HG_PARTITION_BUILD | HG_SORTED_BUCKETS | HG_LONG_SUMMARY;
    if (cfg->flags & ~known) return fail(HG_ERR_INVALID_ARG, "unknown flags 0x%x", cfg->flags & ~known);
    if ((cfg->flags & HG_PLAIN_BUILD) && (cfg->flags & HG_PARTITION_BUILD))
        return fail(HG_ERR_INVALID_ARG, "HG_PLAIN_BUILD and HG_PARTITION_BUILD are exclusive");
    if ((cfg->flags & HG_INDEX_VALUES) && cfg->value_bytes)
        return fail(HG_ERR_INVALID_ARG, "HG_INDEX_VALUES needs value_bytes = 0");
    if (n > 0 && !d_keys) return fail(HG_ERR_INVALID_ARG, "d_keys is NULL");
    if (n > 0 && !aligned(d_keys, cfg->key_bytes))
        return fail(HG_ERR_INVALID_ARG, "d_keys is not %u-byte aligned", cfg->key_bytes);
    if (cfg->value_bytes == 4 && n > 0 && !d_values) return fail(HG_ERR_INVALID_ARG, "d_values is NULL");
    if (cfg->value_bytes == 0 && d_values) return fail(HG_ERR_INVALID_ARG, "d_values given with value_bytes = 0");
    if (d_values && !aligned(d_values, 4)) return fail(HG_ERR_INVALID_ARG, "d_values is not 4-byte aligned");

    cudaStream_t st = reinterpret_cast<cudaStream_t>(s);
    Table* t = new (std::nothrow) Table();
    if (!t) return fail(HG_ERR_OOM, "host allocation failed");
    cudaGetDevice(&t->device);
    t->key_bytes = cfg->key_bytes;
    t->has_values = (cfg->value_bytes == 4 || (cfg->flags & HG_INDEX_VALUES)) ? 1 : 0;
    t->flags = cfg->flags;
    t->n = n;
    t->B = cfg->num_buckets;
    t->seed = cfg->seed;
    t->H = make_hasher(cfg->key_bytes, cfg->num_buckets, cfg->seed);

    // 16 spare bytes after offsets and keys: bulk copies of a bin may round their end up to 16 bytes
    cudaError_t e = dev_alloc(reinterpret_cast<void**>(&t->offsets), (t->B + 1) * sizeof(uint32_t) + 16, st);
    if (e == cudaSuccess) e = dev_alloc(&t->keys, n * t->key_bytes + 16, st);
    if (e == cudaSuccess && t->has_values) e = dev_alloc(reinterpret_cast<void**>(&t->values), n * 4, st);
    if (e == cudaSuccess) e = dev_alloc(reinterpret_cast<void**>(&t->err), sizeof(uint32_t), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(t->err, 0, sizeof(uint32_t), st);
    if (e != cudaSuccess) {
        hg_status r = cuda_fail(e, "hg_build allocation");
        free_table(t, st);
        return r;
    }
    e = (cfg->flags & HG_LONG_SUMMARY) ? summary_prepare(*t, st) : cudaSuccess;
    if (e == cudaSuccess) e = build_table(*t, d_keys, d_values, st);
    if (e == cudaSuccess && (cfg->flags & HG_SORTED_BUCKETS)) e = sort_buckets(*t, st);
    if (e == cudaSuccess && (cfg->flags & HG_LONG_SUMMARY)) e = summary_finish(*t, st);
    if (e != cudaSuccess) {
        hg_status r = cuda_fail(e, "hg_build");
        free_table(t, st);
        return r;
    }
    *out = reinterpret_cast<hg_table*>(t);
    return HG_OK;
}

hg_status hg_query_count(const hg_table* ht, const void* d_queries, uint64_t q, uint32_t* d_counts,
                         uint64_t* d_total, hg_stream_t s) {
    const Table* t = reinterpret_cast<const Table*>(ht);
    if (!t) return fail(HG_ERR_INVALID_ARG, "table is NULL");
    if (!d_counts && !d_total && q > 0) return fail(HG_ERR_INVALID_ARG, "d_counts and d_total are both NULL");
    if (d_counts && q > 0 && !aligned(d_counts, 4)) return fail(HG_ERR_INVALID_ARG, "d_counts is not 4-byte aligned");
    if (d_total && !aligned(d_total, 8)) return fail(HG_ERR_INVALID_ARG, "d_total is not 8-byte aligned");
    hg_status st = check_queries(t, d_queries, q);
    if (st != HG_OK) return st;
    if ((st = check_device(t)) != HG_OK) return st;
    cudaError_t e = probe_count(*t, d_queries, q, d_counts, d_total, reinterpret_cast<cudaStream_t>(s));
    if (e != cudaSuccess) return cuda_fail(e, "hg_query_count");
    return HG_OK;
}

hg_status hg_query_count_intersect(const hg_table* ht, const void* d_queries, uint64_t q, uint32_t* d_counts,
                                   uint64_t* d_total, hg_stream_t s) {
    const Table* t = reinterpret_cast<const Table*>(ht);
    if (!t) return fail(HG_ERR_INVALID_ARG, "table is NULL");
    if (!d_counts && !d_total && q > 0) return fail(HG_ERR_INVALID_ARG, "d_counts and d_total are both NULL");
    if (d_counts && q > 0 && !aligned(d_counts, 4)) return fail(HG_ERR_INVALID_ARG, "d_counts is not 4-byte aligned");
    if (d_total && !aligned(d_total, 8)) return fail(HG_ERR_INVALID_ARG, "d_total is not 8-byte aligned");
    if (q >= (1ull << 32)) return fail(HG_ERR_INVALID_ARG, "q = %llu must be < 2^32", (unsigned long long)q);
    hg_status st = check_queries(t, d_queries, q);
    if (st != HG_OK) return st;
    if ((st = check_device(t)) != HG_OK) return st;
    cudaError_t e = count_by_intersection(*t, d_queries, q, d_counts, d_total, reinterpret_cast<cudaStream_t>(s));
    if (e != cudaSuccess) return cuda_fail(e, "hg_query_count_intersect");
    return HG_OK;
}

hg_status hg_query_plan_create(const hg_table* ht, const void* d_queries, uint64_t q, hg_stream_t s,
                               hg_query_plan** out) {
    const Table* t = reinterpret_cast<const Table*>(ht);
    if (!out) return fail(HG_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (!t) return fail(HG_ERR_INVALID_ARG, "table is NULL");
    hg_status st = check_queries(t, d_queries, q);
    if (st != HG_OK) return st;
    if ((st = check_device(t)) != HG_OK) return st;
    QueryPlan* p = new (std::nothrow) QueryPlan();
    if (!p) return fail(HG_ERR_OOM, "host allocation failed");
    cudaStream_t cs = reinterpret_cast<cudaStream_t>(s);
    cudaError_t e = plan_queries(*t, d_queries, q, p, cs);
    if (e != cudaSuccess) {
        plan_release(p, cs);
        delete p;
        return cuda_fail(e, "hg_query_plan_create");
    }
    *out = reinterpret_cast<hg_query_plan*>(p);
    return HG_OK;
}

hg_status hg_query_count_plan(const hg_table* ht, const hg_query_plan* hp, uint32_t* d_counts, uint64_t* d_total,
                              hg_stream_t s) {
    const Table* t = reinterpret_cast<const Table*>(ht);
    const QueryPlan* p = reinterpret_cast<const QueryPlan*>(hp);
    if (!t || !p) return fail(HG_ERR_INVALID_ARG, "table or plan is NULL");
    if (p->B != t->B || p->seed != t->seed || p->n != t->n || p->key_bytes != t->key_bytes)
        return fail(HG_ERR_INVALID_ARG, "the plan was made for a table of another shape or seed");
    if (!d_counts && !d_total && p->q > 0) return fail(HG_ERR_INVALID_ARG, "d_counts and d_total are both NULL");
    if (d_counts && p->q > 0 && !aligned(d_counts, 4)) return fail(HG_ERR_INVALID_ARG, "d_counts is not 4-byte aligned");
    if (d_total && !aligned(d_total, 8)) return fail(HG_ERR_INVALID_ARG, "d_total is not 8-byte aligned");
    hg_status st = check_device(t);
    if (st != HG_OK) return st;
    cudaError_t e = count_planned(*t, *p, d_counts, d_total, reinterpret_cast<cudaStream_t>(s));
    if (e != cudaSuccess) return cuda_fail(e, "hg_query_count_plan");
    return HG_OK;
}

hg_status hg_query_plan_free(hg_query_plan* hp, hg_stream_t s) {
    QueryPlan* p = reinterpret_cast<QueryPlan*>(hp);
    if (!p) return HG_OK;
    plan_release(p, reinterpret_cast<cudaStream_t>(s));
    delete p;
    return HG_OK;
}

hg_status hg_join_count(const hg_table* ht, const void* d_queries, uint64_t q, uint64_t* d_total, hg_stream_t s) {
    const Table* t = reinterpret_cast<const Table*>(ht);
    if (!t) return fail(HG_ERR_INVALID_ARG, "table is NULL");
    if (!d_total) return fail(HG_ERR_INVALID_ARG, "d_total is NULL");
    if (!aligned(d_total, 8)) return fail(HG_ERR_INVALID_ARG, "d_total is not 8-byte aligned");
    hg_status st = check_queries(t, d_queries, q);
    if (st != HG_OK) return st;
    if ((st = check_device(t)) != HG_OK) return st;
    cudaError_t e = probe_count(*t, d_queries, q, nullptr, d_total, reinterpret_cast<cudaStream_t>(s));
    if (e != cudaSuccess) return cuda_fail(e, "hg_join_count");
    return HG_OK;
}

hg_status hg_query_gather(const hg_table* ht, const void* d_queries, uint64_t q, uint64_t* d_out_offsets,
                          uint32_t* d_out_values, uint64_t out_capacity, uint64_t* h_total, hg_stream_t s) {
    const Table* t = reinterpret_cast<const Table*>(ht);
    if (!t) return fail(HG_ERR_INVALID_ARG, "table is NULL");
    if (!t->has_values) return fail(HG_ERR_NO_VALUES, "table has no values (build with value_bytes = 4 or HG_INDEX_VALUES)");
    if (!d_out_offsets || !h_total) return fail(HG_ERR_INVALID_ARG, "d_out_offsets and h_total are required");
    if (!aligned(d_out_offsets, 8)) return fail(HG_ERR_INVALID_ARG, "d_out_offsets is not 8-byte aligned");
    if (out_capacity > 0 && !d_out_values) return fail(HG_ERR_INVALID_ARG, "d_out_values is NULL");
    if (d_out_values && !aligned(d_out_values, 4)) return fail(HG_ERR_INVALID_ARG, "d_out_values is not 4-byte aligned");
    hg_status st = check_queries(t, d_queries, q);
    if (st != HG_OK) return st;
    if ((st = check_device(t)) != HG_OK) return st;
    cudaStream_t cs = reinterpret_cast<cudaStream_t>(s);
    GatherCtx ctx;
    cudaError_t e = gather_offsets(*t, d_queries, q, d_out_offsets, &ctx, cs);
    uint64_t total = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&total, d_out_offsets + q, sizeof(uint64_t), cudaMemcpyDeviceToHost, cs);
    if (e == cudaSuccess) e = cudaStreamSynchronize(cs);
    if (e != cudaSuccess) {
        gather_release(&ctx, cs);
        return cuda_fail(e, "hg_query_gather");
    }
    *h_total = total;
    if (total > out_capacity) {
        gather_release(&ctx, cs);
        return fail(HG_ERR_CAPACITY, "gather needs %llu value slots, out_capacity is %llu",
                    (unsigned long long)total, (unsigned long long)out_capacity);
    }
    if (total > 0) e = gather_values(*t, d_queries, q, d_out_offsets, d_out_values, &ctx, cs);
    gather_release(&ctx, cs);
    if (e != cudaSuccess) return cuda_fail(e, "hg_query_gather");
    return HG_OK;
}

hg_status hg_free(hg_table* ht, hg_stream_t s) {
    Table* t = reinterpret_cast<Table*>(ht);
    if (!t) return HG_OK;
    free_table(t, reinterpret_cast<cudaStream_t>(s));
    return HG_OK;
}

hg_status hg_sync(const hg_table* ht, hg_stream_t s) {
    const Table* t = reinterpret_cast<const Table*>(ht);
    if (!t) return fail(HG_ERR_INVALID_ARG, "table is NULL");
    cudaStream_t cs = reinterpret_cast<cudaStream_t>(s);
    cudaError_t e = cudaStreamSynchronize(cs);
    uint32_t err = 0;
    if (e == cudaSuccess) e = cudaMemcpy(&err, t->err, sizeof(err), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && err) e = cudaMemset(t->err, 0, sizeof(uint32_t));
    if (e != cudaSuccess) return cuda_fail(e, "hg_sync");
    if (err & DEVERR_TIMEOUT) return fail(HG_ERR_TIMEOUT, "a kernel gave up a bounded wait (error word 0x%x)", err);
    if (err & DEVERR_BOUNDS)
        return fail(HG_ERR_CUDA, "inconsistent offsets: out-of-range positions were skipped (error word 0x%x)", err);
    return HG_OK;
}

hg_status hg_table_view(const hg_table* ht, const void** d_offsets, const void** d_keys, const void** d_values,
                        uint64_t* n, uint64_t* num_buckets) {
    const Table* t = reinterpret_cast<const Table*>(ht);
    if (!t) return fail(HG_ERR_INVALID_ARG, "table is NULL");
    if (d_offsets) *d_offsets = t->offsets;
    if (d_keys) *d_keys = t->keys;
    if (d_values) *d_values = t->values;
    if (n) *n = t->n;
    if (num_buckets) *num_buckets = t->B;
    return HG_OK;
}

hg_status hg_long_summary_view(const hg_table* ht, const uint32_t** d_n_long, const uint32_t** d_bucket,
                               const uint32_t** d_len, const void** d_keys, const uint32_t** d_counts,
                               uint32_t* cap, uint32_t* slots) {
    const Table* t = reinterpret_cast<const Table*>(ht);
    if (!t) return fail(HG_ERR_INVALID_ARG, "table is NULL");
    if (d_n_long) *d_n_long = t->sum_n_long;
    if (d_bucket) *d_bucket = t->sum_bucket;
    if (d_len) *d_len = t->sum.len;
    if (d_keys) *d_keys = t->sum.keys;
    if (d_counts) *d_counts = t->sum.cnt;
    if (cap) *cap = t->sum_cap;
    if (slots) *slots = SUM_SLOTS;
    return HG_OK;
}

void hg_debug_fail_alloc_after(int64_t n) { g_allocs_before_failure.store(n < 0 ? -1 : n); }

hg_status hg_selftest_bounded_wait(hg_stream_t s) {
    cudaStream_t cs = reinterpret_cast<cudaStream_t>(s);
    uint32_t* err = nullptr;
    cudaError_t e = dev_alloc(reinterpret_cast<void**>(&err), sizeof(uint32_t), cs);
    if (e == cudaSuccess) e = cudaMemsetAsync(err, 0, sizeof(uint32_t), cs);
    if (e == cudaSuccess) e = scan_wait_limit_selftest(err, cs);
    uint32_t h = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h, err, sizeof(h), cudaMemcpyDeviceToHost, cs);
    if (err) dev_free(err, cs);
    if (e == cudaSuccess) e = cudaStreamSynchronize(cs);
    if (e != cudaSuccess) return cuda_fail(e, "hg_selftest_bounded_wait");
    if (h & DEVERR_TIMEOUT) return fail(HG_ERR_TIMEOUT, "the look-back wait ran out as intended");
    return fail(HG_ERR_CUDA, "the look-back wait did not report running out");
}

hg_status hg_probe_stats(const hg_table* ht, const void* d_queries, uint64_t q, uint64_t* d_stats, hg_stream_t s) {
    const Table* t = reinterpret_cast<const Table*>(ht);
    if (!t) return fail(HG_ERR_INVALID_ARG, "table is NULL");
    if (!d_stats || !aligned(d_stats, 8)) return fail(HG_ERR_INVALID_ARG, "d_stats must be 8-byte aligned device memory");
    hg_status st = check_queries(t, d_queries, q);
    if (st != HG_OK) return st;
    if ((st = check_device(t)) != HG_OK) return st;
    cudaError_t e = probe_stats(*t, d_queries, q, d_stats, reinterpret_cast<cudaStream_t>(s));
    if (e != cudaSuccess) return cuda_fail(e, "hg_probe_stats");
    return HG_OK;
}

uint64_t hg_launch_count(void) { return g_launches.load(std::memory_order_relaxed); }

hg_status hg_prof_enable(int on) {
    std::lock_guard<std::mutex> lk(g_prof_mu);
    if (on) prof_clear_locked();
    g_prof_on = on != 0;
    return HG_OK;
}

hg_status hg_prof_read(const char* name, uint64_t* launches, double* total_ms) {
    if (!name || !launches || !total_ms) return fail(HG_ERR_INVALID_ARG, "NULL argument");
    std::lock_guard<std::mutex> lk(g_prof_mu);
    uint64_t cnt = 0;
    double ms = 0.0;
    for (auto& r : g_prof_records) {
        if (std::strcmp(r.name, name) != 0) continue;
        cudaError_t e = cudaEventSynchronize(r.stop);
        if (e != cudaSuccess) return cuda_fail(e, "hg_prof_read");
        float f = 0.f;
        e = cudaEventElapsedTime(&f, r.start, r.stop);
        if (e != cudaSuccess) return cuda_fail(e, "hg_prof_read");
        ms += f;
        ++cnt;
    }
    *launches = cnt;
    *total_ms = ms;
    return HG_OK;
}

const char* hg_prof_names(void) {
    std::lock_guard<std::mutex> lk(g_prof_mu);
    if (g_names_csv.empty()) {
        for (const char* nm : kKernelNames) {
            if (!g_names_csv.empty()) g_names_csv += ",";
            g_names_csv += nm;
        }
    }
    return g_names_csv.c_str();
}

}  // extern "C"
