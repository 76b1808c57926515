/*
 * hashgraph.h -- C ABI of libhashgraph.so, a single-GPU HashGraph static hash
 * table for sm_103a.
 *
 * The table is the CSR ("bipartite graph") layout of HashGraph (Multi-GPU
 * HashGraph paper, Sec. 3.1): an offset array over the V = num_buckets
 * hashed values and a keys array of length N grouped by hashed value, so the
 * keys that hash to bucket i are keys[offset[i]] .. keys[offset[i+1] - 1].
 * Building it is Algorithm 1 (hash, count per bucket, prefix sum, scatter);
 * a query hashes the probe key and walks its bucket (Sec. 3.3), counting
 * every equal key (duplicates included, Sec. 5.4).
 *
 * Conventions shared by every call:
 *  - Pointers named d_* are CUDA device memory on the calling thread's
 *    current device; h_* are host memory.  Key arrays hold uint32_t
 *    (key_bytes = 4) or uint64_t (key_bytes = 8) elements, naturally aligned;
 *    16-byte aligned arrays take the vectorised load path.
 *  - Every call is ordered on the caller's stream `s` (a cudaStream_t; NULL
 *    is the legacy default stream) and returns without waiting for the GPU,
 *    except where stated.  Input buffers are borrowed: they must stay valid
 *    and unmodified until the stream has passed the call.
 *  - Argument errors are reported synchronously and leave no work queued.
 *    Errors found by kernels (a bounded wait that ran out) are recorded in the
 *    table's device error word and reported by hg_sync().
 *  - No call throws across the ABI; hg_last_error() gives a message for the
 *    calling thread's last non-HG_OK status.
 *  - hash(k) = fmix32(k ^ (uint32_t)seed) for 32-bit keys and
 *    fmix64(k ^ seed) for 64-bit keys (the MurmurHash3 finalisers; the paper
 *    names Murmur, Sec. 4.2); bucket(k) = hash(k) mod num_buckets, the
 *    unsigned remainder (Algorithm 1, first loop).
 */
#ifndef HASHGRAPH_H
#define HASHGRAPH_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Same type as cudaStream_t; declared here so that the header needs no CUDA headers. */
typedef struct CUstream_st* hg_stream_t;

typedef struct hg_table hg_table; /* opaque; owns its device arrays */

typedef enum {
    HG_OK = 0,
    HG_ERR_INVALID_ARG = 1, /* a NULL or out-of-range argument; nothing was queued */
    HG_ERR_OOM = 2,         /* a device allocation failed */
    HG_ERR_CUDA = 3,        /* a CUDA runtime call failed; see hg_last_error() */
    HG_ERR_CAPACITY = 4,    /* hg_query_gather: out_capacity < number of matches */
    HG_ERR_NO_VALUES = 5,   /* hg_query_gather on a table without values */
    HG_ERR_TIMEOUT = 6      /* a kernel's bounded wait ran out (reported by hg_sync) */
} hg_status;

/* hg_config.flags */
#define HG_INDEX_VALUES 0x1u  /* key-only input: store each key's input index as its value (Sec. 2: the
                                 value "can be the index in the original input array") */
#define HG_PLAIN_BUILD 0x2u   /* force the direct Algorithm 1 build (global atomics, no partition pass) */
#define HG_PARTITION_BUILD 0x4u /* force the partitioned build (keys binned by bucket range first, the
                                   "efficient HashGraph" of Sec. 3.2) */
#define HG_SORTED_BUCKETS 0x8u /* after the build, sort the keys (with their values) inside every bucket of at
                                  most 16384 keys (8192 for 64-bit keys), so that counting a key in such a
                                  bucket takes two binary searches instead of a walk whose length grows with
                                  the copies of each key (the duplicate-key regime, Sec. 5.4); offsets and
                                  bucket contents are unchanged, only their order inside a bucket is fixed */
#define HG_LONG_SUMMARY 0x10u /* after the build, condense every bucket of more than 8192 keys into its
                                 distinct keys and their multiplicities (at most 64, ascending by key);
                                 hg_query_count and hg_join_count then answer a query on such a bucket by a
                                 binary search of that list instead of a walk over all its copies (the
                                 duplicate-key regime, Sec. 5.4).  A bucket with more distinct keys keeps no
                                 list and is walked as before.  Extra device memory: at most n / 14 bytes
                                 (u32 keys) or n / 10 bytes (u64 keys) */

typedef struct {
    uint32_t key_bytes;   /* 4 or 8 */
    uint32_t value_bytes; /* 0 (keys only) or 4 (uint32_t values) */
    uint64_t num_buckets; /* V in Algorithm 1; 1 <= V <= 2^31 (the paper's 32-bit table size, Sec. 4.3) */
    uint64_t seed;        /* hash seed, XORed into the key before the finaliser */
    uint32_t flags;       /* HG_* flags above */
} hg_config;

/* Message for the calling thread's most recent failing call ("" if none). Never NULL. */
const char* hg_last_error(void);

/* Library version string. */
const char* hg_version(void);

/*
 * hg_build -- Algorithm 1: hash every key, count keys per bucket, exclusive
 * prefix sum of the counts into offset[0..V] (offset[V] = n), scatter keys
 * (and values) into their buckets' ranges.
 *   cfg       table parameters (read during the call only)
 *   d_keys    n keys of cfg->key_bytes each (may be NULL when n == 0)
 *   d_values  n uint32_t values when cfg->value_bytes == 4, else NULL
 *   n         number of keys, 0 <= n < 2^32 (offsets are 32-bit)
 *   out       receives the new table; the table owns offsets (V+1 uint32_t),
 *             keys (n) and values (n, if any), allocated stream-ordered on s
 * The order of keys inside one bucket is unspecified.  Any key value is
 * legal (no sentinel).  On error *out is NULL and nothing stays allocated.
 */
hg_status hg_build(const hg_config* cfg, const void* d_keys, const void* d_values, uint64_t n,
                   hg_stream_t s, hg_table** out);

/*
 * hg_query_count -- for each query slot i, d_counts[i] = number of table keys
 * equal to d_queries[i] (bucket walk, Sec. 3.3; duplicates counted, Sec. 5.4).
 *   d_queries  q keys of the table's key width
 *   d_counts   q uint32_t outputs (may be NULL if d_total is given)
 *   d_total    optional single uint64_t: receives the sum of the counts (the
 *              join cardinality); may be NULL
 * Requires q < 2^32.
 */
hg_status hg_query_count(const hg_table* t, const void* d_queries, uint64_t q, uint32_t* d_counts,
                         uint64_t* d_total, hg_stream_t s);

/*
 * hg_query_gather -- values of every matching key, grouped per query slot.
 *   d_out_offsets  q+1 uint64_t: d_out_offsets[i] .. d_out_offsets[i+1] is slot
 *                  i's segment of d_out_values; d_out_offsets[q] = total
 *   d_out_values   out_capacity uint32_t slots (may be NULL if out_capacity == 0)
 *   h_total        host pointer, receives the total number of matches
 * Two-call pattern: this call synchronises `s` to read the total; if
 * out_capacity < total it returns HG_ERR_CAPACITY with *h_total and
 * d_out_offsets filled and d_out_values untouched.  Order inside a segment
 * is unspecified.  A table built without values and without HG_INDEX_VALUES
 * returns HG_ERR_NO_VALUES.
 */
hg_status hg_query_gather(const hg_table* t, const void* d_queries, uint64_t q, uint64_t* d_out_offsets,
                          uint32_t* d_out_values, uint64_t out_capacity, uint64_t* h_total, hg_stream_t s);

/*
 * Query plans: hg_query_count split in two, so that preparing the queries can
 * overlap the table's build.  hg_query_plan_create reads d_queries and only
 * the table's bucket count, seed and size (not its arrays, which may still be
 * being built on another stream) and groups the queries by the table's bins
 * when that pays (large query sets against tables larger than L2), else keeps
 * the pointer.  hg_query_count_plan then writes the same counts and total as
 * hg_query_count; order it after both the build and the plan creation (for
 * example with cudaStreamWaitEvent).  d_queries must stay valid until the
 * count has completed.  hg_query_plan_free is stream-ordered on `s`.
 */
typedef struct hg_query_plan hg_query_plan; /* opaque; owns the grouped queries and scratch */
hg_status hg_query_plan_create(const hg_table* t, const void* d_queries, uint64_t q, hg_stream_t s,
                               hg_query_plan** out);
hg_status hg_query_count_plan(const hg_table* t, const hg_query_plan* p, uint32_t* d_counts, uint64_t* d_total,
                              hg_stream_t s);
hg_status hg_query_plan_free(hg_query_plan* p, hg_stream_t s);

/*
 * hg_query_count_intersect -- the same per-slot counts (and total) as
 * hg_query_count, computed by the paper's query form (Sec. 3.3): build
 * HG(Q), a HashGraph of the queries with the table's num_buckets and seed
 * whose values are the query slots, intersect bucket i of the table with
 * bucket i of HG(Q) for every i (each query of HG(Q), taken in bucket order,
 * walks its bucket of the table), and write each count to its slot.  q < 2^32.
 * Allocates HG(Q) and its scratch on `s` and frees them before returning.
 */
hg_status hg_query_count_intersect(const hg_table* t, const void* d_queries, uint64_t q, uint32_t* d_counts,
                                   uint64_t* d_total, hg_stream_t s);

/*
 * hg_join_count -- *d_total = sum over query slots of their counts, i.e. the
 * inner-join cardinality of the table's keys with the queries.  d_total is one
 * device uint64_t, overwritten (not accumulated).
 */
hg_status hg_join_count(const hg_table* t, const void* d_queries, uint64_t q, uint64_t* d_total,
                        hg_stream_t s);

/* Stream-ordered release of the table's arrays; the host struct is freed at once. NULL is OK. */
hg_status hg_free(hg_table* t, hg_stream_t s);

/*
 * hg_sync -- wait for `s`, then read and clear the table's device error word.
 * Returns HG_ERR_TIMEOUT if a kernel gave up a bounded wait since the last
 * hg_sync, HG_ERR_CUDA on an asynchronous CUDA error or when a kernel found
 * offsets inconsistent with the keys (the affected writes are skipped, never
 * made out of bounds), else HG_OK.
 */
hg_status hg_sync(const hg_table* t, hg_stream_t s);

/*
 * hg_table_view -- borrow the table's device arrays (valid until hg_free):
 * offsets (uint32_t[V+1]), keys (n elements), values (uint32_t[n] or NULL).
 * Any output pointer may be NULL.
 */
hg_status hg_table_view(const hg_table* t, const void** d_offsets, const void** d_keys,
                        const void** d_values, uint64_t* n, uint64_t* num_buckets);

/*
 * hg_long_summary_view -- borrow a HG_LONG_SUMMARY table's bucket summaries
 * (valid until hg_free; all device arrays, filled once the build's stream
 * has reached the end of hg_build):
 *   d_n_long   uint32_t[1]: number of summarised buckets L (buckets of more
 *              than 8192 keys; L <= *cap)
 *   d_bucket   uint32_t[*cap]: bucket id of summary l, for l < L (any order)
 *   d_len      uint32_t[*cap]: entries of summary l, or 0xFFFFFFFF when the
 *              bucket has more than *slots distinct keys (no summary)
 *   d_keys     key_bytes-wide keys, summary l at [l * *slots, l * *slots + len),
 *              strictly ascending
 *   d_counts   uint32_t, the multiplicity of each of those keys in the bucket
 * A table built without HG_LONG_SUMMARY, or with n <= 8192, has *cap = 0 and
 * NULL arrays.  Any output pointer may be NULL.
 */
hg_status hg_long_summary_view(const hg_table* t, const uint32_t** d_n_long, const uint32_t** d_bucket,
                               const uint32_t** d_len, const void** d_keys, const uint32_t** d_counts,
                               uint32_t* cap, uint32_t* slots);

/*
 * hg_probe_stats -- byte-model helper for diagnostics (not part of a query):
 * for the query slots, d_stats[0] = W, the total number of keys their bucket
 * walks visit (sum of offset[b+1] - offset[b] over slots); d_stats[1] = the
 * part of W in buckets longer than the warp-walk limit (walked by the chunked
 * long-bucket kernel); d_stats[2] = the number of such slots; d_stats[3] =
 * that limit; d_stats[4] = the 32-byte sectors the walks of the other slots
 * touch in the key array; d_stats[5] = the 32-byte sectors of their offset
 * pairs (offset[b], offset[b+1]).  d_stats: 6 device uint64_t, overwritten.
 */
hg_status hg_probe_stats(const hg_table* t, const void* d_queries, uint64_t q, uint64_t* d_stats, hg_stream_t s);

/*
 * hg_build_noalloc -- the direct build (hg_build with HG_PLAIN_BUILD) for
 * callers that cannot allocate device memory.  The paper has no counterpart;
 * this is a deployment convenience.  Some callers run inside a framework that
 * owns all device memory (an inference or serving engine with a fixed memory
 * plan, a plugin that may only use the buffers its host gives it), or must not
 * allocate once running (a real-time loop, where growing a memory pool
 * stalls).  They pass every input and output buffer themselves:
 *   cfg            as for hg_build; only the HG_INDEX_VALUES flag is accepted
 *   d_keys, d_values, n   as for hg_build
 *   d_offsets      out: num_buckets + 1 uint32_t (CSR offsets, d_offsets[V] = n)
 *   d_keys_out     out: n keys grouped by bucket
 *   d_values_out   out: n uint32_t values, required when the table has values
 *                  (value_bytes = 4 or HG_INDEX_VALUES), else NULL
 * The prefix sum's scratch comes from a fixed 64 KiB array inside the library
 * (held on every GPU that loads it until the process exits), which limits
 * num_buckets to 2^23 - 1; larger values return HG_ERR_INVALID_ARG.  Nothing
 * is allocated: no cudaMalloc, cudaMallocAsync or cudaFree is called.
 * The first call on a device looks up the array's device address (with that
 * device current); make that first call before any stream capture.  All calls
 * share the array: calls whose GPU work overlaps (other streams or threads)
 * race on it, so order them on one stream.  Device-side errors are not
 * returned as a status (there is no table to hold an error word): a kernel
 * that gives up a bounded wait leaves d_offsets[V] != n, so a caller checks
 * d_offsets[V] == n after the stream syncs.  The looked-up address is kept for
 * the life of the process, which assumes the device's primary context is not
 * reset (cudaDeviceReset) while the library is loaded.  Asynchronous, like
 * hg_build.
 */
hg_status hg_build_noalloc(const hg_config* cfg, const void* d_keys, const void* d_values, uint64_t n,
                           uint32_t* d_offsets, void* d_keys_out, uint32_t* d_values_out, hg_stream_t s);

/*
 * Batches: many independent tables of 32-bit keys, built and probed together
 * in one persistent kernel launch (captured once in a CUDA graph and
 * replayed).  Each table t is an ordinary HashGraph: its keys are
 * d_keys[key_offsets[t] .. key_offsets[t+1]), its bucket count num_buckets[t],
 * its queries d_queries[query_offsets[t] .. query_offsets[t+1]), and
 * count[i] = the multiplicity of query i among table t's keys (Sec. 3.3,
 * duplicates included).  The hash and seed are those of hg_build.  One CTA
 * builds and probes a table at a time: a table with at most 2^bin_shift
 * buckets and fuse_keys keys entirely in shared memory (histogram, scan and
 * scatter fused); a larger one after partitioning its keys and queries by
 * bin (bucket >> bin_shift, the binning of Sec. 3.2).  The per-table offsets
 * equal hg_build's; the order of keys inside a bucket is unspecified.
 */
typedef struct hg_batch hg_batch; /* opaque; owns the tables' CSR arrays and scratch */

typedef struct {
    uint32_t threads;   /* threads per CTA: 256 or 512 */
    uint32_t bin_shift; /* log2 of buckets per bin: 12 or 13 */
    uint32_t fuse_keys; /* tables with at most this many keys (and 2^bin_shift buckets) take the fused path */
} hg_batch_params;

/*
 * hg_batch_create -- plan a batch and allocate its device arrays.
 *   cfg            key_bytes = 4, value_bytes = 0, seed; num_buckets and flags are ignored
 *   n_tables       >= 1
 *   h_key_offsets  host, n_tables + 1 nondecreasing uint64_t from 0: table t's keys
 *   h_num_buckets  host, n_tables values in [1, 2^21]
 *   h_query_offsets host, n_tables + 1 nondecreasing uint64_t from 0, or NULL (no queries)
 * Each table holds fewer than 2^32 keys and queries.  Copies the host arrays
 * (synchronises `s` once).  Default parameters: 512 threads, bin_shift 13,
 * fuse_keys 16384.
 */
hg_status hg_batch_create(const hg_config* cfg, uint32_t n_tables, const uint64_t* h_key_offsets,
                          const uint64_t* h_num_buckets, const uint64_t* h_query_offsets, hg_stream_t s,
                          hg_batch** out);

/*
 * hg_batch_run -- build every table from d_keys (concatenated as planned) and
 * write d_counts[i] for every query of d_queries; one kernel launch.  The
 * first run with given pointers and parameters captures a CUDA graph on `s`
 * (unless `s` is the legacy default stream or is being captured by the
 * caller, in which case the kernel is launched directly); later runs with the
 * same pointers replay it.  The tables stay readable through hg_batch_view
 * until the next run or hg_batch_free.
 */
hg_status hg_batch_run(hg_batch* b, const uint32_t* d_keys, const uint32_t* d_queries, uint32_t* d_counts,
                       hg_stream_t s);

/*
 * hg_batch_tune -- autotuner: run the batch once per candidate parameter set
 * (threads 256/512, bin_shift 12/13, fuse_keys 2^bin_shift or half of it),
 * time each with CUDA events on `s`, keep the fastest (also returned in
 * *chosen if not NULL).  Synchronises `s`; the outputs hold the last run's.
 */
hg_status hg_batch_tune(hg_batch* b, const uint32_t* d_keys, const uint32_t* d_queries, uint32_t* d_counts,
                        hg_stream_t s, hg_batch_params* chosen);
hg_status hg_batch_set_params(hg_batch* b, const hg_batch_params* p);
hg_status hg_batch_get_params(const hg_batch* b, hg_batch_params* p);

/* Borrow table t's CSR arrays: d_offsets (num_buckets + 1 uint32_t, relative to the table) and d_keys. */
hg_status hg_batch_view(const hg_batch* b, uint32_t table, const void** d_offsets, const void** d_keys, uint64_t* n,
                        uint64_t* num_buckets);
/* Wait for `s`; HG_ERR_CUDA if a batch kernel recorded an out-of-range index. */
hg_status hg_batch_sync(const hg_batch* b, hg_stream_t s);
/*
 * Byte-model helper (diagnostics, not part of a run): d_stats[0] = the sum over
 * every query of its bucket's length in the built tables (the keys its walk
 * visits).  d_stats: 1 device uint64_t, overwritten.  Call after hg_batch_run.
 */
hg_status hg_batch_walk_stats(const hg_batch* b, const uint32_t* d_queries, uint64_t* d_stats, hg_stream_t s);
/* Stream-ordered free of every array the batch owns; NULL is accepted. */
hg_status hg_batch_free(hg_batch* b, hg_stream_t s);

/*
 * Serving: an engine that keeps tables of 32-bit keys resident under a
 * device-memory budget and answers build and probe requests as they arrive
 * (continuous batching).  The engine owns two streams (builds, probes).
 * Residency is decided in arrival order: submitting a build makes its table
 * resident (table bytes = hg_server_table_bytes(n, num_buckets)) and evicts
 * the least recently used tables (a submitted probe marks its table used)
 * until the resident bytes fit the budget; an evicted table's memory is
 * released once the probes already queued for it have finished, and builds
 * start in arrival order once the device holds room.  hg_server_poll()
 * retires finished work, starts builds, and answers all queued probes whose
 * tables exist with one coalesced launch (up to max_batch probes, over many
 * tables; at most two such launches in flight), then reports completed
 * requests.  A probe's counts equal hg_query_count's on the same table.
 * Request buffers (keys, queries, counts) are borrowed until the request is
 * reported complete.  Build scratch is transient and not counted in the
 * budget.  Not thread-safe: call from one host thread.
 */
typedef struct hg_server hg_server;
typedef struct {
    uint64_t builds, probes, probe_launches, evictions; /* since creation */
    uint64_t resident_tables, resident_bytes;           /* after the last poll */
    uint64_t held_bytes;                                /* resident + evicted tables not yet released */
    uint64_t pending, running;                          /* requests queued / launches in flight */
} hg_server_stats_t;

/* budget_bytes > 0; max_batch in [1, 256] probes per coalesced launch. */
hg_status hg_server_create(uint64_t budget_bytes, uint32_t max_batch, hg_server** out);
/* cfg: key_bytes 4, value_bytes 0, flags 0, 1 <= num_buckets <= 2^31.  table_id must not be in use.
   HG_ERR_OOM if the table alone exceeds the budget.  *req_id identifies the request in hg_server_poll. */
hg_status hg_server_submit_build(hg_server* s, uint64_t table_id, const hg_config* cfg, const void* d_keys,
                                 uint64_t n, uint64_t* req_id);
/* The table must be resident (built or queued, not evicted); d_counts: q uint32_t, written on completion. */
hg_status hg_server_submit_probe(hg_server* s, uint64_t table_id, const void* d_queries, uint64_t q,
                                 uint32_t* d_counts, uint64_t* req_id);
/* Drive the engine; report up to max_done completed requests (ids and statuses; HG_OK on success). */
hg_status hg_server_poll(hg_server* s, uint64_t* done_ids, int32_t* done_status, uint32_t max_done,
                         uint32_t* n_done);
hg_status hg_server_stats(const hg_server* s, hg_server_stats_t* out);
/* Borrow a resident, dispatched table (for checks); valid until it is evicted and released. */
hg_status hg_server_table(const hg_server* s, uint64_t table_id, hg_table** out);
/* Device bytes the engine charges for a table of n keys and num_buckets buckets. */
uint64_t hg_server_table_bytes(uint64_t n, uint64_t num_buckets);
/* Wait for all work and free every table, stream and buffer of the engine; NULL is accepted. */
hg_status hg_server_free(hg_server* s);

/*
 * hg_selftest_bounded_wait -- checks the failure path of the kernels' bounded
 * waits without faulting or hanging the GPU: one prefix-sum tile runs while its
 * predecessor never does, so its look-back wait for a flag that nothing sets
 * runs out after about a second and records a timeout.  Synchronises `s`.
 * Returns HG_ERR_TIMEOUT when the wait ran out and was reported (the expected
 * outcome); the context stays usable.
 */
hg_status hg_selftest_bounded_wait(hg_stream_t s);

/*
 * hg_debug_fail_alloc_after -- test hook, host-side fault injection: with
 * n >= 0 the library's device allocations after the next n fail as if the
 * device were out of memory (the calls return HG_ERR_OOM after releasing what
 * they had allocated, and launch nothing on the missing memory); n < 0 turns
 * the injection off.  Process-wide; for tests, not for concurrent use.
 */
void hg_debug_fail_alloc_after(int64_t n);

/* Number of kernels this process has launched through the library so far. */
uint64_t hg_launch_count(void);

/*
 * Per-kernel timing for diagnostics.  While enabled, every kernel the library
 * launches is bracketed by CUDA events on its launching stream.
 * hg_prof_enable(1) also clears the records.  hg_prof_read() synchronises the
 * recorded events and returns, for the kernel named `name` (e.g. "probe"),
 * its launch count and total milliseconds; unknown names give 0 launches.
 * hg_prof_names() returns a comma-separated list of the known kernel names.
 */
hg_status hg_prof_enable(int on);
hg_status hg_prof_read(const char* name, uint64_t* launches, double* total_ms);
const char* hg_prof_names(void);

#ifdef __cplusplus
}
#endif

#endif /* HASHGRAPH_H */
