// Serving: a request engine that keeps HashGraph tables resident on the GPU
// under a device-memory budget and answers build and probe requests as they
// arrive (continuous batching).
//
//  * Residency is decided in arrival order: a build's arrival makes its table
//    resident and, if the budget would be exceeded, evicts the least recently
//    used tables (a probe's arrival marks its table used).  An evicted table's
//    memory is released as soon as the probes that were already queued for it
//    have finished.  Builds run on a build stream, in arrival order, as soon
//    as the device holds room for the new table.
//  * Every probe queued when the probe stream has a free slot is answered by
//    one coalesced launch over all of them (k_probe_multi: one kernel, many
//    (table, queries) pairs), while builds and earlier probe launches are
//    still running, so work from different requests overlaps on the device.
//    A probe whose table is still being built waits for it on the device
//    (stream wait on the build's event), not on the host.
//  * hg_server_poll drives everything: it retires finished launches,
//    dispatches what can start, and reports the requests that completed.
//
// Each probe's counts are exactly those of hg_query_count on the same table
// (the walk of Sec. 3.3, duplicates included); only the launch grouping
// differs.
#include <cstdio>
#include <algorithm>
#include <deque>
#include <list>
#include <new>
#include <unordered_map>
#include <vector>

#include "hg_device.cuh"

namespace hg {
namespace {

constexpr uint32_t MULTI_WALK_LANE = 16;
constexpr int MULTI_THREADS = 256;
constexpr uint32_t SERVE_MAX_BATCH = 256;  // probes per coalesced launch
constexpr int SERVE_PROBE_SLOTS = 2;       // coalesced launches in flight at once

struct ProbeDesc {  // one probe request of a coalesced launch
    const uint32_t* keys;
    const uint32_t* offsets;
    const uint32_t* queries;
    uint32_t* counts;
    Hasher H;
    uint64_t q_begin;  // first global query index of this request
    uint64_t q;
    uint32_t n_keys;
    uint32_t pad;
};

static_assert(sizeof(ProbeDesc) % 8 == 0, "descriptors are copied to shared memory in 8-byte words");

// All queries of all requests as one index space; a warp takes 32 consecutive
// indices, each lane finds its request by binary search over q_begin (the
// descriptors sit in shared memory) and walks its bucket: alone up to
// MULTI_WALK_LANE keys, else with the whole warp.
__global__ void __launch_bounds__(MULTI_THREADS)
k_probe_multi(const ProbeDesc* __restrict__ descs, uint32_t n_desc, uint64_t total) {
    extern __shared__ __align__(16) unsigned char smem[];
    ProbeDesc* s_d = reinterpret_cast<ProbeDesc*>(smem);
    for (uint32_t i = threadIdx.x; i < n_desc * (uint32_t)(sizeof(ProbeDesc) / 8); i += blockDim.x)
        reinterpret_cast<uint64_t*>(s_d)[i] = reinterpret_cast<const uint64_t*>(descs)[i];
    __syncthreads();
    const unsigned lane = lane_id();
    const uint64_t nw = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    for (uint64_t base = (((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5) * 32; base < total;
         base += nw * 32) {
        const uint64_t gi = base + lane;
        const bool ok = gi < total;
        uint32_t r = 0;
        if (ok) {
            uint32_t lo = 0, hi = n_desc;
            while (hi - lo > 1) {
                const uint32_t mid = (lo + hi) >> 1;
                if (s_d[mid].q_begin <= gi) lo = mid; else hi = mid;
            }
            r = lo;
        }
        const ProbeDesc& d = s_d[r];
        uint32_t key = 0, blo = 0, bhi = 0;
        if (ok) {
            key = d.queries[gi - d.q_begin];
            const uint32_t b = bucket_of(key, d.H);
            bhi = min(d.offsets[b + 1], d.n_keys);
            blo = min(d.offsets[b], bhi);
        }
        const uint32_t len = bhi - blo;
        uint32_t cnt = 0;
        if (ok && len <= MULTI_WALK_LANE)
            for (uint32_t x = blo; x < bhi; ++x) cnt += (__ldg(d.keys + x) == key);
        unsigned mm = __ballot_sync(FULL_MASK, ok && len > MULTI_WALK_LANE);
        while (mm) {
            const int src = __ffs(mm) - 1;
            mm &= mm - 1;
            const uint32_t rs = __shfl_sync(FULL_MASK, r, src);
            const uint32_t l = __shfl_sync(FULL_MASK, blo, src);
            const uint32_t h = __shfl_sync(FULL_MASK, bhi, src);
            const uint32_t kk = __shfl_sync(FULL_MASK, key, src);
            const uint32_t* keys = s_d[rs].keys;
            uint32_t c = 0;
            for (uint32_t x = l + lane; x < h; x += 32) c += (__ldg(keys + x) == kk);
            c = __reduce_add_sync(FULL_MASK, c);
            if ((int)lane == src) cnt = c;
        }
        if (ok) d.counts[gi - d.q_begin] = cnt;
    }
}

}  // namespace
}  // namespace hg

using namespace hg;

namespace {

enum ReqKind : int { REQ_BUILD = 0, REQ_PROBE = 1 };

struct SrvTable {
    hg_table* t = nullptr;     // null until the build is dispatched
    uint64_t bytes = 0;
    uint32_t refs = 0;         // probes queued or running against the table
    bool built = false;        // the build's event has been seen complete
    bool evicted = false;      // no longer resident; freed once built and unreferenced
    cudaEvent_t ready = nullptr;
    std::list<uint64_t>::iterator lru;
    const uint32_t* offsets = nullptr;
    const uint32_t* keys = nullptr;
    uint32_t n = 0;
    Hasher H{};
};

struct SrvReq {
    uint64_t id;
    int kind;
    uint64_t table;
    const void* data;
    uint64_t n;
    uint32_t* counts;
    hg_config cfg;
};

struct Launch {
    cudaEvent_t ev = nullptr;
    int kind = REQ_BUILD;
    std::vector<SrvReq> reqs;
    int slot = -1;
};

thread_local char g_smsg[320];

hg_status sfail(hg_status st, const char* msg) {
    set_error_message(msg);
    return st;
}

hg_status scuda(cudaError_t e, const char* what) {
    cudaGetLastError();
    snprintf(g_smsg, sizeof(g_smsg), "%s: %s", what, cudaGetErrorString(e));
    return sfail(e == cudaErrorMemoryAllocation ? HG_ERR_OOM : HG_ERR_CUDA, g_smsg);
}

}  // namespace

struct hg_server {
    int device = 0;
    uint64_t budget = 0;
    uint64_t resident = 0;  // bytes of the resident tables (decided in arrival order)
    uint64_t held = 0;      // bytes allocated on the device (resident + evicted not yet freed)
    uint32_t max_batch = SERVE_MAX_BATCH;
    cudaStream_t build_s = nullptr, probe_s = nullptr;
    std::unordered_map<uint64_t, SrvTable> tables;  // resident and evicted-but-held tables
    std::list<uint64_t> lru;                        // resident tables, least recently used first
    std::deque<SrvReq> pending_builds, pending_probes;
    std::deque<Launch> inflight;
    std::vector<cudaEvent_t> event_pool;
    ProbeDesc* h_desc = nullptr;  // pinned [SERVE_PROBE_SLOTS][SERVE_MAX_BATCH]
    ProbeDesc* d_desc = nullptr;
    bool slot_busy[SERVE_PROBE_SLOTS] = {false, false};
    uint64_t next_id = 1;
    std::deque<std::pair<uint64_t, int>> done;  // (request id, status) not yet reported
    hg_server_stats_t st{};
};

namespace {

cudaEvent_t take_ev(hg_server* s) {
    if (!s->event_pool.empty()) {
        cudaEvent_t e = s->event_pool.back();
        s->event_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreateWithFlags(&e, cudaEventDisableTiming);
    return e;
}

// Frees an evicted table once its build has finished and no probe uses it.
void release_if_idle(hg_server* s, uint64_t id) {
    auto it = s->tables.find(id);
    if (it == s->tables.end()) return;
    SrvTable& t = it->second;
    if (!t.evicted || t.refs || !t.built) return;
    if (t.t) {  // (a build that failed allocated nothing)
        hg_free(t.t, reinterpret_cast<hg_stream_t>(s->build_s));
        s->held -= t.bytes;
    }
    if (t.ready) s->event_pool.push_back(t.ready);
    s->tables.erase(it);
}

void evict(hg_server* s, uint64_t id) {
    SrvTable& t = s->tables[id];
    t.evicted = true;
    s->lru.erase(t.lru);
    s->resident -= t.bytes;
    s->st.evictions++;
    release_if_idle(s, id);
}

// The head build starts once the device holds room for it (evicted tables
// still in use are freed as their probes finish).
bool dispatch_build(hg_server* s, SrvReq& r) {
    SrvTable& tb = s->tables[r.table];
    if (s->held + tb.bytes > s->budget) return false;
    hg_table* t = nullptr;
    hg_status st = hg_build(&r.cfg, r.data, nullptr, r.n, reinterpret_cast<hg_stream_t>(s->build_s), &t);
    if (st != HG_OK) {
        // the table never comes to exist: its probes fail with it
        s->done.push_back({r.id, st});
        tb.t = nullptr;
        tb.built = true;
        if (!tb.evicted) evict(s, r.table);
        return true;
    }
    tb.t = t;
    tb.ready = take_ev(s);
    const void* o = nullptr;
    const void* k = nullptr;
    uint64_t n = 0, B = 0;
    hg_table_view(t, &o, &k, nullptr, &n, &B);
    tb.offsets = static_cast<const uint32_t*>(o);
    tb.keys = static_cast<const uint32_t*>(k);
    tb.n = (uint32_t)n;
    tb.H = make_hasher(4, B, r.cfg.seed);
    cudaEventRecord(tb.ready, s->build_s);
    s->held += tb.bytes;
    Launch L;
    L.ev = take_ev(s);
    cudaEventRecord(L.ev, s->build_s);
    L.kind = REQ_BUILD;
    L.reqs.push_back(r);
    s->inflight.push_back(std::move(L));
    s->st.builds++;
    return true;
}

hg_status dispatch_probes(hg_server* s) {
    while (!s->pending_probes.empty()) {
        int slot = -1;
        for (int i = 0; i < SERVE_PROBE_SLOTS; ++i)
            if (!s->slot_busy[i]) slot = i;
        if (slot < 0) return HG_OK;
        ProbeDesc* hd = s->h_desc + (size_t)slot * SERVE_MAX_BATCH;
        Launch L;
        L.kind = REQ_PROBE;
        L.slot = slot;
        uint64_t total = 0;
        std::vector<uint64_t> waited;
        std::deque<SrvReq> later;  // probes whose table's build has not started yet
        while (!s->pending_probes.empty() && L.reqs.size() < s->max_batch) {
            SrvReq r = s->pending_probes.front();
            s->pending_probes.pop_front();
            SrvTable& t = s->tables[r.table];
            if (!t.t) {
                if (t.built) {  // its build failed
                    t.refs--;
                    s->done.push_back({r.id, HG_ERR_INVALID_ARG});
                    release_if_idle(s, r.table);
                } else {
                    later.push_back(r);
                }
                continue;
            }
            if (!t.built) {
                bool seen = false;
                for (uint64_t w : waited) seen |= (w == r.table);
                if (!seen) {
                    cudaStreamWaitEvent(s->probe_s, t.ready, 0);
                    waited.push_back(r.table);
                }
            }
            ProbeDesc& d = hd[L.reqs.size()];
            d.keys = t.keys;
            d.offsets = t.offsets;
            d.queries = static_cast<const uint32_t*>(r.data);
            d.counts = r.counts;
            d.H = t.H;
            d.q_begin = total;
            d.q = r.n;
            d.n_keys = t.n;
            d.pad = 0;
            total += r.n;
            L.reqs.push_back(r);
        }
        for (auto it = later.rbegin(); it != later.rend(); ++it) s->pending_probes.push_front(*it);
        if (L.reqs.empty()) return HG_OK;
        const uint32_t nd = (uint32_t)L.reqs.size();
        ProbeDesc* dd = s->d_desc + (size_t)slot * SERVE_MAX_BATCH;
        cudaError_t e = cudaMemcpyAsync(dd, hd, sizeof(ProbeDesc) * nd, cudaMemcpyHostToDevice, s->probe_s);
        if (e == cudaSuccess && total) {
            const size_t smem = sizeof(ProbeDesc) * nd;
            int per_sm = 0;
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_probe_multi, MULTI_THREADS, smem);
            if (per_sm < 1) per_sm = 1;
            const uint64_t need_blocks = (total + MULTI_THREADS - 1) / MULTI_THREADS;
            const unsigned g = (unsigned)std::min<uint64_t>(need_blocks, (uint64_t)num_sms() * per_sm);
            launch_begin("probe_multi", s->probe_s);
            k_probe_multi<<<g, MULTI_THREADS, smem, s->probe_s>>>(dd, nd, total);
            launch_end("probe_multi", s->probe_s);
            e = cudaGetLastError();
        }
        if (e != cudaSuccess) return scuda(e, "hg_server_poll (probe launch)");
        L.ev = take_ev(s);
        cudaEventRecord(L.ev, s->probe_s);
        s->slot_busy[slot] = true;
        s->st.probe_launches++;
        s->st.probes += nd;
        s->inflight.push_back(std::move(L));
        if (!later.empty()) return HG_OK;  // the rest waits for builds
    }
    return HG_OK;
}

void retire(hg_server* s) {
    for (auto it = s->inflight.begin(); it != s->inflight.end();) {
        if (cudaEventQuery(it->ev) != cudaSuccess) {
            ++it;
            continue;
        }
        for (SrvReq& r : it->reqs) {
            auto tt = s->tables.find(r.table);
            if (tt != s->tables.end()) {
                if (it->kind == REQ_BUILD) tt->second.built = true;
                else if (tt->second.refs) tt->second.refs--;
            }
            s->done.push_back({r.id, HG_OK});
            release_if_idle(s, r.table);
        }
        if (it->slot >= 0) s->slot_busy[it->slot] = false;
        s->event_pool.push_back(it->ev);
        it = s->inflight.erase(it);
    }
}

void free_server(hg_server* s) {
    if (s->build_s) cudaStreamSynchronize(s->build_s);
    if (s->probe_s) cudaStreamSynchronize(s->probe_s);
    for (auto& kv : s->tables) {
        if (kv.second.t) hg_free(kv.second.t, reinterpret_cast<hg_stream_t>(s->build_s));
        if (kv.second.ready) cudaEventDestroy(kv.second.ready);
    }
    for (Launch& L : s->inflight)
        if (L.ev) cudaEventDestroy(L.ev);
    for (cudaEvent_t e : s->event_pool) cudaEventDestroy(e);
    if (s->build_s) cudaStreamSynchronize(s->build_s);
    if (s->d_desc) cudaFree(s->d_desc);
    if (s->h_desc) cudaFreeHost(s->h_desc);
    if (s->build_s) cudaStreamDestroy(s->build_s);
    if (s->probe_s) cudaStreamDestroy(s->probe_s);
    delete s;
}

}  // namespace

extern "C" {

hg_status hg_server_create(uint64_t budget_bytes, uint32_t max_batch, hg_server** out) {
    if (!out) return sfail(HG_ERR_INVALID_ARG, "hg_server_create: out is NULL");
    *out = nullptr;
    if (budget_bytes == 0) return sfail(HG_ERR_INVALID_ARG, "hg_server_create: budget_bytes is 0");
    if (max_batch == 0 || max_batch > SERVE_MAX_BATCH)
        return sfail(HG_ERR_INVALID_ARG, "hg_server_create: max_batch must be in [1, 256]");
    hg_server* s = new (std::nothrow) hg_server;
    if (!s) return sfail(HG_ERR_OOM, "hg_server_create: host allocation failed");
    cudaGetDevice(&s->device);
    s->budget = budget_bytes;
    s->max_batch = max_batch;
    cudaError_t e = cudaStreamCreateWithFlags(&s->build_s, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s->probe_s, cudaStreamNonBlocking);
    if (e == cudaSuccess)
        e = cudaHostAlloc(reinterpret_cast<void**>(&s->h_desc), sizeof(ProbeDesc) * SERVE_PROBE_SLOTS * SERVE_MAX_BATCH,
                          cudaHostAllocDefault);
    if (e == cudaSuccess)
        e = cudaMalloc(reinterpret_cast<void**>(&s->d_desc), sizeof(ProbeDesc) * SERVE_PROBE_SLOTS * SERVE_MAX_BATCH);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_probe_multi, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)(sizeof(ProbeDesc) * SERVE_MAX_BATCH));
    if (e != cudaSuccess) {
        hg_status r = scuda(e, "hg_server_create");
        free_server(s);
        return r;
    }
    *out = s;
    return HG_OK;
}

hg_status hg_server_submit_build(hg_server* s, uint64_t table_id, const hg_config* cfg, const void* d_keys,
                                 uint64_t n, uint64_t* req_id) {
    if (!s || !cfg || !req_id || (n && !d_keys))
        return sfail(HG_ERR_INVALID_ARG, "hg_server_submit_build: NULL argument");
    if (cfg->key_bytes != 4 || cfg->value_bytes != 0 || cfg->flags != 0 || cfg->num_buckets < 1 ||
        cfg->num_buckets > (1ull << 31) || n > 0xffffffffull)
        return sfail(HG_ERR_INVALID_ARG,
                     "hg_server_submit_build: served tables hold 32-bit keys, no values, 1 <= num_buckets <= 2^31");
    if (s->tables.count(table_id)) return sfail(HG_ERR_INVALID_ARG, "hg_server_submit_build: table id in use");
    const uint64_t need = hg_server_table_bytes(n, cfg->num_buckets);
    if (need > s->budget) return sfail(HG_ERR_OOM, "hg_server_submit_build: the table alone exceeds the budget");
    // residency is decided in arrival order: least recently used tables leave first
    while (s->resident + need > s->budget) evict(s, s->lru.front());
    SrvTable& tb = s->tables[table_id];
    tb.bytes = need;
    s->lru.push_back(table_id);
    tb.lru = std::prev(s->lru.end());
    s->resident += need;
    SrvReq r{};
    r.id = s->next_id++;
    r.kind = REQ_BUILD;
    r.table = table_id;
    r.data = d_keys;
    r.n = n;
    r.cfg = *cfg;
    s->pending_builds.push_back(r);
    *req_id = r.id;
    return HG_OK;
}

hg_status hg_server_submit_probe(hg_server* s, uint64_t table_id, const void* d_queries, uint64_t q,
                                 uint32_t* d_counts, uint64_t* req_id) {
    if (!s || !req_id || (q && (!d_queries || !d_counts)))
        return sfail(HG_ERR_INVALID_ARG, "hg_server_submit_probe: NULL argument");
    if (q > 0xffffffffull) return sfail(HG_ERR_INVALID_ARG, "hg_server_submit_probe: more than 2^32 - 1 queries");
    auto it = s->tables.find(table_id);
    if (it == s->tables.end() || it->second.evicted)
        return sfail(HG_ERR_INVALID_ARG, "hg_server_submit_probe: the table is not resident (never built or evicted)");
    SrvTable& t = it->second;
    t.refs++;  // held until this probe completes
    s->lru.splice(s->lru.end(), s->lru, t.lru);
    SrvReq r{};
    r.id = s->next_id++;
    r.kind = REQ_PROBE;
    r.table = table_id;
    r.data = d_queries;
    r.n = q;
    r.counts = d_counts;
    s->pending_probes.push_back(r);
    *req_id = r.id;
    return HG_OK;
}

hg_status hg_server_poll(hg_server* s, uint64_t* done_ids, int32_t* done_status, uint32_t max_done,
                         uint32_t* n_done) {
    if (!s || !n_done || (max_done && (!done_ids || !done_status)))
        return sfail(HG_ERR_INVALID_ARG, "hg_server_poll: NULL argument");
    *n_done = 0;
    retire(s);
    while (!s->pending_builds.empty() && dispatch_build(s, s->pending_builds.front())) s->pending_builds.pop_front();
    hg_status st = dispatch_probes(s);
    if (st != HG_OK) return st;
    uint32_t k = 0;
    while (k < max_done && !s->done.empty()) {
        done_ids[k] = s->done.front().first;
        done_status[k] = s->done.front().second;
        s->done.pop_front();
        ++k;
    }
    *n_done = k;
    s->st.resident_tables = s->lru.size();
    s->st.resident_bytes = s->resident;
    s->st.held_bytes = s->held;
    s->st.pending = s->pending_builds.size() + s->pending_probes.size();
    s->st.running = s->inflight.size();
    return HG_OK;
}

hg_status hg_server_stats(const hg_server* s, hg_server_stats_t* out) {
    if (!s || !out) return sfail(HG_ERR_INVALID_ARG, "hg_server_stats: NULL argument");
    *out = s->st;
    return HG_OK;
}

hg_status hg_server_table(const hg_server* s, uint64_t table_id, hg_table** out) {
    if (!s || !out) return sfail(HG_ERR_INVALID_ARG, "hg_server_table: NULL argument");
    auto it = s->tables.find(table_id);
    const bool ok = it != s->tables.end() && !it->second.evicted && it->second.t;
    *out = ok ? it->second.t : nullptr;
    return ok ? HG_OK : sfail(HG_ERR_INVALID_ARG, "hg_server_table: not resident or not yet built");
}

uint64_t hg_server_table_bytes(uint64_t n, uint64_t num_buckets) { return 4 * n + 4 * (num_buckets + 1) + 32; }

hg_status hg_server_free(hg_server* s) {
    if (s) free_server(s);
    return HG_OK;
}

}  // extern "C"
