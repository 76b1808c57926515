/*
 * HashGraph CPU oracle -- TEST INFRASTRUCTURE, NOT PART OF THE PRODUCT.
 *
 * A plain, single-threaded, obviously correct restatement of what the
 * HashGraph build and probe compute (Green et al.'s CSR hash table as used in
 * "Scalable Hash Table for NUMA Systems", the multi-GPU HashGraph: Sec. 3.1
 * and Algorithm 1; querying in Sec. 3.3).
 * Only the test suite, the smoke check and the benchmark's CPU-baseline leg
 * may load this code.  It shares nothing with the CUDA path: its own hash,
 * its own loops, no headers in common.
 *
 * Readings of the paper that this file fixes (each also stated at the
 * function it affects):
 *   - hash(e) is the MurmurHash3 finaliser of (key XOR seed): fmix32 for
 *     32-bit keys, fmix64 for 64-bit keys (the paper names "Murmur" only).
 *   - the bucket of a key is hash mod V by unsigned integer remainder
 *     (Algorithm 1, first loop), 64-bit for 64-bit keys.
 *   - PrefixSum in Algorithm 1 is exclusive and offset has V + 1 entries with
 *     offset[V] = N (Sec. 3.1: offset[i] points at the first key of hash i).
 *   - inside a bucket the oracle keeps input order (its scatter is a
 *     sequential loop); the paper's atomics leave that order free.
 *   - a query slot's count is the number of input keys equal to it
 *     (Sec. 5.4, query performance counts every occurrence).
 *
 * Parity pins: none of these functions is trusted on its own; the
 * "not gpu" tests check them against published MurmurHash3 vectors, brute
 * force, sorting and the CSR invariants.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* MurmurHash3 32-bit finaliser (Appleby's MurmurHash3, fmix32). */
uint32_t hgo_fmix32(uint32_t h) {
    h ^= h >> 16;
    h *= 0x85ebca6bu;
    h ^= h >> 13;
    h *= 0xc2b2ae35u;
    h ^= h >> 16;
    return h;
}

/* MurmurHash3 64-bit finaliser (fmix64). */
uint64_t hgo_fmix64(uint64_t k) {
    k ^= k >> 33;
    k *= 0xff51afd7ed558ccdULL;
    k ^= k >> 33;
    k *= 0xc4ceb9fe1a85ec53ULL;
    k ^= k >> 33;
    return k;
}

/* hash(e) mod V for element i of a 4- or 8-byte key array
 * (Sec. 2 hash definition; Algorithm 1, first loop). */
static uint64_t hashed_value(int key_bytes, const void* A, uint64_t i, uint64_t seed, uint64_t V) {
    if (key_bytes == 4) {
        uint32_t e = ((const uint32_t*)A)[i];
        return (uint64_t)hgo_fmix32(e ^ (uint32_t)seed) % V;
    } else {
        uint64_t e = ((const uint64_t*)A)[i];
        return hgo_fmix64(e ^ seed) % V;
    }
}

static int key_equal(int key_bytes, const void* a, uint64_t i, const void* b, uint64_t j) {
    if (key_bytes == 4) return ((const uint32_t*)a)[i] == ((const uint32_t*)b)[j];
    return ((const uint64_t*)a)[i] == ((const uint64_t*)b)[j];
}

static void copy_key(int key_bytes, void* dst, uint64_t j, const void* src, uint64_t i) {
    if (key_bytes == 4) ((uint32_t*)dst)[j] = ((const uint32_t*)src)[i];
    else ((uint64_t*)dst)[j] = ((const uint64_t*)src)[i];
}

/* Bucket of every key: out[i] = hash(A[i]) mod V. */
void hgo_buckets(int key_bytes, const void* A, uint64_t n, uint64_t seed, uint64_t V, uint64_t* out) {
    for (uint64_t i = 0; i < n; ++i) out[i] = hashed_value(key_bytes, A, i, seed, V);
}

/*
 * Algorithm 1 (Single-GPU HashGraph build), run sequentially.
 *   A[0..N)          input keys (key_bytes = 4 or 8)
 *   vals             optional payload per key (may be NULL)
 *   index_values     if nonzero and vals is NULL, the payload is the key's
 *                    index in A (Sec. 2: the value "can be the index in the
 *                    original input array")
 *   offset[0..V]     out: CSR offsets, offset[V] = N
 *   keys_out[0..N)   out: keys grouped by hashed value
 *   vals_out[0..N)   out: payloads in the same order (may be NULL)
 * Returns 0, or -1 on bad arguments or allocation failure.
 */
int hgo_build(int key_bytes, const void* A, const uint32_t* vals, int index_values,
              uint64_t N, uint64_t V, uint64_t seed,
              uint64_t* offset, void* keys_out, uint32_t* vals_out) {
    if ((key_bytes != 4 && key_bytes != 8) || V == 0) return -1;
    uint64_t* H_A = (uint64_t*)malloc((N ? N : 1) * sizeof(uint64_t));
    uint64_t* CounterArray = (uint64_t*)malloc(V * sizeof(uint64_t));
    if (!H_A || !CounterArray) { free(H_A); free(CounterArray); return -1; }

    /* loop 1: H_A[i] = hash(A[i]) mod V */
    for (uint64_t i = 0; i < N; ++i) H_A[i] = hashed_value(key_bytes, A, i, seed, V);

    /* loop 2: CounterArray[i] = 0 */
    for (uint64_t i = 0; i < V; ++i) CounterArray[i] = 0;

    /* loop 3: CounterArray[H_A[i]] += 1 */
    for (uint64_t i = 0; i < N; ++i) CounterArray[H_A[i]] += 1;

    /* offset = PrefixSum(CounterArray), exclusive, with offset[V] = N */
    offset[0] = 0;
    for (uint64_t i = 0; i < V; ++i) offset[i + 1] = offset[i] + CounterArray[i];

    /* loop 4: CounterArray[i] = 0 */
    for (uint64_t i = 0; i < V; ++i) CounterArray[i] = 0;

    /* loop 5: pos = CounterArray[H_A[i]]++; keys[pos + offset[H_A[i]]] = A[i] */
    for (uint64_t i = 0; i < N; ++i) {
        uint64_t h = H_A[i];
        uint64_t pos = CounterArray[h]++;
        uint64_t dst = pos + offset[h];
        copy_key(key_bytes, keys_out, dst, A, i);
        if (vals_out) {
            if (vals) vals_out[dst] = vals[i];
            else if (index_values) vals_out[dst] = (uint32_t)i;
        }
    }
    free(H_A);
    free(CounterArray);
    return 0;
}

/*
 * Querying (Sec. 3.3): a query hashes to bucket i, and the keys of that
 * bucket are keys[offset[i]] .. keys[offset[i+1] - 1]; the count of a query
 * slot is the number of those keys equal to it (every occurrence counts).
 * counts[0..Q) is written as 64-bit.
 */
void hgo_query_count(int key_bytes, const uint64_t* offset, const void* keys, uint64_t V, uint64_t seed,
                     const void* queries, uint64_t Q, uint64_t* counts) {
    for (uint64_t s = 0; s < Q; ++s) {
        uint64_t i = hashed_value(key_bytes, queries, s, seed, V);
        uint64_t c = 0;
        for (uint64_t j = offset[i]; j < offset[i + 1]; ++j)
            if (key_equal(key_bytes, keys, j, queries, s)) ++c;
        counts[s] = c;
    }
}

/* Join cardinality: the sum of the per-slot counts. */
uint64_t hgo_join_count(int key_bytes, const uint64_t* offset, const void* keys, uint64_t V, uint64_t seed,
                        const void* queries, uint64_t Q) {
    uint64_t total = 0;
    for (uint64_t s = 0; s < Q; ++s) {
        uint64_t i = hashed_value(key_bytes, queries, s, seed, V);
        for (uint64_t j = offset[i]; j < offset[i + 1]; ++j)
            if (key_equal(key_bytes, keys, j, queries, s)) ++total;
    }
    return total;
}

/*
 * Gather: for each query slot, the payloads of the matching keys in the
 * order the bucket is walked.  out_offsets[0..Q] (64-bit) delimits each
 * slot's segment of out_vals.  If out_vals is NULL or capacity is too small,
 * only out_offsets is written.  Returns the total number of matches.
 */
uint64_t hgo_query_gather(int key_bytes, const uint64_t* offset, const void* keys, const uint32_t* vals,
                          uint64_t V, uint64_t seed, const void* queries, uint64_t Q,
                          uint64_t* out_offsets, uint32_t* out_vals, uint64_t capacity) {
    out_offsets[0] = 0;
    for (uint64_t s = 0; s < Q; ++s) {
        uint64_t i = hashed_value(key_bytes, queries, s, seed, V);
        uint64_t c = 0;
        for (uint64_t j = offset[i]; j < offset[i + 1]; ++j)
            if (key_equal(key_bytes, keys, j, queries, s)) ++c;
        out_offsets[s + 1] = out_offsets[s] + c;
    }
    uint64_t total = out_offsets[Q];
    if (!out_vals || capacity < total) return total;
    for (uint64_t s = 0; s < Q; ++s) {
        uint64_t i = hashed_value(key_bytes, queries, s, seed, V);
        uint64_t w = out_offsets[s];
        for (uint64_t j = offset[i]; j < offset[i + 1]; ++j)
            if (key_equal(key_bytes, keys, j, queries, s)) out_vals[w++] = vals[j];
    }
    return total;
}

/* Definition of a count without any table: #{i : A[i] == q} (linear scan). */
uint64_t hgo_count_linear(int key_bytes, const void* A, uint64_t N, const void* q_ptr) {
    uint64_t c = 0;
    for (uint64_t i = 0; i < N; ++i)
        if (key_equal(key_bytes, A, i, q_ptr, 0)) ++c;
    return c;
}
