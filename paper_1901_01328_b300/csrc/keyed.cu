// A6 Keyed reduction: per-key count and sum of a nonresident value column
// over a KPA sorted by key.
//
// A key's rows are one contiguous run, so its count and sum are differences
// of prefix quantities at run boundaries (heads):
//     count(run) = next head row - head row
//     sum(run)   = P(next head) - P(head),  P(i) = sum of v over rows < i,
// exactly, modulo 2^64.  The kernel therefore needs only a plain prefix sum
// of the gathered values plus the position of the last head, never a
// segmented reduction.  Tiles of 4096 rows arrive by bulk copy (TMA), two in
// flight per CTA; tiles chain their running totals with a decoupled
// look-back (bounded wait); a head writes its key, and the previous run's
// count and sum, at output index = number of heads before it.
#include "common.cuh"

namespace sbh {
namespace {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr int kIpt = 16;
constexpr int kTile = kThreads * kIpt;
constexpr uint64_t kNoRow = ~0ull;

// Running totals over a range of rows.  last_p is the sum of the values from
// the start of the range up to (not including) its last head.
struct Agg {
    uint64_t heads, last_row, sum, last_p;
};

__device__ __forceinline__ Agg agg_identity() { return {0ull, kNoRow, 0ull, 0ull}; }

__device__ __forceinline__ Agg agg_combine(const Agg& a, const Agg& b) {
    Agg r;
    r.heads = a.heads + b.heads;
    r.sum = a.sum + b.sum;
    if (b.heads) {
        r.last_row = b.last_row;
        r.last_p = a.sum + b.last_p;
    } else {
        r.last_row = a.last_row;
        r.last_p = a.last_p;
    }
    return r;
}

struct TileRec {
    Agg agg;
    Agg prefix;
};
constexpr uint32_t kRecAgg = 1, kRecPrefix = 2;

__device__ __forceinline__ void store_agg(Agg* dst, const Agg& v) {
    volatile uint64_t* d = reinterpret_cast<volatile uint64_t*>(dst);
    d[0] = v.heads;
    d[1] = v.last_row;
    d[2] = v.sum;
    d[3] = v.last_p;
}
__device__ __forceinline__ Agg load_agg(const Agg* src) {
    const volatile uint64_t* s = reinterpret_cast<const volatile uint64_t*>(src);
    return {s[0], s[1], s[2], s[3]};
}

struct KeyedSmem {
    uint64_t keys[2][kTile];
    uint32_t ptrs[2][kTile];
    Agg warp_agg[kWarps];
    Agg warp_prefix[kWarps];
    uint32_t tile_of[2];
    uint64_t mbar[2];
};

__device__ __forceinline__ uint64_t shfl_u64(uint64_t v, int src) { return __shfl_sync(0xffffffffu, v, src); }
__device__ __forceinline__ uint64_t shfl_up_u64(uint64_t v, int o) { return __shfl_up_sync(0xffffffffu, v, o); }

// kVals: 0 = count only (ptrs and values are not read); 4 or 8 = value bytes.
template <int kVals>
__global__ void __launch_bounds__(kThreads, 2)
keyed_kernel(const uint64_t* __restrict__ keys, const uint32_t* __restrict__ ptrs, uint32_t n,
             const void* __restrict__ val_col, uint64_t* __restrict__ out_keys, uint64_t* __restrict__ out_counts,
             uint64_t* __restrict__ out_sums, uint64_t cap, uint64_t* __restrict__ nkeys_out,
             uint32_t* __restrict__ flags, TileRec* __restrict__ recs, uint32_t* __restrict__ tile_counter,
             uint32_t spin_limit, uint32_t* __restrict__ status, int bulk_ok) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    KeyedSmem& sm = *reinterpret_cast<KeyedSmem*>(smem_raw);
    const uint32_t tid = threadIdx.x, lane = lane_id(), warp = tid / 32;
    const uint32_t ntiles = (n + kTile - 1) / kTile;
    const uint32_t nfull = n / kTile;
    const uint32_t lt = lanemask_lt();
    constexpr uint32_t kBytes = kTile * (sizeof(uint64_t) + (kVals ? sizeof(uint32_t) : 0));

    auto issue = [&](int b, uint32_t t) {  // thread 0 only
        if (t < ntiles && bulk_ok && t < nfull) {
            mbar_expect_tx(&sm.mbar[b], kBytes);
            bulk_load(sm.keys[b], keys + (size_t)t * kTile, kTile * sizeof(uint64_t), &sm.mbar[b]);
            if (kVals) bulk_load(sm.ptrs[b], ptrs + (size_t)t * kTile, kTile * sizeof(uint32_t), &sm.mbar[b]);
        }
    };

    uint32_t next_id = 0;
    if (tid == 0) {
        mbar_init(&sm.mbar[0], 1);
        mbar_init(&sm.mbar[1], 1);
        fence_mbar_init();
        for (int b = 0; b < 2; ++b) {
            const uint32_t t = atomicAdd(tile_counter, 1u);
            sm.tile_of[b] = t;
            issue(b, t);
        }
        next_id = atomicAdd(tile_counter, 1u);
    }
    __syncthreads();
    uint32_t phase[2] = {0u, 0u};

    for (uint32_t it = 0;; ++it) {
        const int b = it & 1;
        const uint32_t tile = sm.tile_of[b];
        if (tile >= ntiles) break;
        const uint32_t base = tile * kTile;
        const uint32_t valid = min(n - base, (uint32_t)kTile);
        if (bulk_ok && tile < nfull) {
            uint32_t polls = 0;
            while (!mbar_try_wait(&sm.mbar[b], phase[b]))
                if (wait_expired(polls, spin_limit, status)) break;
            phase[b] ^= 1u;
        } else {
            for (uint32_t s = tid; s < valid; s += kThreads) {
                sm.keys[b][s] = ld_stream(keys + base + s);
                if (kVals) sm.ptrs[b][s] = ld_stream(ptrs + base + s);
            }
        }
        __syncthreads();

        // ---- rows of this thread (warp-striped), heads, gathered values
        const uint32_t wofs = warp * 32 * kIpt;  // first row of this warp in the tile
        uint64_t k[kIpt];
        uint64_t v[kIpt];
        uint32_t hmask = 0;  // bit j: row (j, lane) is a head
#pragma unroll
        for (int j = 0; j < kIpt; ++j) {
            const uint32_t s = wofs + j * 32 + lane;
            k[j] = s < valid ? sm.keys[b][s] : 0ull;
        }
        {
            // the row before the warp's first row
            uint64_t before = 0;
            bool have_before = true;
            if (wofs > 0) before = sm.keys[b][wofs - 1];
            else if (base > 0) before = keys[base - 1];
            else have_before = false;
            uint64_t prev31 = before;  // key of lane 31 in the previous item
#pragma unroll
            for (int j = 0; j < kIpt; ++j) {
                const uint32_t s = wofs + j * 32 + lane;
                uint64_t pk = shfl_up_u64(k[j], 1);
                if (lane == 0) pk = prev31;
                const bool first_row = (j == 0 && lane == 0 && !have_before);
                if (s < valid && (first_row || pk != k[j])) hmask |= 1u << j;
                prev31 = shfl_u64(k[j], 31);
            }
        }
        if (kVals) {
#pragma unroll
            for (int j = 0; j < kIpt; ++j) {
                const uint32_t s = wofs + j * 32 + lane;
                if (s < valid) {
                    const uint32_t p = sm.ptrs[b][s];
                    if (kVals == 8) v[j] = __ldg(static_cast<const unsigned long long*>(val_col) + p);
                    else v[j] = __ldg(static_cast<const unsigned int*>(val_col) + p);
                } else {
                    v[j] = 0;
                }
            }
        } else {
#pragma unroll
            for (int j = 0; j < kIpt; ++j) v[j] = 0;
        }

        // ---- warp aggregate (rows in order: item j, then lane)
        Agg wa = agg_identity();
        {
            uint64_t run_sum = 0;  // sum over the warp's rows so far
#pragma unroll
            for (int j = 0; j < kIpt; ++j) {
                const uint32_t m = __ballot_sync(0xffffffffu, (hmask >> j) & 1u);
                uint64_t incl = v[j];
                if (kVals) {
#pragma unroll
                    for (int o = 1; o < 32; o <<= 1) {
                        const uint64_t y = shfl_up_u64(incl, o);
                        if (lane >= (uint32_t)o) incl += y;
                    }
                }
                if (m) {
                    const int last = 31 - __clz(m);
                    wa.heads += __popc(m);
                    wa.last_row = base + wofs + j * 32 + last;
                    if (kVals) wa.last_p = run_sum + shfl_u64(incl - v[j], last);
                }
                if (kVals) run_sum += shfl_u64(incl, 31);
            }
            wa.sum = run_sum;
        }
        if (lane == 0) sm.warp_agg[warp] = wa;
        __syncthreads();

        // ---- tile aggregate, publish, look back, per-warp prefixes (thread 0)
        if (tid == 0) {
            Agg t = sm.warp_agg[0];
            for (int w = 1; w < kWarps; ++w) t = agg_combine(t, sm.warp_agg[w]);
            Agg excl = agg_identity();
            if (tile == 0) {
                store_agg(&recs[0].prefix, t);
                __threadfence();
                st_release(flags, kRecPrefix);
            } else {
                store_agg(&recs[tile].agg, t);
                __threadfence();
                st_release(flags + tile, kRecAgg);
                uint32_t j = tile - 1;
                uint32_t polls = 0;
                bool have = false;
                for (;;) {
                    const uint32_t f = ld_acquire(flags + j);
                    if (f == 0) {
                        if (wait_expired(polls, spin_limit, status)) break;
                        continue;
                    }
                    const Agg r = load_agg(f == kRecPrefix ? &recs[j].prefix : &recs[j].agg);
                    excl = have ? agg_combine(r, excl) : r;
                    have = true;
                    if (f == kRecPrefix || j == 0) break;
                    --j;
                }
                store_agg(&recs[tile].prefix, agg_combine(excl, t));
                __threadfence();
                st_release(flags + tile, kRecPrefix);
            }
            Agg run = excl;
            for (int w = 0; w < kWarps; ++w) {
                sm.warp_prefix[w] = run;
                run = agg_combine(run, sm.warp_agg[w]);
            }
            if (base + valid == n) {  // the last tile closes the last run
                if (run.heads) {
                    const uint64_t g = run.heads - 1;
                    if (g < cap) {
                        if (out_counts) out_counts[g] = n - run.last_row;
                        if (kVals && out_sums) out_sums[g] = run.sum - run.last_p;
                    }
                }
                *nkeys_out = run.heads;
            }
        }
        __syncthreads();

        // ---- emit: each head writes its key and closes the previous run
        {
            const Agg wp = sm.warp_prefix[warp];
            uint64_t heads = wp.heads;          // heads before the current item
            uint64_t prev_row = wp.last_row;    // last head before the current item
            uint64_t prev_p = wp.last_p;        // P at that head
            uint64_t run_p = wp.sum;            // P at the current item's first row
#pragma unroll
            for (int j = 0; j < kIpt; ++j) {
                const uint32_t m = __ballot_sync(0xffffffffu, (hmask >> j) & 1u);
                uint64_t incl = v[j];
                if (kVals) {
#pragma unroll
                    for (int o = 1; o < 32; o <<= 1) {
                        const uint64_t y = shfl_up_u64(incl, o);
                        if (lane >= (uint32_t)o) incl += y;
                    }
                }
                const uint64_t p_row = run_p + incl - v[j];  // P at this row
                const uint32_t below = m & lt;
                const int src = below ? 31 - __clz(below) : 0;
                const uint64_t p_src = kVals ? shfl_u64(p_row, src) : 0ull;
                if ((m >> lane) & 1u) {
                    const uint64_t row = base + wofs + j * 32 + lane;
                    const uint64_t g = heads + __popc(below);
                    const uint64_t pr = below ? (uint64_t)(base + wofs + j * 32 + src) : prev_row;
                    const uint64_t pp = below ? p_src : prev_p;
                    if (g < cap) out_keys[g] = k[j];
                    if (g >= 1 && g - 1 < cap) {
                        if (out_counts) out_counts[g - 1] = row - pr;
                        if (kVals && out_sums) out_sums[g - 1] = p_row - pp;
                    }
                }
                if (m) {
                    const int last = 31 - __clz(m);
                    heads += __popc(m);
                    prev_row = base + wofs + j * 32 + last;
                    if (kVals) prev_p = shfl_u64(p_row, last);
                }
                if (kVals) run_p += shfl_u64(incl, 31);
            }
        }
        __syncthreads();  // the buffer is free again
        if (tid == 0) {
            fence_proxy_async_smem();
            sm.tile_of[b] = next_id;
            issue(b, next_id);
            next_id = atomicAdd(tile_counter, 1u);
        }
    }
}

template <int kVals>
int launch_keyed(const uint64_t* keys, const uint32_t* ptrs, uint64_t n, const void* vals, uint64_t* ok,
                 uint64_t* oc, uint64_t* os, uint64_t cap, uint64_t* nkeys, void* scratch, cudaStream_t s) {
    const uint64_t ntiles = (n + kTile - 1) / kTile;
    Carver c(scratch);
    uint32_t* counter = c.take<uint32_t>(1);
    uint32_t* flags = c.take<uint32_t>(ntiles);
    const size_t zero_bytes = c.off;
    TileRec* recs = c.take<TileRec>(ntiles);
    SBH_CUDA(cudaMemsetAsync(counter, 0, zero_bytes, s));
    auto kern = keyed_kernel<kVals>;
    const size_t smem = sizeof(KeyedSmem);
    SBH_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int per_sm = 0;
    SBH_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kThreads, smem));
    if (per_sm < 1) per_sm = 1;
    const unsigned grid = (unsigned)min_u64(ntiles, (uint64_t)num_sms() * per_sm);
    const int bulk_ok = ((reinterpret_cast<uintptr_t>(keys) | (kVals ? reinterpret_cast<uintptr_t>(ptrs) : 0)) & 15) == 0;
    SBH_TIMED("keyed_reduce", s,
              kern<<<grid, kThreads, smem, s>>>(keys, ptrs, (uint32_t)n, vals, ok, oc, os, cap, nkeys, flags, recs,
                                                counter, spin_limit(), status_word(), bulk_ok));
    SBH_LAUNCHED();
    return SBH_OK;
}

size_t keyed_scratch(uint64_t n) {
    const uint64_t ntiles = (n + kTile - 1) / kTile;
    Carver c(nullptr);
    c.take<uint32_t>(1);
    c.take<uint32_t>(ntiles);
    c.take<TileRec>(ntiles);
    return c.bytes();
}

}  // namespace
}  // namespace sbh

extern "C" int sbh_group_reduce(const uint64_t* d_keys, const uint32_t* d_ptrs, uint64_t n, const void* d_val_col,
                                int val_bytes, uint64_t* d_out_keys, uint64_t* d_out_counts, uint64_t* d_out_sums,
                                uint64_t cap, uint64_t* d_nkeys, void* d_scratch, size_t* scratch_bytes,
                                void* stream) {
    using namespace sbh;
    clear_error();
    if (n > 0xFFFFFFFFull) { set_error("n must be < 2^32"); return SBH_EINVAL; }
    bool done = false;
    int rc = scratch_check(d_scratch, scratch_bytes, keyed_scratch(n), &done);
    if (rc || done) return rc;
    if (!d_nkeys) { set_error("d_nkeys is NULL"); return SBH_EINVAL; }
    cudaStream_t s = as_stream(stream);
    if (n == 0) {
        SBH_CUDA(cudaMemsetAsync(d_nkeys, 0, sizeof(uint64_t), s));
        return SBH_OK;
    }
    if (!d_keys || (cap && !d_out_keys)) { set_error("null pointer"); return SBH_EINVAL; }
    const bool with_vals = d_val_col && d_out_sums;
    if (with_vals && val_bytes != 4 && val_bytes != 8) { set_error("val_bytes must be 4 or 8"); return SBH_EINVAL; }
    if (with_vals && !d_ptrs) { set_error("d_ptrs is NULL"); return SBH_EINVAL; }
    if (!with_vals) return launch_keyed<0>(d_keys, d_ptrs, n, nullptr, d_out_keys, d_out_counts, nullptr, cap, d_nkeys, d_scratch, s);
    if (val_bytes == 8)
        return launch_keyed<8>(d_keys, d_ptrs, n, d_val_col, d_out_keys, d_out_counts, d_out_sums, cap, d_nkeys, d_scratch, s);
    return launch_keyed<4>(d_keys, d_ptrs, n, d_val_col, d_out_keys, d_out_counts, d_out_sums, cap, d_nkeys, d_scratch, s);
}
