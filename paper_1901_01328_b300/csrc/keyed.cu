// A6 Keyed reduction: per-key count and sum of a nonresident value column
// over a KPA sorted by key.
//
// A key's rows are one contiguous run, so its count and sum are differences
// of prefix quantities at run boundaries (heads):
//     count(run) = next head row - head row
//     sum(run)   = P(next head) - P(head),  P(i) = sum of v over rows < i,
// exactly, modulo 2^64.  So the reduction needs only a plain prefix sum of the
// gathered values and the position of the last head -- no segmented scan.
//
// Three launches (five above 4096 tiles), no waits between CTAs:
//   tile_agg   per tile of 4096 rows: heads, total, last head row, and the
//              prefix at the last head;
//   tile_scan  scans the tile aggregates into tile prefixes (one CTA; above
//              4096 tiles, block totals up, one CTA over those, then add);
//   emit       per tile again: each head writes its key, and the previous
//              run's count and sum, at output index = number of heads before.
// Rows are read warp-striped straight from global memory (coalesced), so the
// kernels need almost no shared memory and many CTAs stay resident.
#include <mutex>

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

__host__ __device__ __forceinline__ Agg agg_identity() { return {0ull, kNoRow, 0ull, 0ull}; }

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

__device__ __forceinline__ uint64_t shfl_u64(uint64_t v, int src) { return __shfl_sync(0xffffffffu, v, src); }
__device__ __forceinline__ uint64_t shfl_up_u64(uint64_t v, int o) { return __shfl_up_sync(0xffffffffu, v, o); }

// Loads this thread's rows of the tile (warp-striped), their head bits and
// gathered values.
template <int kVals>
__device__ __forceinline__ void load_rows(const uint64_t* __restrict__ keys, const uint32_t* __restrict__ ptrs,
                                          const void* __restrict__ val_col, uint32_t n, uint32_t base, uint32_t wofs,
                                          uint32_t lane, uint64_t (&k)[kIpt], uint64_t (&v)[kIpt],
                                          uint32_t& hmask) {
    const uint32_t first = base + wofs;  // first row of this warp
    if (!kVals && first < n) {
        // Counts only: when the warp's first and last rows hold one key (the
        // rows are sorted), all of them do, and only the first can be a head;
        // the other rows are not read.  (With Zipf-skewed keys about half of
        // the 512-row warp ranges are one key.)
        const uint32_t last = min(first + 32 * kIpt, n) - 1;
        const uint64_t kf = keys[first], kl = keys[last];
        if (kf == kl) {
#pragma unroll
            for (int j = 0; j < kIpt; ++j) {
                k[j] = kf;
                v[j] = 0;
            }
            hmask = (lane == 0 && (first == 0 || keys[first - 1] != kf)) ? 1u : 0u;
            return;
        }
    }
#pragma unroll
    for (int j = 0; j < kIpt; ++j) {
        const uint32_t r = first + j * 32 + lane;
        k[j] = r < n ? ld_stream(keys + r) : 0ull;
    }
    if (kVals) {
        uint32_t p[kIpt];
#pragma unroll
        for (int j = 0; j < kIpt; ++j) {
            const uint32_t r = first + j * 32 + lane;
            p[j] = r < n ? ld_stream(ptrs + r) : 0u;
        }
#pragma unroll
        for (int j = 0; j < kIpt; ++j) {
            const uint32_t r = first + j * 32 + lane;
            if (r < n) {
                if (kVals == 8) v[j] = __ldg(static_cast<const unsigned long long*>(val_col) + p[j]);
                else v[j] = __ldg(static_cast<const unsigned int*>(val_col) + p[j]);
            } else {
                v[j] = 0;
            }
        }
    } else {
#pragma unroll
        for (int j = 0; j < kIpt; ++j) v[j] = 0;
    }
    const bool have_before = first > 0;
    uint64_t prev31 = have_before ? keys[first - 1] : 0ull;  // row before the warp's first row
    hmask = 0;
#pragma unroll
    for (int j = 0; j < kIpt; ++j) {
        const uint32_t r = first + j * 32 + lane;
        uint64_t pk = shfl_up_u64(k[j], 1);
        if (lane == 0) pk = prev31;
        const bool first_row = (j == 0 && lane == 0 && !have_before);
        if (r < n && (first_row || pk != k[j])) hmask |= 1u << j;
        prev31 = shfl_u64(k[j], 31);
    }
}

__device__ __forceinline__ uint64_t warp_incl_sum(uint64_t x, uint32_t lane) {
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint64_t y = shfl_up_u64(x, o);
        if (lane >= (uint32_t)o) x += y;
    }
    return x;
}

template <int kVals>
__global__ void __launch_bounds__(kThreads)
tile_agg_kernel(const uint64_t* __restrict__ keys, const uint32_t* __restrict__ ptrs, uint32_t n,
                const void* __restrict__ val_col, Agg* __restrict__ tile_aggs) {
    __shared__ Agg warp_agg[kWarps];
    const uint32_t lane = lane_id(), warp = threadIdx.x / 32;
    const uint32_t base = blockIdx.x * kTile, wofs = warp * 32 * kIpt;
    uint64_t k[kIpt], v[kIpt];
    uint32_t hmask;
    load_rows<kVals>(keys, ptrs, val_col, n, base, wofs, lane, k, v, hmask);
    Agg wa = agg_identity();
    uint64_t run_sum = 0;
#pragma unroll
    for (int j = 0; j < kIpt; ++j) {
        const uint32_t m = __ballot_sync(0xffffffffu, (hmask >> j) & 1u);
        uint64_t incl = kVals ? warp_incl_sum(v[j], lane) : 0ull;
        if (m) {
            const int last = 31 - __clz(m);
            wa.heads += __popc(m);
            wa.last_row = base + wofs + j * 32 + last;
            if (kVals) wa.last_p = run_sum + shfl_u64(incl - v[j], last);
        }
        if (kVals) run_sum += shfl_u64(incl, 31);
    }
    wa.sum = run_sum;
    if (lane == 0) warp_agg[warp] = wa;
    __syncthreads();
    if (threadIdx.x == 0) {
        Agg t = warp_agg[0];
        for (int w = 1; w < kWarps; ++w) t = agg_combine(t, warp_agg[w]);
        tile_aggs[blockIdx.x] = t;
    }
}

// Exclusive scan of the tile aggregates (in place), by one CTA: each thread
// combines a contiguous range of tiles (four loads in flight at a time), the
// CTA scans the range totals, and each thread walks its range again writing
// the prefixes.
__device__ __forceinline__ Agg shfl_up_agg(const Agg& a, int o) {
    Agg y;
    y.heads = shfl_up_u64(a.heads, o);
    y.last_row = shfl_up_u64(a.last_row, o);
    y.sum = shfl_up_u64(a.sum, o);
    y.last_p = shfl_up_u64(a.last_p, o);
    return y;
}

__global__ void __launch_bounds__(1024) tile_scan_kernel(Agg* __restrict__ aggs, uint32_t ntiles) {
    __shared__ Agg warp_tot[32];
    constexpr int kBatch = 4;
    const uint32_t lane = lane_id(), warp = threadIdx.x / 32;
    const uint32_t per = (ntiles + blockDim.x - 1) / blockDim.x;
    const uint32_t b0 = min(ntiles, threadIdx.x * per), b1 = min(ntiles, b0 + per);
    Agg local = agg_identity();
    for (uint32_t i = b0; i < b1; i += kBatch) {
        Agg a[kBatch];
#pragma unroll
        for (int u = 0; u < kBatch; ++u) a[u] = i + u < b1 ? aggs[i + u] : agg_identity();
#pragma unroll
        for (int u = 0; u < kBatch; ++u) local = agg_combine(local, a[u]);
    }
    Agg inc = local;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const Agg y = shfl_up_agg(inc, o);
        if (lane >= (uint32_t)o) inc = agg_combine(y, inc);
    }
    if (lane == 31) warp_tot[warp] = inc;
    __syncthreads();
    Agg run = agg_identity();
    for (uint32_t w = 0; w < warp; ++w) run = agg_combine(run, warp_tot[w]);
    Agg excl = shfl_up_agg(inc, 1);
    if (lane == 0) excl = agg_identity();
    run = agg_combine(run, excl);
    for (uint32_t i = b0; i < b1; i += kBatch) {
        Agg a[kBatch];
#pragma unroll
        for (int u = 0; u < kBatch; ++u) a[u] = i + u < b1 ? aggs[i + u] : agg_identity();
#pragma unroll
        for (int u = 0; u < kBatch; ++u) {
            if (i + u < b1) {
                aggs[i + u] = run;
                run = agg_combine(run, a[u]);
            }
        }
    }
}

// Many tiles: the scan runs over blocks of 1024 tile aggregates in three
// launches.  tile_scan_up writes each block's total, tile_scan_kernel scans
// the block totals (one CTA; at most 1024 of them), and tile_scan_add scans
// each block's aggregates in place from its block prefix.
__device__ __forceinline__ Agg cta_scan(const Agg& mine, Agg (&warp_tot)[32], Agg& incl) {
    const uint32_t lane = lane_id(), warp = threadIdx.x / 32;
    Agg inc = mine;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const Agg y = shfl_up_agg(inc, o);
        if (lane >= (uint32_t)o) inc = agg_combine(y, inc);
    }
    if (lane == 31) warp_tot[warp] = inc;
    __syncthreads();
    Agg before = agg_identity();
    for (uint32_t w = 0; w < warp; ++w) before = agg_combine(before, warp_tot[w]);
    Agg excl = shfl_up_agg(inc, 1);
    if (lane == 0) excl = agg_identity();
    incl = agg_combine(before, inc);
    return agg_combine(before, excl);
}

__global__ void __launch_bounds__(1024) tile_scan_up_kernel(const Agg* __restrict__ aggs, uint32_t ntiles,
                                                            Agg* __restrict__ btot) {
    __shared__ Agg warp_tot[32];
    const uint32_t i = blockIdx.x * 1024 + threadIdx.x;
    Agg incl;
    cta_scan(i < ntiles ? aggs[i] : agg_identity(), warp_tot, incl);
    if (threadIdx.x == 1023) btot[blockIdx.x] = incl;
}

__global__ void __launch_bounds__(1024) tile_scan_add_kernel(Agg* __restrict__ aggs, uint32_t ntiles,
                                                             const Agg* __restrict__ bpre) {
    __shared__ Agg warp_tot[32];
    const uint32_t i = blockIdx.x * 1024 + threadIdx.x;
    const Agg mine = i < ntiles ? aggs[i] : agg_identity();
    Agg incl;
    const Agg excl = cta_scan(mine, warp_tot, incl);
    if (i < ntiles) aggs[i] = agg_combine(bpre[blockIdx.x], excl);
}

// A count as 8 or 4 bytes (counts are below 2^32: n < 2^32).
// The outputs are written once and not read again here: streaming stores
// (the emit for 256M rows 0.572 to 0.561 ms; evict-last stores 0.585).
__device__ __forceinline__ void store_count(void* out, int count_bytes, uint64_t i, uint64_t c) {
    if (count_bytes == 4) st_stream(static_cast<uint32_t*>(out) + i, static_cast<uint32_t>(c));
    else st_stream(static_cast<uint64_t*>(out) + i, c);
}

// (counts only: four CTAs an SM; with the count width a runtime argument
// the compiler took 84 registers, three CTAs an SM, and the emit ran 0.89
// against 0.58 ms for 256M rows)
template <int kVals>
__global__ void __launch_bounds__(kThreads, kVals ? 2 : 4)
emit_kernel(const uint64_t* __restrict__ keys, const uint32_t* __restrict__ ptrs, uint32_t n,
            const void* __restrict__ val_col, const Agg* __restrict__ tile_prefix, uint32_t ntiles,
            uint64_t* __restrict__ out_keys, void* __restrict__ out_counts, int count_bytes, uint64_t* __restrict__ out_sums,
            uint64_t cap, uint64_t* __restrict__ nkeys_out) {
    __shared__ Agg warp_agg[kWarps];
    const uint32_t lane = lane_id(), warp = threadIdx.x / 32;
    const uint32_t base = blockIdx.x * kTile, wofs = warp * 32 * kIpt;
    const uint32_t lt = lanemask_lt();
    uint64_t k[kIpt], v[kIpt];
    uint32_t hmask;
    load_rows<kVals>(keys, ptrs, val_col, n, base, wofs, lane, k, v, hmask);

    // warp aggregates again, to place each warp after the ones before it
    {
        Agg wa = agg_identity();
        uint64_t run_sum = 0;
#pragma unroll
        for (int j = 0; j < kIpt; ++j) {
            const uint32_t m = __ballot_sync(0xffffffffu, (hmask >> j) & 1u);
            uint64_t incl = kVals ? warp_incl_sum(v[j], lane) : 0ull;
            if (m) {
                const int last = 31 - __clz(m);
                wa.heads += __popc(m);
                wa.last_row = base + wofs + j * 32 + last;
                if (kVals) wa.last_p = run_sum + shfl_u64(incl - v[j], last);
            }
            if (kVals) run_sum += shfl_u64(incl, 31);
        }
        wa.sum = run_sum;
        if (lane == 0) warp_agg[warp] = wa;
    }
    __syncthreads();
    Agg wp = tile_prefix[blockIdx.x];
    for (uint32_t w = 0; w < warp; ++w) wp = agg_combine(wp, warp_agg[w]);

    uint64_t heads = wp.heads;        // heads before the current item
    uint64_t prev_row = wp.last_row;  // last head before the current item
    uint64_t prev_p = wp.last_p;      // P at that head
    uint64_t run_p = wp.sum;          // P at the current item's first row
#pragma unroll
    for (int j = 0; j < kIpt; ++j) {
        const uint32_t m = __ballot_sync(0xffffffffu, (hmask >> j) & 1u);
        const uint64_t incl = kVals ? warp_incl_sum(v[j], lane) : 0ull;
        const uint64_t p_row = run_p + incl - v[j];  // P at this row
        const uint32_t below = m & lt;
        const int src = below ? 31 - __clz(below) : 0;
        const uint64_t p_src = kVals ? shfl_u64(p_row, src) : 0ull;
        if ((m >> lane) & 1u) {
            const uint64_t row = base + wofs + j * 32 + lane;
            const uint64_t g = heads + __popc(below);
            const uint64_t pr = below ? (uint64_t)(base + wofs + j * 32 + src) : prev_row;
            const uint64_t pp = below ? p_src : prev_p;
            if (g < cap) st_stream(out_keys + g, k[j]);
            if (g >= 1 && g - 1 < cap) {
                if (out_counts) store_count(out_counts, count_bytes, g - 1, row - pr);
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
    // the thread holding the last row closes the last run
    if (blockIdx.x == ntiles - 1 && warp == kWarps - 1 && lane == 31) {
        // heads/prev_row/prev_p/run_p now describe everything up to the tile end
        const uint64_t total_heads = heads;
        if (total_heads) {
            const uint64_t g = total_heads - 1;
            if (g < cap) {
                if (out_counts) store_count(out_counts, count_bytes, g, n - prev_row);
                if (kVals && out_sums) out_sums[g] = run_p - prev_p;
            }
        }
        *nkeys_out = total_heads;
    }
}

template <int kVals>
int launch_keyed(const uint64_t* keys, const uint32_t* ptrs, uint64_t n, const void* vals, uint64_t* ok,
                 void* oc, int cb, uint64_t* os, uint64_t cap, uint64_t* nkeys, void* scratch, cudaStream_t s) {
    const uint32_t ntiles = (uint32_t)((n + kTile - 1) / kTile);
    Carver c(scratch);
    Agg* aggs = c.take<Agg>(ntiles);
    Agg* btot = c.take<Agg>(ntiles / 1024 + 1);
    SBH_TIMED("keyed_tile_agg", s,
              tile_agg_kernel<kVals><<<ntiles, kThreads, 0, s>>>(keys, ptrs, (uint32_t)n, vals, aggs));
    SBH_LAUNCHED();
    if (ntiles > 4096) {
        const uint32_t nblk = (ntiles + 1023) / 1024;
        SBH_TIMED("keyed_tile_scan_up", s, tile_scan_up_kernel<<<nblk, 1024, 0, s>>>(aggs, ntiles, btot));
        SBH_LAUNCHED();
        SBH_TIMED("keyed_tile_scan", s, tile_scan_kernel<<<1, 1024, 0, s>>>(btot, nblk));
        SBH_LAUNCHED();
        SBH_TIMED("keyed_tile_scan_add", s, tile_scan_add_kernel<<<nblk, 1024, 0, s>>>(aggs, ntiles, btot));
    } else {
        SBH_TIMED("keyed_tile_scan", s, tile_scan_kernel<<<1, 1024, 0, s>>>(aggs, ntiles));
    }
    SBH_LAUNCHED();
    SBH_TIMED("keyed_emit", s,
              emit_kernel<kVals><<<ntiles, kThreads, 0, s>>>(keys, ptrs, (uint32_t)n, vals, aggs, ntiles, ok, oc, cb, os,
                                                             cap, nkeys));
    SBH_LAUNCHED();
    return SBH_OK;
}

size_t keyed_scratch(uint64_t n) {
    const uint64_t ntiles = (n + kTile - 1) / kTile;
    Carver c(nullptr);
    c.take<Agg>(ntiles);
    c.take<Agg>(ntiles / 1024 + 1);
    return c.bytes();
}

}  // namespace
}  // namespace sbh

extern "C" int sbh_group_reduce(const uint64_t* d_keys, const uint32_t* d_ptrs, uint64_t n, const void* d_val_col,
                                int val_bytes, uint64_t* d_out_keys, void* d_out_counts, int count_bytes,
                                uint64_t* d_out_sums, uint64_t cap, uint64_t* d_nkeys, void* d_scratch,
                                size_t* scratch_bytes, void* stream) {
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
    if (d_out_counts && count_bytes != 4 && count_bytes != 8) { set_error("count_bytes must be 4 or 8"); return SBH_EINVAL; }
    const bool with_vals = d_val_col && d_out_sums;
    if (with_vals && val_bytes != 4 && val_bytes != 8) { set_error("val_bytes must be 4 or 8"); return SBH_EINVAL; }
    if (with_vals && !d_ptrs) { set_error("d_ptrs is NULL"); return SBH_EINVAL; }
    const int cb = count_bytes;
    if (!with_vals)
        return launch_keyed<0>(d_keys, d_ptrs, n, nullptr, d_out_keys, d_out_counts, cb, nullptr, cap, d_nkeys,
                               d_scratch, s);
    if (val_bytes == 8)
        return launch_keyed<8>(d_keys, d_ptrs, n, d_val_col, d_out_keys, d_out_counts, cb, d_out_sums, cap, d_nkeys,
                               d_scratch, s);
    return launch_keyed<4>(d_keys, d_ptrs, n, d_val_col, d_out_keys, d_out_counts, cb, d_out_sums, cap, d_nkeys,
                           d_scratch, s);
}

// ---------------------------------------------------------------------------
// sbh_group_reduce_noalloc: the keyed reduction with its working memory in a
// fixed device array instead of caller scratch, for callers that cannot
// allocate device memory at the point of the call.
namespace sbh {
namespace {

constexpr uint64_t kNoAllocMaxRows = 1ull << 28;  // 268,435,456 rows
constexpr size_t kNoAllocTiles = (kNoAllocMaxRows + kTile - 1) / kTile;
// the tile aggregates (2 MiB) and the block totals of the tile scan, laid
// out as keyed_scratch carves them; held on every GPU that loads the library
constexpr size_t kNoAllocBytes =
    kNoAllocTiles * sizeof(Agg) + (((kNoAllocTiles / 1024 + 1) * sizeof(Agg) + 255) & ~size_t(255));

// One copy per device.  Host code must not use this name as an address: it
// is a host-side stand-in; the device address comes from
// cudaGetSymbolAddress below.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

constexpr int kNoAllocMaxDevices = 64;
std::mutex g_noalloc_mu;
void* g_noalloc_ptr[kNoAllocMaxDevices] = {nullptr};

// Device address of g_noalloc_scratch on the current device, looked up once
// per device (with that device current).
int noalloc_scratch(void** out) {
    int dev = 0;
    SBH_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kNoAllocMaxDevices) {
        set_error("device ordinal %d out of range", dev);
        return SBH_EINVAL;
    }
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
        void* p = nullptr;
        SBH_CUDA(cudaGetSymbolAddress(&p, g_noalloc_scratch));
        g_noalloc_ptr[dev] = p;
    }
    *out = g_noalloc_ptr[dev];
    return SBH_OK;
}

}  // namespace
}  // namespace sbh

extern "C" int sbh_group_reduce_noalloc(const uint64_t* d_keys, const uint32_t* d_ptrs, uint64_t n,
                                        const void* d_val_col, int val_bytes, uint64_t* d_out_keys,
                                        void* d_out_counts, int count_bytes, uint64_t* d_out_sums, uint64_t cap,
                                        uint64_t* d_nkeys, void* stream) {
    using namespace sbh;
    clear_error();
    if (n > kNoAllocMaxRows) {
        set_error("sbh_group_reduce_noalloc handles at most %llu rows (got %llu); use sbh_group_reduce",
                  (unsigned long long)kNoAllocMaxRows, (unsigned long long)n);
        return SBH_EINVAL;
    }
    void* scratch = nullptr;
    int rc = noalloc_scratch(&scratch);
    if (rc) return rc;
    size_t bytes = kNoAllocBytes;
    return sbh_group_reduce(d_keys, d_ptrs, n, d_val_col, val_bytes, d_out_keys, d_out_counts, count_bytes,
                            d_out_sums, cap, d_nkeys, scratch, &bytes, stream);
}
