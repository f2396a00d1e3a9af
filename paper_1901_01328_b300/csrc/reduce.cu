// A7 top-K per key, on a KPA sorted by key.
//
// A key's rows are one contiguous run (a segment), so the work splits by
// segment once the segments are known:
//   heads_count   per tile of 4096 rows: number of segment heads;
//   heads_scan    one CTA: exclusive scan of the tile counts, and the
//                 number of segments;
//   heads_emit    per tile: each head writes its key to the output and its
//                 row to seg_start, at index = number of heads before it;
//   small         grid-stride over segments: a segment of at most 64 rows is
//                 reduced by one thread (its pointers read in order, values
//                 gathered), a longer one is listed as medium (up to 4096
//                 rows) or long;
//   medium        one warp per listed medium segment, then a warp merge;
//   long_scan     one CTA: every listed segment is cut into chunks of 16384
//                 rows; exclusive scan of the chunk counts;
//   long_chunks   grid-stride over chunks: a CTA reduces a chunk (each
//                 thread a strided share, then warp and CTA merges); a
//                 one-chunk segment writes its result, otherwise the chunk's
//                 list goes to scratch and the CTA that finishes last (an
//                 atomic count per segment, no waiting) merges the segment's
//                 lists and writes the result.
// No kernel waits on another CTA.
#include "common.cuh"

namespace sbh {
namespace {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr int kIpt = 16;
constexpr int kTile = kThreads * kIpt;
constexpr uint32_t kLaneMax = 64;     // longest segment reduced by one thread
constexpr uint32_t kWarpMax = 4096;   // longest segment reduced by one warp
constexpr uint32_t kChunk = 16384;    // rows of a long segment per CTA

// ------------------------------------------------------------ aggregates
// The best K (value, ptr) pairs seen, ordered by value descending, then ptr
// ascending; n of them are valid.
template <int KMAX>
struct TopK {
    uint32_t n;
    uint64_t v[KMAX];
    uint32_t p[KMAX];
    __device__ __forceinline__ static TopK identity() {
        TopK t;
        t.n = 0;
#pragma unroll
        for (int s = 0; s < KMAX; ++s) { t.v[s] = 0; t.p[s] = 0xFFFFFFFFu; }
        return t;
    }
    __device__ __forceinline__ static bool better(uint64_t va, uint32_t pa, uint64_t vb, uint32_t pb) {
        return va > vb || (va == vb && pa < pb);
    }
    // insert one pair, keeping at most k
    __device__ __forceinline__ void add_row(uint64_t val, uint32_t ptr, int k) {
        if (n == (uint32_t)k && !better(val, ptr, v[k - 1], p[k - 1])) return;
        uint32_t pos = n < (uint32_t)k ? n : (uint32_t)k - 1;
#pragma unroll
        for (int s = KMAX - 1; s > 0; --s) {
            if (s <= (int)pos && better(val, ptr, v[s - 1], p[s - 1])) {
                v[s] = v[s - 1];
                p[s] = p[s - 1];
                pos = s - 1;
            }
        }
        v[pos] = val;
        p[pos] = ptr;
        if (n < (uint32_t)k) ++n;
    }
    // merge another list into this one, keeping at most k
    __device__ __forceinline__ void absorb(const TopK& b, int k) {
#pragma unroll
        for (int s = 0; s < KMAX; ++s)
            if (s < (int)b.n) add_row(b.v[s], b.p[s], k);
    }
    __device__ __forceinline__ void shfl_xor(const TopK& src, int o) {
        n = __shfl_xor_sync(0xffffffffu, src.n, o);
#pragma unroll
        for (int s = 0; s < KMAX; ++s) {
            v[s] = __shfl_xor_sync(0xffffffffu, src.v[s], o);
            p[s] = __shfl_xor_sync(0xffffffffu, src.p[s], o);
        }
    }
};

template <int KMAX>
__device__ __forceinline__ void emit(uint64_t g, const TopK<KMAX>& a, int k, uint64_t cap, uint8_t* nvalid,
                                     uint64_t* vals, uint32_t* ptrs) {
    if (g >= cap) return;
    nvalid[g] = static_cast<uint8_t>(a.n);
#pragma unroll
    for (int s = 0; s < KMAX; ++s) {
        if (s < k) {
            vals[g * k + s] = s < (int)a.n ? a.v[s] : SBH_TOPK_PAD_VAL;
            ptrs[g * k + s] = s < (int)a.n ? a.p[s] : SBH_TOPK_PAD_PTR;
        }
    }
}

template <int kVals>
__device__ __forceinline__ uint64_t gather(const void* col, uint32_t p) {
    if (kVals == 8) return __ldg(static_cast<const unsigned long long*>(col) + p);
    return __ldg(static_cast<const unsigned int*>(col) + p);
}

// ------------------------------------------------------------ segment heads
// Head bits of this thread's rows (warp-striped: row = base + warp's first
// row + j * 32 + lane).
__device__ __forceinline__ uint32_t head_bits(const uint64_t* __restrict__ keys, uint32_t n, uint32_t first,
                                              uint32_t lane, uint64_t (&k)[kIpt]) {
#pragma unroll
    for (int j = 0; j < kIpt; ++j) {
        const uint32_t r = first + j * 32 + lane;
        k[j] = r < n ? ld_stream(keys + r) : 0ull;
    }
    uint64_t prev = first > 0 ? keys[first - 1] : 0ull;
    uint32_t hmask = 0;
#pragma unroll
    for (int j = 0; j < kIpt; ++j) {
        const uint32_t r = first + j * 32 + lane;
        uint64_t pk = __shfl_up_sync(0xffffffffu, k[j], 1);
        if (lane == 0) pk = prev;
        if (r < n && (r == 0 || pk != k[j])) hmask |= 1u << j;
        prev = __shfl_sync(0xffffffffu, k[j], 31);
    }
    return hmask;
}

__global__ void __launch_bounds__(kThreads) heads_count_kernel(const uint64_t* __restrict__ keys, uint32_t n,
                                                               uint32_t* __restrict__ tile_cnt) {
    __shared__ uint32_t wc[kWarps];
    const uint32_t lane = lane_id(), warp = threadIdx.x / 32;
    const uint32_t first = blockIdx.x * kTile + warp * 32 * kIpt;
    uint64_t k[kIpt];
    const uint32_t hmask = head_bits(keys, n, first, lane, k);
    const uint32_t c = __reduce_add_sync(0xffffffffu, __popc(hmask));
    if (lane == 0) wc[warp] = c;
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t t = 0;
        for (int w = 0; w < kWarps; ++w) t += wc[w];
        tile_cnt[blockIdx.x] = t;
    }
}

// Exclusive scan of the tile head counts in place (one CTA); the number of
// segments goes to *nseg_out (and to nseg32 for the later kernels).
__global__ void __launch_bounds__(1024) heads_scan_kernel(uint32_t* __restrict__ cnt, uint32_t ntiles,
                                                          uint64_t* __restrict__ nseg_out,
                                                          uint32_t* __restrict__ nseg32, uint32_t* __restrict__ seg_start,
                                                          uint32_t n) {
    __shared__ uint32_t wt[32];
    __shared__ uint32_t carry;
    const uint32_t lane = lane_id(), warp = threadIdx.x / 32;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (uint32_t c0 = 0; c0 < ntiles; c0 += blockDim.x) {
        const uint32_t i = c0 + threadIdx.x;
        const uint32_t v = i < ntiles ? cnt[i] : 0u;
        uint32_t x = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= (uint32_t)o) x += y;
        }
        if (lane == 31) wt[warp] = x;
        __syncthreads();
        uint32_t before = carry;
        for (uint32_t w = 0; w < warp; ++w) before += wt[w];
        if (i < ntiles) cnt[i] = before + x - v;
        __syncthreads();
        if (threadIdx.x == blockDim.x - 1) carry = before + x;
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        *nseg_out = carry;
        *nseg32 = carry;
        seg_start[carry] = n;  // the end of the last segment
    }
}

__global__ void __launch_bounds__(kThreads) heads_emit_kernel(const uint64_t* __restrict__ keys, uint32_t n,
                                                              const uint32_t* __restrict__ tile_base,
                                                              uint64_t* __restrict__ out_keys, uint64_t cap,
                                                              uint32_t* __restrict__ seg_start) {
    __shared__ uint32_t wc[kWarps];
    const uint32_t lane = lane_id(), warp = threadIdx.x / 32;
    const uint32_t first = blockIdx.x * kTile + warp * 32 * kIpt;
    uint64_t k[kIpt];
    const uint32_t hmask = head_bits(keys, n, first, lane, k);
    const uint32_t c = __reduce_add_sync(0xffffffffu, __popc(hmask));
    if (lane == 0) wc[warp] = c;
    __syncthreads();
    uint32_t g = tile_base[blockIdx.x];
    for (uint32_t w = 0; w < warp; ++w) g += wc[w];
    const uint32_t lt = lanemask_lt();
#pragma unroll
    for (int j = 0; j < kIpt; ++j) {
        const uint32_t m = __ballot_sync(0xffffffffu, (hmask >> j) & 1u);
        if ((m >> lane) & 1u) {
            const uint32_t gi = g + __popc(m & lt);
            seg_start[gi] = first + j * 32 + lane;
            if (gi < cap) out_keys[gi] = k[j];
        }
        g += __popc(m);
    }
}

// ------------------------------------------------------------ short segments
template <int KMAX, int kVals>
__global__ void __launch_bounds__(kThreads) small_kernel(const uint32_t* __restrict__ ptrs,
                                                         const void* __restrict__ val_col,
                                                         const uint32_t* __restrict__ seg_start,
                                                         const uint32_t* __restrict__ nseg_p, int k, uint64_t cap,
                                                         uint8_t* __restrict__ nvalid, uint64_t* __restrict__ vals,
                                                         uint32_t* __restrict__ optrs,
                                                         uint32_t* __restrict__ long_list,
                                                         uint32_t* __restrict__ nlong,
                                                         uint32_t* __restrict__ mid_list,
                                                         uint32_t* __restrict__ nmid) {
    const uint32_t nseg = *nseg_p;
    const uint32_t stride = gridDim.x * blockDim.x;
    for (uint32_t g = blockIdx.x * blockDim.x + threadIdx.x; g < nseg; g += stride) {
        const uint32_t s = seg_start[g], e = seg_start[g + 1];
        if (e - s > kWarpMax) {
            long_list[atomicAdd(nlong, 1u)] = g;
            continue;
        }
        if (e - s > kLaneMax) {
            mid_list[atomicAdd(nmid, 1u)] = g;
            continue;
        }
        // four rows at a time: loads first, so that they are in flight together
        TopK<KMAX> t = TopK<KMAX>::identity();
        for (uint32_t rb = s; rb < e; rb += 4) {
            uint32_t p[4];
            uint64_t v[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) p[u] = rb + u < e ? __ldg(ptrs + rb + u) : 0u;
#pragma unroll
            for (int u = 0; u < 4; ++u) v[u] = rb + u < e ? gather<kVals>(val_col, p[u]) : 0ull;
#pragma unroll
            for (int u = 0; u < 4; ++u)
                if (rb + u < e) t.add_row(v[u], p[u], k);
        }
        emit(g, t, k, cap, nvalid, vals, optrs);
    }
}

// ------------------------------------------------------------ medium segments
template <int KMAX, int kVals>
__global__ void __launch_bounds__(kThreads) medium_kernel(const uint32_t* __restrict__ ptrs,
                                                          const void* __restrict__ val_col,
                                                          const uint32_t* __restrict__ seg_start,
                                                          const uint32_t* __restrict__ mid_list,
                                                          const uint32_t* __restrict__ nmid_p, int k, uint64_t cap,
                                                          uint8_t* __restrict__ nvalid, uint64_t* __restrict__ vals,
                                                          uint32_t* __restrict__ optrs) {
    const uint32_t nmid = *nmid_p;
    const uint32_t lane = lane_id();
    const uint32_t warps = gridDim.x * (blockDim.x / 32);
    for (uint32_t i = blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32; i < nmid; i += warps) {
        const uint32_t g = mid_list[i];
        const uint32_t s = seg_start[g], e = seg_start[g + 1];
        TopK<KMAX> t = TopK<KMAX>::identity();
        for (uint32_t rb = s + lane; rb < e; rb += 4 * 32) {
            uint32_t p[4];
            uint64_t v[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) p[u] = rb + u * 32 < e ? __ldg(ptrs + rb + u * 32) : 0u;
#pragma unroll
            for (int u = 0; u < 4; ++u) v[u] = rb + u * 32 < e ? gather<kVals>(val_col, p[u]) : 0ull;
#pragma unroll
            for (int u = 0; u < 4; ++u)
                if (rb + u * 32 < e) t.add_row(v[u], p[u], k);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            TopK<KMAX> y;
            y.shfl_xor(t, o);
            t.absorb(y, k);
        }
        if (lane == 0) emit(g, t, k, cap, nvalid, vals, optrs);
    }
}

// ------------------------------------------------------------ long segments
// Chunk counts of the listed segments, scanned (one CTA); chunk_off[i] is the
// first chunk of list entry i, chunk_off[nlong] the total.
__global__ void __launch_bounds__(1024) long_scan_kernel(const uint32_t* __restrict__ long_list,
                                                         const uint32_t* __restrict__ nlong_p,
                                                         const uint32_t* __restrict__ seg_start,
                                                         uint32_t* __restrict__ chunk_off) {
    __shared__ uint32_t wt[32];
    __shared__ uint32_t carry;
    const uint32_t nlong = *nlong_p;
    const uint32_t lane = lane_id(), warp = threadIdx.x / 32;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (uint32_t c0 = 0; c0 < nlong; c0 += blockDim.x) {
        const uint32_t i = c0 + threadIdx.x;
        uint32_t v = 0;
        if (i < nlong) {
            const uint32_t g = long_list[i];
            v = (seg_start[g + 1] - seg_start[g] + kChunk - 1) / kChunk;
        }
        uint32_t x = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= (uint32_t)o) x += y;
        }
        if (lane == 31) wt[warp] = x;
        __syncthreads();
        uint32_t before = carry;
        for (uint32_t w = 0; w < warp; ++w) before += wt[w];
        if (i < nlong) chunk_off[i] = before + x - v;
        __syncthreads();
        if (threadIdx.x == blockDim.x - 1) carry = before + x;
        __syncthreads();
    }
    if (threadIdx.x == 0) chunk_off[nlong] = carry;
}

// Merge of the CTA's per-thread lists into thread 0's.
template <int KMAX>
__device__ __forceinline__ TopK<KMAX> block_merge(TopK<KMAX> t, int k, TopK<KMAX>* wsm) {
    const uint32_t lane = lane_id(), warp = threadIdx.x / 32;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        TopK<KMAX> y;
        y.shfl_xor(t, o);
        t.absorb(y, k);
    }
    if (lane == 0) wsm[warp] = t;
    __syncthreads();
    if (threadIdx.x == 0)
        for (int w = 1; w < kWarps; ++w) t.absorb(wsm[w], k);
    __syncthreads();
    return t;
}

template <int KMAX, int kVals>
__global__ void __launch_bounds__(kThreads) long_kernel(const uint32_t* __restrict__ ptrs,
                                                        const void* __restrict__ val_col,
                                                        const uint32_t* __restrict__ seg_start,
                                                        const uint32_t* __restrict__ long_list,
                                                        const uint32_t* __restrict__ nlong_p,
                                                        const uint32_t* __restrict__ chunk_off,
                                                        uint32_t* __restrict__ done, TopK<KMAX>* __restrict__ partial,
                                                        int k, uint64_t cap, uint8_t* __restrict__ nvalid,
                                                        uint64_t* __restrict__ vals, uint32_t* __restrict__ optrs) {
    __shared__ TopK<KMAX> wsm[kWarps];
    __shared__ uint32_t last;
    const uint32_t nlong = *nlong_p;
    const uint32_t total = chunk_off[nlong];
    for (uint32_t w = blockIdx.x; w < total; w += gridDim.x) {
        // list entry of chunk w: last i with chunk_off[i] <= w
        uint32_t lo = 0, hi = nlong;
        while (hi - lo > 1) {
            const uint32_t mid = (lo + hi) / 2;
            if (chunk_off[mid] <= w) lo = mid;
            else hi = mid;
        }
        const uint32_t g = long_list[lo];
        const uint32_t c = w - chunk_off[lo], nch = chunk_off[lo + 1] - chunk_off[lo];
        const uint32_t s = seg_start[g], e = seg_start[g + 1];
        const uint32_t r0 = s + c * kChunk, r1 = min(e, r0 + kChunk);
        // eight rows of a thread at a time: their pointer loads, then their
        // value gathers, are all in flight together
        TopK<KMAX> t = TopK<KMAX>::identity();
        for (uint32_t rb = r0 + threadIdx.x; rb < r1; rb += 8 * kThreads) {
            uint32_t p[8];
            uint64_t v[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const uint32_t r = rb + u * kThreads;
                p[u] = r < r1 ? ld_stream(ptrs + r) : 0u;
            }
#pragma unroll
            for (int u = 0; u < 8; ++u) v[u] = rb + u * kThreads < r1 ? gather<kVals>(val_col, p[u]) : 0ull;
#pragma unroll
            for (int u = 0; u < 8; ++u)
                if (rb + u * kThreads < r1) t.add_row(v[u], p[u], k);
        }
        t = block_merge(t, k, wsm);
        if (nch == 1) {
            if (threadIdx.x == 0) emit(g, t, k, cap, nvalid, vals, optrs);
            continue;
        }
        if (threadIdx.x == 0) {
            partial[w] = t;
            __threadfence();
            last = atomicAdd(done + lo, 1u) == nch - 1;
        }
        __syncthreads();
        if (last) {
            // every other chunk of the segment has published its list
            __threadfence();
            TopK<KMAX> m = TopK<KMAX>::identity();
            for (uint32_t q = threadIdx.x; q < nch; q += kThreads) {
                const TopK<KMAX>* src = partial + chunk_off[lo] + q;
                TopK<KMAX> y;
                y.n = __ldcg(&src->n);
#pragma unroll
                for (int i = 0; i < KMAX; ++i) {
                    y.v[i] = __ldcg(reinterpret_cast<const unsigned long long*>(&src->v[i]));
                    y.p[i] = __ldcg(&src->p[i]);
                }
                m.absorb(y, k);
            }
            m = block_merge(m, k, wsm);
            if (threadIdx.x == 0) emit(g, m, k, cap, nvalid, vals, optrs);
        }
        __syncthreads();
    }
}

// ------------------------------------------------------------ scratch and launch
struct TopkScratch {
    uint32_t* tile_cnt;   // ntiles
    uint32_t* seg_start;  // n + 1
    uint32_t* long_list;  // n / (kLaneMax + 1) + 1
    uint32_t* chunk_off;  // n / (kLaneMax + 1) + 2
    uint32_t* mid_list;   // n / (kLaneMax + 1) + 1
    uint32_t* small;      // nseg, nlong, nmid
    uint32_t* done;       // n / (kWarpMax + 1) + 1 (zeroed with small)
    void* partial;        // max chunks
    size_t zero_bytes;
    size_t total;
};

template <int KMAX>
TopkScratch topk_carve(void* base, uint64_t n) {
    Carver c(base);
    TopkScratch t;
    const uint64_t ntiles = (n + kTile - 1) / kTile;
    const uint64_t maxmid = n / (kLaneMax + 1) + 1;
    const uint64_t maxlong = n / (kWarpMax + 1) + 1;
    t.tile_cnt = c.take<uint32_t>(ntiles);
    t.seg_start = c.take<uint32_t>(n + 1);
    t.long_list = c.take<uint32_t>(maxlong);
    t.chunk_off = c.take<uint32_t>(maxlong + 1);
    t.mid_list = c.take<uint32_t>(maxmid);
    t.small = c.take<uint32_t>(3);
    const size_t z0 = c.off - 3 * sizeof(uint32_t);
    t.done = c.take<uint32_t>(maxlong);
    t.zero_bytes = c.off - z0;
    t.partial = c.take<TopK<KMAX>>(n / kChunk + maxlong);
    t.total = c.bytes();
    return t;
}

template <int KMAX, int kVals>
int topk_run(const uint64_t* keys, const uint32_t* ptrs, uint64_t n, const void* vals, int K, uint64_t* ok,
             uint8_t* onv, uint64_t* ov, uint32_t* op, uint64_t cap, uint64_t* nkeys, void* scratch, cudaStream_t s) {
    TopkScratch t = topk_carve<KMAX>(scratch, n);
    const uint32_t n32 = static_cast<uint32_t>(n);
    const uint32_t ntiles = static_cast<uint32_t>((n + kTile - 1) / kTile);
    const int sms = num_sms();
    SBH_CUDA(cudaMemsetAsync(t.small, 0, t.zero_bytes, s));
    SBH_TIMED("topk_heads_count", s, heads_count_kernel<<<ntiles, kThreads, 0, s>>>(keys, n32, t.tile_cnt));
    SBH_LAUNCHED();
    SBH_TIMED("topk_heads_scan", s,
              heads_scan_kernel<<<1, 1024, 0, s>>>(t.tile_cnt, ntiles, nkeys, t.small, t.seg_start, n32));
    SBH_LAUNCHED();
    SBH_TIMED("topk_heads_emit", s,
              heads_emit_kernel<<<ntiles, kThreads, 0, s>>>(keys, n32, t.tile_cnt, ok, cap, t.seg_start));
    SBH_LAUNCHED();
    const unsigned sgrid = (unsigned)min_u64((n + kThreads - 1) / kThreads, (uint64_t)sms * 8);
    SBH_TIMED("topk_small", s,
              (small_kernel<KMAX, kVals><<<sgrid, kThreads, 0, s>>>(ptrs, vals, t.seg_start, t.small, K, cap, onv, ov,
                                                                   op, t.long_list, t.small + 1, t.mid_list,
                                                                   t.small + 2)));
    SBH_LAUNCHED();
    SBH_TIMED("topk_medium", s,
              (medium_kernel<KMAX, kVals><<<(unsigned)sms * 8, kThreads, 0, s>>>(ptrs, vals, t.seg_start, t.mid_list,
                                                                               t.small + 2, K, cap, onv, ov, op)));
    SBH_LAUNCHED();
    SBH_TIMED("topk_long_scan", s,
              long_scan_kernel<<<1, 1024, 0, s>>>(t.long_list, t.small + 1, t.seg_start, t.chunk_off));
    SBH_LAUNCHED();
    const unsigned lgrid = (unsigned)min_u64(n / kChunk + 64, (uint64_t)sms * 4);
    SBH_TIMED("topk_long", s,
              (long_kernel<KMAX, kVals><<<lgrid, kThreads, 0, s>>>(
                  ptrs, vals, t.seg_start, t.long_list, t.small + 1, t.chunk_off, t.done,
                  static_cast<TopK<KMAX>*>(t.partial), K, cap, onv, ov, op)));
    SBH_LAUNCHED();
    return SBH_OK;
}

template <int KMAX>
int topk_dispatch(const uint64_t* keys, const uint32_t* ptrs, uint64_t n, const void* vals, int vb, int K,
                  uint64_t* ok, uint8_t* onv, uint64_t* ov, uint32_t* op, uint64_t cap, uint64_t* nkeys,
                  void* scratch, cudaStream_t s) {
    if (vb == 8) return topk_run<KMAX, 8>(keys, ptrs, n, vals, K, ok, onv, ov, op, cap, nkeys, scratch, s);
    return topk_run<KMAX, 4>(keys, ptrs, n, vals, K, ok, onv, ov, op, cap, nkeys, scratch, s);
}

// ------------------------------------------------------------ median and distinct values per key
// The KPA is re-ordered by (key, value): a stable sort of (value, row) by
// value, then a stable sort of (key, row) by key.  Inside each key's run the
// values are then ascending: the median is the run's middle row, and the
// distinct values are the rows that start the run or differ from the row
// before (a keyed sum of those flags).
template <int kVals>
__global__ void __launch_bounds__(256) mu_gather_kernel(const uint32_t* __restrict__ ptrs, uint32_t n,
                                                        const void* __restrict__ col, uint64_t* __restrict__ v,
                                                        uint32_t* __restrict__ idx) {
    const uint32_t stride = gridDim.x * blockDim.x;
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        v[i] = gather<kVals>(col, ld_stream(ptrs + i));
        idx[i] = i;
    }
}

__global__ void __launch_bounds__(256) mu_keys_kernel(const uint64_t* __restrict__ keys,
                                                      const uint32_t* __restrict__ idx, uint32_t n,
                                                      uint64_t* __restrict__ k2) {
    const uint32_t stride = gridDim.x * blockDim.x;
    for (uint32_t j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += stride) k2[j] = __ldg(keys + idx[j]);
}

// w[j] = the value of row j in (key, value) order; f[j] = 1 where a key's run
// starts or the value changes; iota[j] = j.
__global__ void __launch_bounds__(256) mu_flags_kernel(const uint64_t* __restrict__ k3,
                                                       const uint32_t* __restrict__ idx3, uint32_t n,
                                                       const uint64_t* __restrict__ v, uint64_t* __restrict__ w,
                                                       uint32_t* __restrict__ f, uint32_t* __restrict__ iota) {
    const uint32_t stride = gridDim.x * blockDim.x;
    for (uint32_t j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += stride) {
        const uint64_t x = __ldg(v + idx3[j]);
        w[j] = x;
        iota[j] = j;
        f[j] = (j == 0 || k3[j] != k3[j - 1] || x != __ldg(v + idx3[j - 1])) ? 1u : 0u;
    }
}

__global__ void __launch_bounds__(256) mu_median_kernel(const uint32_t* __restrict__ seg_start,
                                                        const uint32_t* __restrict__ nseg_p,
                                                        const uint64_t* __restrict__ w, uint64_t cap,
                                                        uint64_t* __restrict__ median) {
    const uint32_t nseg = *nseg_p;
    const uint32_t stride = gridDim.x * blockDim.x;
    for (uint32_t g = blockIdx.x * blockDim.x + threadIdx.x; g < nseg && g < cap; g += stride) {
        const uint32_t s = seg_start[g], e = seg_start[g + 1];
        median[g] = w[s + (e - s - 1) / 2];
    }
}

struct MuScratch {
    uint64_t *v, *v1, *k2, *k3, *w, *counts;
    uint32_t *idx, *idx1, *idx3, *f, *iota, *tile_cnt, *seg_start, *small;
    uint64_t* nseg;
    void* sort_scr;
    size_t sort_bytes;
    void* red_scr;
    size_t red_bytes;
    size_t total;
};

MuScratch mu_carve(void* base, uint64_t n) {
    Carver c(base);
    MuScratch t;
    const uint64_t ntiles = (n + kTile - 1) / kTile;
    t.v = c.take<uint64_t>(n);
    t.v1 = c.take<uint64_t>(n);
    t.k2 = c.take<uint64_t>(n);
    t.k3 = c.take<uint64_t>(n);
    t.w = c.take<uint64_t>(n);
    t.counts = c.take<uint64_t>(n);
    t.idx = c.take<uint32_t>(n);
    t.idx1 = c.take<uint32_t>(n);
    t.idx3 = c.take<uint32_t>(n);
    t.f = c.take<uint32_t>(n);
    t.iota = c.take<uint32_t>(n);
    t.tile_cnt = c.take<uint32_t>(ntiles);
    t.seg_start = c.take<uint32_t>(n + 1);
    t.small = c.take<uint32_t>(2);
    t.nseg = c.take<uint64_t>(1);
    size_t sb = 0, rb = 0;
    sbh_kpa_sort(nullptr, nullptr, nullptr, nullptr, n, nullptr, &sb, nullptr);
    sbh_group_reduce(nullptr, nullptr, n, nullptr, 4, nullptr, nullptr, 8, nullptr, 0, nullptr, nullptr, &rb, nullptr);
    t.sort_bytes = sb;
    t.red_bytes = rb;
    t.sort_scr = c.take<char>(sb);
    t.red_scr = c.take<char>(rb);
    t.total = c.bytes();
    return t;
}

template <int kVals>
int mu_run(const uint64_t* keys, const uint32_t* ptrs, uint64_t n, const void* col, uint64_t* ok, uint64_t* omed,
           uint64_t* ouni, uint64_t cap, uint64_t* nkeys, void* scratch, cudaStream_t s) {
    MuScratch t = mu_carve(scratch, n);
    const uint32_t n32 = static_cast<uint32_t>(n);
    const uint32_t ntiles = static_cast<uint32_t>((n + kTile - 1) / kTile);
    const unsigned grid = (unsigned)min_u64((n + 255) / 256, (uint64_t)num_sms() * 8);
    SBH_TIMED("mu_gather", s, mu_gather_kernel<kVals><<<grid, 256, 0, s>>>(ptrs, n32, col, t.v, t.idx));
    SBH_LAUNCHED();
    size_t sb = t.sort_bytes;
    int rc = sbh_kpa_sort(t.v, t.idx, t.v1, t.idx1, n, t.sort_scr, &sb, s);  // by value
    if (rc) return rc;
    SBH_TIMED("mu_keys", s, mu_keys_kernel<<<grid, 256, 0, s>>>(keys, t.idx1, n32, t.k2));
    SBH_LAUNCHED();
    sb = t.sort_bytes;
    rc = sbh_kpa_sort(t.k2, t.idx1, t.k3, t.idx3, n, t.sort_scr, &sb, s);  // then by key, stably
    if (rc) return rc;
    SBH_TIMED("mu_flags", s, mu_flags_kernel<<<grid, 256, 0, s>>>(t.k3, t.idx3, n32, t.v, t.w, t.f, t.iota));
    SBH_LAUNCHED();
    // distinct values per key: the keyed sum of the flags (also writes the keys)
    size_t rb = t.red_bytes;
    rc = sbh_group_reduce(t.k3, t.iota, n, t.f, 4, ok, t.counts, 8, ouni, cap, nkeys, t.red_scr, &rb, s);
    if (rc) return rc;
    // the runs of the re-ordered KPA, then each run's middle row
    SBH_CUDA(cudaMemsetAsync(t.small, 0, 2 * sizeof(uint32_t), s));
    SBH_TIMED("mu_heads_count", s, heads_count_kernel<<<ntiles, kThreads, 0, s>>>(t.k3, n32, t.tile_cnt));
    SBH_LAUNCHED();
    SBH_TIMED("mu_heads_scan", s,
              heads_scan_kernel<<<1, 1024, 0, s>>>(t.tile_cnt, ntiles, t.nseg, t.small, t.seg_start, n32));
    SBH_LAUNCHED();
    SBH_TIMED("mu_heads_emit", s,
              heads_emit_kernel<<<ntiles, kThreads, 0, s>>>(t.k3, n32, t.tile_cnt, nullptr, 0, t.seg_start));
    SBH_LAUNCHED();
    SBH_TIMED("mu_median", s, mu_median_kernel<<<grid, 256, 0, s>>>(t.seg_start, t.small, t.w, cap, omed));
    SBH_LAUNCHED();
    return SBH_OK;
}

}  // namespace
}  // namespace sbh

extern "C" {

int sbh_topk(const uint64_t* d_keys, const uint32_t* d_ptrs, uint64_t n, const void* d_val_col, int val_bytes,
             int K, uint64_t* d_out_keys, uint8_t* d_out_nvalid, uint64_t* d_out_vals, uint32_t* d_out_ptrs,
             uint64_t cap, uint64_t* d_nkeys, void* d_scratch, size_t* scratch_bytes, void* stream) {
    using namespace sbh;
    clear_error();
    if (K < 1 || K > SBH_TOPK_MAX_K) { set_error("K must be in [1, %d]", SBH_TOPK_MAX_K); return SBH_EINVAL; }
    if (n >= 0xFFFFFFFFull) { set_error("n must be < 2^32 - 1"); return SBH_EINVAL; }
    bool done = false;
    const size_t need = K <= 4 ? topk_carve<4>(nullptr, n).total : topk_carve<8>(nullptr, n).total;
    int rc = scratch_check(d_scratch, scratch_bytes, need, &done);
    if (rc || done) return rc;
    if (!d_nkeys) { set_error("d_nkeys is NULL"); return SBH_EINVAL; }
    cudaStream_t s = as_stream(stream);
    if (n == 0) {
        SBH_CUDA(cudaMemsetAsync(d_nkeys, 0, sizeof(uint64_t), s));
        return SBH_OK;
    }
    if (!d_keys || !d_ptrs || !d_val_col || (cap && (!d_out_keys || !d_out_nvalid || !d_out_vals || !d_out_ptrs))) {
        set_error("null pointer");
        return SBH_EINVAL;
    }
    if (val_bytes != 4 && val_bytes != 8) { set_error("val_bytes must be 4 or 8"); return SBH_EINVAL; }
    if (K <= 4)
        return topk_dispatch<4>(d_keys, d_ptrs, n, d_val_col, val_bytes, K, d_out_keys, d_out_nvalid, d_out_vals,
                                d_out_ptrs, cap, d_nkeys, d_scratch, s);
    return topk_dispatch<8>(d_keys, d_ptrs, n, d_val_col, val_bytes, K, d_out_keys, d_out_nvalid, d_out_vals,
                            d_out_ptrs, cap, d_nkeys, d_scratch, s);
}

int sbh_median_unique(const uint64_t* d_keys, const uint32_t* d_ptrs, uint64_t n, const void* d_val_col,
                      int val_bytes, uint64_t* d_out_keys, uint64_t* d_out_median, uint64_t* d_out_unique,
                      uint64_t cap, uint64_t* d_nkeys, void* d_scratch, size_t* scratch_bytes, void* stream) {
    using namespace sbh;
    clear_error();
    if (n >= 0xFFFFFFFFull) { set_error("n must be < 2^32 - 1"); return SBH_EINVAL; }
    bool done = false;
    int rc = scratch_check(d_scratch, scratch_bytes, mu_carve(nullptr, n).total, &done);
    if (rc || done) return rc;
    if (!d_nkeys) { set_error("d_nkeys is NULL"); return SBH_EINVAL; }
    cudaStream_t s = as_stream(stream);
    if (n == 0) {
        SBH_CUDA(cudaMemsetAsync(d_nkeys, 0, sizeof(uint64_t), s));
        return SBH_OK;
    }
    if (!d_keys || !d_ptrs || !d_val_col || (cap && (!d_out_keys || !d_out_median || !d_out_unique))) {
        set_error("null pointer");
        return SBH_EINVAL;
    }
    if (val_bytes != 4 && val_bytes != 8) { set_error("val_bytes must be 4 or 8"); return SBH_EINVAL; }
    if (val_bytes == 8)
        return mu_run<8>(d_keys, d_ptrs, n, d_val_col, d_out_keys, d_out_median, d_out_unique, cap, d_nkeys,
                         d_scratch, s);
    return mu_run<4>(d_keys, d_ptrs, n, d_val_col, d_out_keys, d_out_median, d_out_unique, cap, d_nkeys, d_scratch,
                     s);
}

}  // extern "C"
