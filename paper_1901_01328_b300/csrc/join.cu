// A8 Join of two KPAs sorted in (key, ptr) order: every (ptrL, ptrR) with
// equal keys, in (key, ptrL, ptrR) order.
//
//   count  each row i of L finds its key's row range [lo, hi) in R; a thread
//          takes kIpt consecutive rows of L, searches the first row's range
//          by bisection and every later row's by galloping on from the
//          previous row's range (the keys ascend, so a range starts where the
//          previous one ended; with the windows' key densities a step or
//          two); per-block sums of the match counts hi - lo.
//   scan   one block scans the block sums; the grand total is the pair count.
//   emit   each block rescans its rows' counts from its block offset; row i
//          writes (ptrL[i], ptrR[lo + j]) for j < hi - lo.  Rows of L come in
//          (key, ptrL) order and each R range in ptrR order, so the pairs come
//          out in (key, ptrL, ptrR) order.
#include "common.cuh"

namespace sbh {
namespace {

constexpr int kThreads = 256;
constexpr int kIpt = 8;
constexpr int kTile = kThreads * kIpt;

__device__ __forceinline__ uint32_t lower_bound_key(const uint64_t* a, uint32_t n, uint64_t v) {
    uint32_t lo = 0, hi = n;
    while (lo < hi) {
        const uint32_t mid = (lo + hi) / 2;
        if (a[mid] < v) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}
__device__ __forceinline__ uint32_t upper_bound_key(const uint64_t* a, uint32_t lo, uint32_t n, uint64_t v) {
    uint32_t hi = n;
    while (lo < hi) {
        const uint32_t mid = (lo + hi) / 2;
        if (a[mid] <= v) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

// First i in [from, n) with a[i] >= v (or > v when kUpper), for a sorted
// ascending and every a[i] with from <= i < the answer below (above) v:
// doubling steps, then bisection of the last step.
template <bool kUpper>
__device__ __forceinline__ uint32_t gallop(const uint64_t* a, uint32_t n, uint32_t from, uint64_t v) {
    uint32_t lo = from, hi = from, step = 1;
    while (hi < n && (kUpper ? a[hi] <= v : a[hi] < v)) {
        lo = hi + 1;
        hi = (n - hi > step) ? hi + step : n;
        step <<= 1;
    }
    while (lo < hi) {
        const uint32_t mid = (lo + hi) / 2;
        if (kUpper ? a[mid] <= v : a[mid] < v) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

// The R range [lo, hi) of every row of this thread's kIpt consecutive rows
// of one sorted L segment set (the single-window join: one segment).
// seg_of(i) returns the segment of row i; segments change only forward.
__device__ __forceinline__ uint64_t count_rows(const uint64_t* __restrict__ lk, uint32_t nl, uint32_t i0,
                                               const uint64_t* __restrict__ rk, const uint64_t* __restrict__ l_off,
                                               const uint64_t* __restrict__ r_start,
                                               const uint64_t* __restrict__ r_len, uint32_t nseg, uint32_t nr,
                                               uint32_t* __restrict__ rlo, uint32_t* __restrict__ cnt) {
    uint64_t local = 0;
    uint32_t a = 0, seg_end = 0, lo = 0, hi = 0, n = 0, rs = 0;
    const uint64_t* seg = rk;
    uint64_t prevk = 0;
    bool have = false;
#pragma unroll
    for (int t = 0; t < kIpt; ++t) {
        const uint32_t i = i0 + t;
        if (i >= nl) break;
        const uint64_t k = lk[i];
        if (!have || i >= seg_end) {  // the first row, or a row of a later segment
            if (l_off) {
                uint32_t x = have ? a : 0, y = nseg;  // last segment with l_off <= i
                while (y - x > 1) {
                    const uint32_t mid = (x + y) / 2;
                    if (l_off[mid] <= i) x = mid;
                    else y = mid;
                }
                a = x;
                seg_end = a + 1 < nseg ? static_cast<uint32_t>(l_off[a + 1]) : nl;
                rs = static_cast<uint32_t>(r_start[a]);
                n = static_cast<uint32_t>(r_len[a]);
            } else {
                seg_end = nl;
                rs = 0;
                n = nr;
            }
            seg = rk + rs;
            lo = lower_bound_key(seg, n, k);
            hi = upper_bound_key(seg, lo, n, k);
            have = true;
        } else if (k != prevk) {  // k > prevk: its range starts at or after hi
            lo = gallop<false>(seg, n, hi, k);
            hi = gallop<true>(seg, n, lo, k);
        }
        prevk = k;
        rlo[i] = rs + lo;
        cnt[i] = hi - lo;
        local += hi - lo;
    }
    return local;
}

__device__ __forceinline__ uint64_t block_sum(uint64_t v, uint64_t* red) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane_id() == 0) red[threadIdx.x / 32] = v;
    __syncthreads();
    uint64_t t = 0;
    for (int w = 0; w < kThreads / 32; ++w) t += red[w];
    return t;
}

__global__ void __launch_bounds__(kThreads)
join_count_kernel(const uint64_t* __restrict__ lk, uint32_t nl, const uint64_t* __restrict__ rk, uint32_t nr,
                  uint32_t* __restrict__ rlo, uint32_t* __restrict__ cnt, uint64_t* __restrict__ bsum) {
    __shared__ uint64_t red[kThreads / 32];
    const uint32_t base = blockIdx.x * kTile;
    const uint64_t local =
        count_rows(lk, nl, base + threadIdx.x * kIpt, rk, nullptr, nullptr, nullptr, 1, nr, rlo, cnt);
    const uint64_t t = block_sum(local, red);
    if (threadIdx.x == 0) bsum[blockIdx.x] = t;
}

// Exclusive scan of the block sums in place; *total receives the sum.
__global__ void __launch_bounds__(1024) scan_blocks_kernel(uint64_t* __restrict__ bsum, uint32_t nb,
                                                           uint64_t* __restrict__ total) {
    __shared__ uint64_t warp_tot[32];
    __shared__ uint64_t carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (uint32_t c0 = 0; c0 < nb; c0 += blockDim.x) {
        const uint32_t i = c0 + threadIdx.x;
        const uint64_t v = i < nb ? bsum[i] : 0;
        uint64_t x = v;
        for (int o = 1; o < 32; o <<= 1) {
            const uint64_t y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane_id() >= (uint32_t)o) x += y;
        }
        if (lane_id() == 31) warp_tot[threadIdx.x / 32] = x;
        __syncthreads();
        uint64_t before = carry;
        for (uint32_t w = 0; w < threadIdx.x / 32; ++w) before += warp_tot[w];
        if (i < nb) bsum[i] = before + x - v;
        __syncthreads();
        if (threadIdx.x == blockDim.x - 1) carry = before + x;
        __syncthreads();
    }
    if (threadIdx.x == 0) *total = carry;
}

__global__ void __launch_bounds__(kThreads)
join_emit_kernel(const uint32_t* __restrict__ lp, uint32_t nl, const uint32_t* __restrict__ rp,
                 const uint32_t* __restrict__ rlo, const uint32_t* __restrict__ cnt,
                 const uint64_t* __restrict__ boff, uint32_t* __restrict__ out_l, uint32_t* __restrict__ out_r,
                 uint64_t cap) {
    __shared__ uint64_t warp_tot[kThreads / 32];
    // thread-blocked rows: thread t owns rows base + t*kIpt .. + kIpt - 1
    const uint32_t base = blockIdx.x * kTile;
    const uint32_t first = base + threadIdx.x * kIpt;
    uint32_t c[kIpt];
    uint64_t mine = 0;
#pragma unroll
    for (int t = 0; t < kIpt; ++t) {
        c[t] = (first + t < nl) ? cnt[first + t] : 0u;
        mine += c[t];
    }
    uint64_t x = mine;
    for (int o = 1; o < 32; o <<= 1) {
        const uint64_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane_id() >= (uint32_t)o) x += y;
    }
    if (lane_id() == 31) warp_tot[threadIdx.x / 32] = x;
    __syncthreads();
    uint64_t off = boff[blockIdx.x];
    for (uint32_t w = 0; w < threadIdx.x / 32; ++w) off += warp_tot[w];
    off += x - mine;
#pragma unroll
    for (int t = 0; t < kIpt; ++t) {
        if (c[t]) {
            const uint32_t i = first + t;
            const uint32_t pl = lp[i];
            const uint32_t lo = rlo[i];
            for (uint32_t j = 0; j < c[t]; ++j) {
                const uint64_t o = off + j;
                if (o < cap) {
                    out_l[o] = pl;
                    out_r[o] = rp[lo + j];
                }
            }
            off += c[t];
        }
    }
}

// ---------------------------------------------------------------- many independent joins
// L rows [l_off[g], l_off[g + 1]) join R rows [r_start[g], r_start[g] +
// r_len[g]) (segment g).  Row i of L finds its segment by binary search on
// l_off, then its key's range in its R segment; rlo holds absolute R rows, so
// the emit kernel above serves unchanged.
__global__ void __launch_bounds__(kThreads)
join_seg_count_kernel(const uint64_t* __restrict__ lk, uint32_t nl, const uint64_t* __restrict__ rk,
                      const uint64_t* __restrict__ l_off, const uint64_t* __restrict__ r_start,
                      const uint64_t* __restrict__ r_len, uint32_t nseg, uint32_t* __restrict__ rlo,
                      uint32_t* __restrict__ cnt, uint64_t* __restrict__ bsum) {
    __shared__ uint64_t red[kThreads / 32];
    const uint32_t base = blockIdx.x * kTile;
    const uint64_t local =
        count_rows(lk, nl, base + threadIdx.x * kIpt, rk, l_off, r_start, r_len, nseg, 0, rlo, cnt);
    const uint64_t t = block_sum(local, red);
    if (threadIdx.x == 0) bsum[blockIdx.x] = t;
}

// seg_pairs[g] = the first output pair of segment g (the pairs of all L rows
// before l_off[g]), from the scanned block offsets and the counts of the
// rows before it in its block; one warp per segment; seg_pairs[nseg] = total.
__global__ void join_seg_offsets_kernel(const uint64_t* __restrict__ l_off, uint32_t nseg, uint32_t nl,
                                        const uint32_t* __restrict__ cnt, const uint64_t* __restrict__ boff,
                                        const uint64_t* __restrict__ total, uint64_t* __restrict__ seg_pairs) {
    const uint32_t g = blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
    if (g > nseg) return;
    const uint64_t row = g < nseg ? l_off[g] : nl;
    if (row >= nl) {
        if (lane_id() == 0) seg_pairs[g] = *total;
        return;
    }
    const uint32_t blk = static_cast<uint32_t>(row / kTile);
    uint64_t v = 0;
    for (uint32_t i = blk * kTile + lane_id(); i < row; i += 32) v += cnt[i];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane_id() == 0) seg_pairs[g] = boff[blk] + v;
}

}  // namespace
}  // namespace sbh

extern "C" int sbh_join_segments(int nseg, const uint64_t* d_lkeys, const uint32_t* d_lptrs, const uint64_t* l_off,
                                 const uint64_t* d_rkeys, const uint32_t* d_rptrs, const uint64_t* r_start,
                                 const uint64_t* r_len, uint32_t* d_out_l, uint32_t* d_out_r, uint64_t cap,
                                 uint64_t* d_npairs, uint64_t* d_seg_pairs, int reuse_counts, void* d_scratch,
                                 size_t* scratch_bytes, void* stream) {
    using namespace sbh;
    clear_error();
    if (nseg < 1 || !l_off || !r_start || !r_len) { set_error("bad segment arrays"); return SBH_EINVAL; }
    if (l_off[0] != 0) { set_error("l_off[0] must be 0"); return SBH_EINVAL; }
    for (int g = 0; g < nseg; ++g) {
        if (l_off[g + 1] < l_off[g]) { set_error("l_off must be non-decreasing"); return SBH_EINVAL; }
        if (r_start[g] + r_len[g] > 0xFFFFFFFFull) { set_error("segment %d of R reaches past 2^32 rows", g); return SBH_EINVAL; }
    }
    const uint64_t nl = l_off[nseg];
    if (nl > 0xFFFFFFFFull) { set_error("L must have < 2^32 rows"); return SBH_EINVAL; }
    const uint64_t nblocks = (nl + kTile - 1) / kTile;
    Carver c(nullptr);
    c.take<uint32_t>(nl);
    c.take<uint32_t>(nl);
    c.take<uint64_t>(nblocks + 1);
    c.take<uint64_t>(3 * (size_t)nseg + 1);
    bool done = false;
    int rc = scratch_check(d_scratch, scratch_bytes, c.bytes(), &done);
    if (rc || done) return rc;
    if (!d_npairs || !d_seg_pairs) { set_error("d_npairs or d_seg_pairs is NULL"); return SBH_EINVAL; }
    cudaStream_t s = as_stream(stream);
    if (nl == 0) {
        SBH_CUDA(cudaMemsetAsync(d_npairs, 0, sizeof(uint64_t), s));
        SBH_CUDA(cudaMemsetAsync(d_seg_pairs, 0, (nseg + 1) * sizeof(uint64_t), s));
        return SBH_OK;
    }
    if (!d_lkeys || !d_lptrs || !d_rkeys || !d_rptrs || (cap && (!d_out_l || !d_out_r))) {
        set_error("null pointer");
        return SBH_EINVAL;
    }
    Carver w(d_scratch);
    uint32_t* rlo = w.take<uint32_t>(nl);
    uint32_t* cnt = w.take<uint32_t>(nl);
    uint64_t* bsum = w.take<uint64_t>(nblocks + 1);
    uint64_t* segs = w.take<uint64_t>(3 * (size_t)nseg + 1);  // l_off (nseg + 1), r_start, r_len
    if (reuse_counts) {  // the counts, scanned offsets and totals of an earlier call are in the scratch
        if (cap) {
            SBH_TIMED("join_emit", s,
                      join_emit_kernel<<<(unsigned)nblocks, kThreads, 0, s>>>(d_lptrs, (uint32_t)nl, d_rptrs, rlo, cnt,
                                                                              bsum, d_out_l, d_out_r, cap));
            SBH_LAUNCHED();
        }
        return SBH_OK;
    }
    SBH_CUDA(cudaMemcpyAsync(segs, l_off, (nseg + 1) * sizeof(uint64_t), cudaMemcpyHostToDevice, s));
    SBH_CUDA(cudaMemcpyAsync(segs + nseg + 1, r_start, nseg * sizeof(uint64_t), cudaMemcpyHostToDevice, s));
    SBH_CUDA(cudaMemcpyAsync(segs + 2 * nseg + 1, r_len, nseg * sizeof(uint64_t), cudaMemcpyHostToDevice, s));
    SBH_TIMED("join_seg_count", s,
              join_seg_count_kernel<<<(unsigned)nblocks, kThreads, 0, s>>>(d_lkeys, (uint32_t)nl, d_rkeys, segs,
                                                                           segs + nseg + 1, segs + 2 * nseg + 1,
                                                                           (uint32_t)nseg, rlo, cnt, bsum));
    SBH_LAUNCHED();
    SBH_TIMED("join_scan", s, scan_blocks_kernel<<<1, 1024, 0, s>>>(bsum, (uint32_t)nblocks, d_npairs));
    SBH_LAUNCHED();
    SBH_TIMED("join_seg_offsets", s,
              join_seg_offsets_kernel<<<(unsigned)((nseg + 1 + 7) / 8), 256, 0, s>>>(segs, (uint32_t)nseg,
                                                                                    (uint32_t)nl, cnt, bsum, d_npairs,
                                                                                    d_seg_pairs));
    SBH_LAUNCHED();
    if (cap) {
        SBH_TIMED("join_emit", s,
                  join_emit_kernel<<<(unsigned)nblocks, kThreads, 0, s>>>(d_lptrs, (uint32_t)nl, d_rptrs, rlo, cnt,
                                                                          bsum, d_out_l, d_out_r, cap));
        SBH_LAUNCHED();
    }
    return SBH_OK;
}

extern "C" int sbh_join(const uint64_t* d_lkeys, const uint32_t* d_lptrs, uint64_t nl, const uint64_t* d_rkeys,
                        const uint32_t* d_rptrs, uint64_t nr, uint32_t* d_out_l, uint32_t* d_out_r, uint64_t cap,
                        uint64_t* d_npairs, void* d_scratch, size_t* scratch_bytes, void* stream) {
    using namespace sbh;
    clear_error();
    if (nl > 0xFFFFFFFFull || nr > 0xFFFFFFFFull) { set_error("inputs must be < 2^32 rows"); return SBH_EINVAL; }
    const uint64_t nblocks = (nl + kTile - 1) / kTile;
    Carver c(nullptr);
    c.take<uint32_t>(nl);
    c.take<uint32_t>(nl);
    c.take<uint64_t>(nblocks + 1);
    bool done = false;
    int rc = scratch_check(d_scratch, scratch_bytes, c.bytes(), &done);
    if (rc || done) return rc;
    if (!d_npairs) { set_error("d_npairs is NULL"); return SBH_EINVAL; }
    cudaStream_t s = as_stream(stream);
    if (nl == 0 || nr == 0) {
        SBH_CUDA(cudaMemsetAsync(d_npairs, 0, sizeof(uint64_t), s));
        return SBH_OK;
    }
    if (!d_lkeys || !d_lptrs || !d_rkeys || !d_rptrs || (cap && (!d_out_l || !d_out_r))) {
        set_error("null pointer");
        return SBH_EINVAL;
    }
    Carver w(d_scratch);
    uint32_t* rlo = w.take<uint32_t>(nl);
    uint32_t* cnt = w.take<uint32_t>(nl);
    uint64_t* bsum = w.take<uint64_t>(nblocks + 1);
    SBH_TIMED("join_count", s, join_count_kernel<<<(unsigned)nblocks, kThreads, 0, s>>>(d_lkeys, (uint32_t)nl, d_rkeys, (uint32_t)nr, rlo, cnt,
                                                              bsum));
    SBH_LAUNCHED();
    SBH_TIMED("join_scan", s, scan_blocks_kernel<<<1, 1024, 0, s>>>(bsum, (uint32_t)nblocks, d_npairs));
    SBH_LAUNCHED();
    SBH_TIMED("join_emit", s, join_emit_kernel<<<(unsigned)nblocks, kThreads, 0, s>>>(d_lptrs, (uint32_t)nl, d_rptrs, rlo, cnt, bsum, d_out_l,
                                                             d_out_r, cap));
    SBH_LAUNCHED();
    return SBH_OK;
}
