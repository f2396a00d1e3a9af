// Radix-pass machinery shared by the plain sort (radix_sort.cu) and the
// learned partition sort (learned.cu): every pass orders pairs (key, ptr) by
// one 8-bit digit of a value derived from the key (the key itself, or a
// bucket id), stably.
//
// Per sort:
//   upsweep   one read of the keys builds the 256-bin histogram of every
//             digit position of the value.
//   plan      exclusive scan of each histogram (global digit offsets); a
//             position whose digit is the same for every key is skipped; the
//             ping-pong buffer of each active pass is chosen so that the last
//             one writes the output.
//   passes    small sorts: one onesweep kernel per pass (persistent CTAs take
//             tiles in order from a counter, rank each tile with a warp
//             multisplit, and find their global offsets by decoupled
//             look-back over earlier tiles, with bounded waits).
//             Large sorts: each CTA owns one contiguous chunk of tiles;
//             count -> scan -> scatter kernels give every chunk its global
//             digit offsets up front, so no CTA ever waits on another and the
//             next tile of a chunk can be brought in by bulk copy (TMA) while
//             the current one is ranked and scattered.
//   copy      only when no pass ran (or an in-place sort ends in the
//             temporary buffer).
#pragma once

#include <cstdlib>
#include <string>
#include <type_traits>

#include "common.cuh"

namespace sbh {
namespace {


constexpr int kRadixBits = 8;
constexpr int kRadix = 1 << kRadixBits;
constexpr int kPositions = 64 / kRadixBits;
constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr int kIpt = 16;                    // keys per thread
constexpr int kTile = kThreads * kIpt;      // keys per tile

// look-back record: [63:62] flag, [61:56] epoch (pass + 1), [55:0] count
constexpr uint64_t kFlagAgg = 1ull << 62;
constexpr uint64_t kFlagPrefix = 2ull << 62;
constexpr uint64_t kValueMask = (1ull << 56) - 1;

struct Plan {
    int active[kPositions];
    int src[kPositions];  // 0 = input, 1 = temporary, 2 = output
    int dst[kPositions];
    int copy_src;         // -1 = no copy, else the buffer to copy to the output
    int npasses;
};

struct Buffers {
    const uint64_t* in_k;
    const uint32_t* in_p;
    uint64_t* tmp_k;
    uint32_t* tmp_p;
    uint64_t* out_k;
    uint32_t* out_p;
    // optional 16-bit values carried with the rows (the learned sort's bucket
    // ids); null when the digit comes from the key
    const uint16_t* in_v = nullptr;
    uint16_t* tmp_v = nullptr;
    uint16_t* out_v = nullptr;
    __device__ __forceinline__ const uint16_t* vals(int sel) const { return sel == 0 ? in_v : (sel == 1 ? tmp_v : out_v); }
    __device__ __forceinline__ uint16_t* wvals(int sel) const { return sel == 1 ? tmp_v : out_v; }
    __device__ __forceinline__ const uint64_t* keys(int sel) const { return sel == 0 ? in_k : (sel == 1 ? tmp_k : out_k); }
    __device__ __forceinline__ const uint32_t* ptrs(int sel) const { return sel == 0 ? in_p : (sel == 1 ? tmp_p : out_p); }
    __device__ __forceinline__ uint64_t* wkeys(int sel) const { return sel == 1 ? tmp_k : out_k; }
    __device__ __forceinline__ uint32_t* wptrs(int sel) const { return sel == 1 ? tmp_p : out_p; }
};

// ------------------------------------------------------------------ upsweep
// Equal digits in a row are counted in registers first: skewed keys (a heavy
// key, constant high bytes) would otherwise serialise on one bin.
struct RunCounter {
    uint32_t last[kPositions], run[kPositions];
    __device__ __forceinline__ RunCounter() {
#pragma unroll
        for (int p = 0; p < kPositions; ++p) { last[p] = 0; run[p] = 0; }
    }
    __device__ __forceinline__ void add(uint64_t k, uint32_t* h) {
#pragma unroll
        for (int p = 0; p < kPositions; ++p) {
            const uint32_t d = static_cast<uint32_t>(k >> (p * kRadixBits)) & (kRadix - 1);
            if (d == last[p]) {
                ++run[p];
            } else {
                if (run[p]) atomicAdd(&h[p * kRadix + last[p]], run[p]);
                last[p] = d;
                run[p] = 1;
            }
        }
    }
    __device__ __forceinline__ void flush(uint32_t* h) {
#pragma unroll
        for (int p = 0; p < kPositions; ++p)
            if (run[p]) atomicAdd(&h[p * kRadix + last[p]], run[p]);
    }
};

// Histogram of every digit position of value_of(key); positions at or above
// npos are counted as all-zero (constant, so their passes are skipped).
template <typename ValueFn>
__global__ void __launch_bounds__(256) upsweep_kernel(const uint64_t* __restrict__ keys, uint32_t n,
                                                      uint32_t* __restrict__ ghist, ValueFn value_of, int npos) {
    __shared__ uint32_t h[kPositions * kRadix];
    for (int i = threadIdx.x; i < kPositions * kRadix; i += blockDim.x) h[i] = 0;
    __syncthreads();
    RunCounter rc;
    const uint32_t nthreads = gridDim.x * blockDim.x;
    const uint32_t tid = blockIdx.x * blockDim.x + threadIdx.x;
    uint32_t done = 0;
    if ((reinterpret_cast<uintptr_t>(keys) & 15) == 0) {
        // four keys per step with two 16-byte loads issued together
        const uint32_t nq = n / 4;
        const ulonglong2* q = reinterpret_cast<const ulonglong2*>(keys);
        for (uint32_t i = tid; i < nq; i += nthreads) {
            const ulonglong2 a = __ldcs(q + 2 * i);
            const ulonglong2 b = __ldcs(q + 2 * i + 1);
            rc.add(value_of(a.x), h);
            rc.add(value_of(a.y), h);
            rc.add(value_of(b.x), h);
            rc.add(value_of(b.y), h);
        }
        done = nq * 4;
    }
    for (uint32_t i = done + tid; i < n; i += nthreads) rc.add(value_of(ld_stream(keys + i)), h);
    rc.flush(h);
    __syncthreads();
    for (int i = threadIdx.x; i < npos * kRadix; i += blockDim.x)
        if (h[i]) atomicAdd(&ghist[i], h[i]);
    if (blockIdx.x == 0 && threadIdx.x == 0)
        for (int p = npos; p < kPositions; ++p) atomicAdd(&ghist[p * kRadix], n);
}

// ------------------------------------------------------------------ plan
__global__ void __launch_bounds__(kRadix) plan_kernel(const uint32_t* __restrict__ ghist, uint32_t n,
                                                      uint32_t* __restrict__ gbase, Plan* __restrict__ plan,
                                                      int in_place) {
    __shared__ uint32_t warp_sums[kRadix / 32];
    __shared__ int s_active[kPositions];
    const int d = threadIdx.x;
    for (int p = 0; p < kPositions; ++p) {
        const uint32_t c = ghist[p * kRadix + d];
        const int constant = __syncthreads_or(c == n);
        // block exclusive scan of c over the 256 digits
        uint32_t x = c;
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane_id() >= (uint32_t)o) x += y;
        }
        if (lane_id() == 31) warp_sums[d / 32] = x;
        __syncthreads();
        uint32_t before = 0;
        for (int w = 0; w < d / 32; ++w) before += warp_sums[w];
        gbase[p * kRadix + d] = before + x - c;
        if (d == 0) s_active[p] = !constant;
        __syncthreads();
    }
    if (d == 0) {
        Plan pl;
        int a = 0;
        for (int p = 0; p < kPositions; ++p) a += s_active[p];
        int i = 0, prev = 0;
        for (int p = 0; p < kPositions; ++p) {
            pl.active[p] = s_active[p];
            pl.src[p] = pl.dst[p] = 0;
            if (!s_active[p]) continue;
            int dst;
            if (in_place) dst = (i % 2 == 0) ? 1 : 2;
            else dst = ((a - 1 - i) % 2 == 0) ? 2 : 1;
            pl.src[p] = (i == 0) ? 0 : prev;
            pl.dst[p] = dst;
            prev = dst;
            ++i;
        }
        if (a == 0) pl.copy_src = in_place ? -1 : 0;
        else pl.copy_src = (prev == 2) ? -1 : prev;
        pl.npasses = a;
        *plan = pl;
    }
}

// ------------------------------------------------------------------ onesweep
// The value whose 8-bit digits a sort pass orders by: the key itself for the
// plain radix sort.
struct RadixValue {
    __device__ __forceinline__ uint64_t operator()(uint64_t k) const { return k; }
};

template <typename ValueFn>
struct DigitOf {
    ValueFn value;
    int shift;
    __device__ __forceinline__ uint32_t operator()(uint64_t k) const {
        return static_cast<uint32_t>(value(k) >> shift) & (kRadix - 1);
    }
};

struct SortSmem {
    uint64_t keys[2][kTile];  // double-buffered input tiles, reused to stage
    uint32_t ptrs[2][kTile];  // the scatter in digit order
    uint32_t whist[kWarps][kRadix + 1];  // +1: sentinel digit of rows past the end
    uint32_t local_start[kRadix];
    uint32_t gbase_rel[kRadix];
    uint32_t scan_tmp[kWarps];
    uint32_t tile_of[2];
    uint64_t mbar[2];
};

// One pass of the stable LSD sort.  Persistent CTAs take tile ids in order
// from a counter.  Each CTA keeps two tiles in flight: while it ranks and
// scatters one, a bulk copy (TMA) brings the next one into shared memory.
template <typename ValueFn>
__global__ void __launch_bounds__(kThreads, 2)
onesweep_kernel(Buffers buf, uint32_t n, int pos, const Plan* __restrict__ plan, const uint32_t* __restrict__ gbase,
                uint64_t* __restrict__ lookback, uint32_t* __restrict__ tile_counter, uint32_t spin_limit,
                int skip_publish_tile0, uint32_t* __restrict__ status, ValueFn value_of, int bulk_ok) {
    const DigitOf<ValueFn> digit_of{value_of, pos * kRadixBits};
    if (!plan->active[pos]) return;
    const int src = plan->src[pos], dst = plan->dst[pos];
    const uint64_t* __restrict__ in_k = buf.keys(src);
    const uint32_t* __restrict__ in_p = buf.ptrs(src);
    uint64_t* __restrict__ out_k = buf.wkeys(dst);
    uint32_t* __restrict__ out_p = buf.wptrs(dst);
    const uint64_t epoch = static_cast<uint64_t>(pos + 1) << 56;
    const uint32_t ntiles = (n + kTile - 1) / kTile;
    const uint32_t nfull = n / kTile;  // tiles that are loaded with bulk copies (when bulk_ok)

    extern __shared__ __align__(128) unsigned char smem_raw[];
    SortSmem& sm = *reinterpret_cast<SortSmem*>(smem_raw);
    const uint32_t tid = threadIdx.x, lane = lane_id(), warp = tid / 32;

    auto issue = [&](int b, uint32_t t) {  // thread 0 only
        if (t < ntiles && bulk_ok && t < nfull) {
            mbar_expect_tx(&sm.mbar[b], kTile * (sizeof(uint64_t) + sizeof(uint32_t)));
            bulk_load(sm.keys[b], in_k + (size_t)t * kTile, kTile * sizeof(uint64_t), &sm.mbar[b]);
            bulk_load(sm.ptrs[b], in_p + (size_t)t * kTile, kTile * sizeof(uint32_t), &sm.mbar[b]);
        }
    };

    const uint32_t my_gbase = gbase[pos * kRadix + tid];  // global offset of digit tid
    uint32_t next_id = 0;
    if (tid == 0) {
        mbar_init(&sm.mbar[0], 1);
        mbar_init(&sm.mbar[1], 1);
        fence_mbar_init();
        for (int b = 0; b < 2; ++b) {
            const uint32_t t = atomicAdd(tile_counter + pos, 1u);
            sm.tile_of[b] = t;
            issue(b, t);
        }
        next_id = atomicAdd(tile_counter + pos, 1u);
    }
    __syncthreads();
    uint32_t phase[2] = {0u, 0u};

    for (uint32_t it = 0;; ++it) {
        const int b = it & 1;
        const uint32_t tile = sm.tile_of[b];
        if (tile >= ntiles) break;  // ids grow per CTA: the other buffer is past the end too
        const uint32_t base = tile * kTile;
        const uint32_t valid = min(n - base, (uint32_t)kTile);
        for (int i = tid; i < kWarps * (kRadix + 1); i += kThreads) (&sm.whist[0][0])[i] = 0;

        // ---- wait for the tile (bulk copy) or load it (ragged or unaligned)
        if (bulk_ok && tile < nfull) {
            uint32_t polls = 0;
            while (!mbar_try_wait(&sm.mbar[b], phase[b]))
                if (wait_expired(polls, spin_limit, status)) break;
            phase[b] ^= 1u;
        } else {
            for (uint32_t s = tid; s < valid; s += kThreads) {
                sm.keys[b][s] = ld_stream(in_k + base + s);
                sm.ptrs[b][s] = ld_stream(in_p + base + s);
            }
        }
        __syncthreads();

        // ---- registers (warp-striped: warp w owns 32*kIpt consecutive rows)
        uint64_t k[kIpt];
        uint32_t p[kIpt];
        const uint32_t wofs = warp * 32 * kIpt + lane;
#pragma unroll
        for (int j = 0; j < kIpt; ++j) {
            const uint32_t s = wofs + j * 32;
            k[j] = sm.keys[b][s];
            p[j] = sm.ptrs[b][s];
        }

        // ---- warp multisplit: rank of each key among equal digits of its warp.
        // The leader of each group of equal digits adds the group size to the
        // warp's counter; atomics of one warp to one address take effect in
        // issue order, so items keep their (item, lane) order.
        uint32_t rank[kIpt];
        const uint32_t lt = lanemask_lt();
#pragma unroll
        for (int j = 0; j < kIpt; ++j) {
            const uint32_t d = (wofs + j * 32 < valid) ? digit_of(k[j]) : kRadix;
            const uint32_t peers = __match_any_sync(0xffffffffu, d);
            const int leader = __ffs(peers) - 1;
            uint32_t c = 0;
            if ((int)lane == leader) c = atomicAdd(&sm.whist[warp][d], (uint32_t)__popc(peers));
            rank[j] = __popc(peers & lt) + __shfl_sync(0xffffffffu, c, leader);
        }
        __syncthreads();

        // ---- per digit (thread = digit): warp offsets, tile count, publish
        const uint32_t d = tid;
        uint32_t cnt = 0;
#pragma unroll
        for (int w = 0; w < kWarps; ++w) {
            const uint32_t c = sm.whist[w][d];
            sm.whist[w][d] = cnt;
            cnt += c;
        }
        // Records carry their value in the same word, so relaxed accesses
        // suffice: no other data is published through them.
        uint64_t* rec = lookback + (uint64_t)tile * kRadix + d;
        if (!(skip_publish_tile0 && tile == 0)) st_relaxed(rec, (tile == 0 ? kFlagPrefix : kFlagAgg) | epoch | cnt);

        uint32_t x = cnt;  // block exclusive scan of the tile counts over digits
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= (uint32_t)o) x += y;
        }
        if (lane == 31) sm.scan_tmp[warp] = x;

        uint64_t excl = 0;  // decoupled look-back over earlier tiles (bounded)
        if (tile > 0) {
            uint32_t t = tile - 1;
            uint32_t polls = 0;
            for (;;) {
                const uint64_t r = ld_relaxed(lookback + (uint64_t)t * kRadix + d);
                if ((r & (3ull << 62)) == 0 || (r & (63ull << 56)) != epoch) {
                    if (wait_expired(polls, spin_limit, status)) break;
                    continue;
                }
                excl += r & kValueMask;
                if ((r & (3ull << 62)) == kFlagPrefix || t == 0) break;
                --t;
            }
            st_relaxed(rec, kFlagPrefix | epoch | ((excl + cnt) & kValueMask));
        }
        __syncthreads();
        uint32_t before = 0;
#pragma unroll
        for (int w = 0; w < kWarps; ++w) before += (w < (int)warp) ? sm.scan_tmp[w] : 0u;
        const uint32_t lstart = before + x - cnt;
        sm.local_start[d] = lstart;
        sm.gbase_rel[d] = my_gbase + static_cast<uint32_t>(excl) - lstart;
        __syncthreads();

        // ---- stage keys and ptrs in digit order (the tile's own buffer)
#pragma unroll
        for (int j = 0; j < kIpt; ++j) {
            if (wofs + j * 32 < valid) {
                const uint32_t dj = digit_of(k[j]);
                const uint32_t slot = sm.local_start[dj] + sm.whist[warp][dj] + rank[j];
                sm.keys[b][slot] = k[j];
                sm.ptrs[b][slot] = p[j];
            }
        }
        __syncthreads();
        // ---- scatter: consecutive slots of one digit go to consecutive rows
#pragma unroll
        for (int j = 0; j < kIpt; ++j) {
            const uint32_t s = tid + j * kThreads;
            if (s < valid) {
                const uint64_t kk = sm.keys[b][s];
                const uint32_t g = sm.gbase_rel[digit_of(kk)] + s;
                if (g < n) {  // false only after an expired wait
                    out_k[g] = kk;
                    out_p[g] = sm.ptrs[b][s];
                }
            }
        }
        __syncthreads();  // the buffer is free again
        if (tid == 0) {
            fence_proxy_async_smem();
            sm.tile_of[b] = next_id;
            issue(b, next_id);
            next_id = atomicAdd(tile_counter + pos, 1u);
        }
    }
}

// ------------------------------------------------------------------ copy
__global__ void copy_kernel(Buffers buf, uint32_t n, const Plan* __restrict__ plan) {
    const int sel = plan->copy_src;
    if (sel < 0) return;
    const uint64_t* __restrict__ sk = buf.keys(sel);
    const uint32_t* __restrict__ sp = buf.ptrs(sel);
    const uint32_t stride = gridDim.x * blockDim.x;
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        buf.out_k[i] = sk[i];
        buf.out_p[i] = sp[i];
    }
}

// Lanes of the warp whose digit equals this lane's, from one ballot per digit
// bit (digits below 2^nbits).
template <int kBits>
__device__ __forceinline__ uint32_t warp_peers(uint32_t d) {
    uint32_t peers = 0xffffffffu;
#pragma unroll
    for (int bit = 0; bit < kBits; ++bit) {
        const uint32_t on = (d >> bit) & 1u;
        const uint32_t bal = __ballot_sync(0xffffffffu, on);
        peers &= on ? bal : ~bal;
    }
    return peers;
}

// ------------------------------------------------------------------ chunked passes
constexpr uint32_t kMaxChunks = 1024;
constexpr uint64_t kChunkedMinRows = 1u << 21;  // below this the onesweep kernel is used

// Digit histogram of each chunk.
template <typename ValueFn>
__global__ void __launch_bounds__(1024)
chunk_count_kernel(Buffers buf, uint32_t n, int pos, const Plan* __restrict__ plan, uint32_t chunk,
                   uint32_t* __restrict__ chunk_hist, ValueFn value_of) {
    if (!plan->active[pos]) return;
    __shared__ uint32_t h[kRadix];
    const DigitOf<ValueFn> digit_of{value_of, pos * kRadixBits};
    const uint64_t* __restrict__ in_k = buf.keys(plan->src[pos]);
    for (int i = threadIdx.x; i < kRadix; i += blockDim.x) h[i] = 0;
    __syncthreads();
    const uint32_t lo = blockIdx.x * chunk;
    const uint32_t hi = min(n, lo + chunk);
    uint32_t last = 0, run = 0;
    auto add = [&](uint64_t k) {
        const uint32_t d = digit_of(k);
        if (d == last) {
            ++run;
        } else {
            if (run) atomicAdd(&h[last], run);
            last = d;
            run = 1;
        }
    };
    uint32_t done = lo;
    if (lo < hi && (reinterpret_cast<uintptr_t>(in_k + lo) & 15) == 0) {
        const uint32_t nq = (hi - lo) / 4;
        const ulonglong2* q = reinterpret_cast<const ulonglong2*>(in_k + lo);
        for (uint32_t i = threadIdx.x; i < nq; i += blockDim.x) {
            const ulonglong2 a = __ldcs(q + 2 * i);
            const ulonglong2 b = __ldcs(q + 2 * i + 1);
            add(a.x);
            add(a.y);
            add(b.x);
            add(b.y);
        }
        done = lo + nq * 4;
    }
    for (uint32_t i = done + threadIdx.x; i < hi; i += blockDim.x) add(ld_stream(in_k + i));
    if (run) atomicAdd(&h[last], run);
    __syncthreads();
    for (int i = threadIdx.x; i < kRadix; i += blockDim.x) chunk_hist[blockIdx.x * kRadix + i] = h[i];
}

// Global offset of every (chunk, digit): the digit's global base plus the
// counts of that digit in earlier chunks.  1024 threads: digit = tid % 256,
// one of four chunk groups = tid / 256.
__global__ void __launch_bounds__(1024)
chunk_scan_kernel(const Plan* __restrict__ plan, int pos, const uint32_t* __restrict__ chunk_hist, uint32_t nchunks,
                  const uint32_t* __restrict__ gbase, uint32_t* __restrict__ chunk_base) {
    if (!plan->active[pos]) return;
    __shared__ uint32_t gsum[4][kRadix];
    const uint32_t d = threadIdx.x & (kRadix - 1), g = threadIdx.x / kRadix;
    const uint32_t per = (nchunks + 3) / 4;
    const uint32_t c0 = min(nchunks, g * per), c1 = min(nchunks, c0 + per);
    uint32_t s = 0;
#pragma unroll 8
    for (uint32_t c = c0; c < c1; ++c) s += chunk_hist[c * kRadix + d];
    gsum[g][d] = s;
    __syncthreads();
    uint32_t run = gbase[pos * kRadix + d];
    for (uint32_t gg = 0; gg < g; ++gg) run += gsum[gg][d];
#pragma unroll 8
    for (uint32_t c = c0; c < c1; ++c) {
        const uint32_t v = chunk_hist[c * kRadix + d];
        chunk_base[c * kRadix + d] = run;
        run += v;
    }
}

// Ranks and scatters one chunk, tile by tile, with running digit offsets.
// 512 threads x 8 rows per tile: twice the warps of the onesweep kernel for
// the same tile, to hide the latency of the ranking chain.
constexpr int kSThreads = 512;
constexpr int kSWarps = kSThreads / 32;

template <int TILE, bool kCarry>
struct ScatterSmem {
    using Tag = typename std::conditional<kCarry, uint16_t, uint8_t>::type;
    uint64_t keys[2][TILE];  // double-buffered input tiles, reused to stage
    uint32_t ptrs[2][TILE];  // the scatter in digit order
    uint16_t vals[kCarry ? 2 : 1][kCarry ? TILE : 8];  // carried values of the input tiles
    Tag dig[TILE];           // digit (or carried value) of each staged row
    // per-warp digit counts, two 16-bit counters per word (digits 2w, 2w+1;
    // word 128 holds the sentinel digit of rows past the end)
    uint32_t whist2[kSWarps][kRadix / 2 + 1];
    uint16_t local_start[kRadix];
    uint32_t gbase_rel[kRadix];
    uint32_t scan_tmp[4];
    uint64_t mbar[2];
};

template <typename ValueFn, int TILE, bool kCarry = false>
__global__ void __launch_bounds__(kSThreads, TILE <= 4096 ? 2 : 1)
chunk_scatter_kernel(Buffers buf, uint32_t n, int pos, const Plan* __restrict__ plan, uint32_t chunk,
                     const uint32_t* __restrict__ chunk_base, ValueFn value_of, int bulk_ok, uint32_t spin_limit,
                     uint32_t* __restrict__ status) {
    if (!plan->active[pos]) return;
    const DigitOf<ValueFn> digit_of{value_of, pos * kRadixBits};
    const int src = plan->src[pos], dst = plan->dst[pos];
    const uint64_t* __restrict__ in_k = buf.keys(src);
    const uint32_t* __restrict__ in_p = buf.ptrs(src);
    uint64_t* __restrict__ out_k = buf.wkeys(dst);
    uint32_t* __restrict__ out_p = buf.wptrs(dst);
    const uint16_t* __restrict__ in_v = kCarry ? buf.vals(src) : nullptr;
    uint16_t* __restrict__ out_v = kCarry ? buf.wvals(dst) : nullptr;
    const uint32_t lo = blockIdx.x * chunk;
    const uint32_t hi = min(n, lo + chunk);
    if (lo >= hi) return;
    const uint32_t ntl = (hi - lo + TILE - 1) / TILE;

    extern __shared__ __align__(128) unsigned char smem_raw[];
    ScatterSmem<TILE, kCarry>& sm = *reinterpret_cast<ScatterSmem<TILE, kCarry>*>(smem_raw);
    constexpr int kSIpt = TILE / kSThreads;
    const uint32_t tid = threadIdx.x, lane = lane_id(), warp = tid / 32;
    // thread t < 128 carries the next output rows of digits 2t and 2t + 1
    uint32_t run0 = 0, run1 = 0;
    if (tid < kRadix / 2) {
        run0 = chunk_base[blockIdx.x * kRadix + 2 * tid];
        run1 = chunk_base[blockIdx.x * kRadix + 2 * tid + 1];
    }

    auto bulk_tile = [&](uint32_t i) { return bulk_ok && lo + (i + 1) * TILE <= hi; };
    auto issue = [&](int b, uint32_t i) {  // thread 0 only
        if (i < ntl && bulk_tile(i)) {
            mbar_expect_tx(&sm.mbar[b], TILE * (sizeof(uint64_t) + sizeof(uint32_t) + (kCarry ? sizeof(uint16_t) : 0)));
            bulk_load(sm.keys[b], in_k + lo + (size_t)i * TILE, TILE * sizeof(uint64_t), &sm.mbar[b]);
            bulk_load(sm.ptrs[b], in_p + lo + (size_t)i * TILE, TILE * sizeof(uint32_t), &sm.mbar[b]);
            if (kCarry) bulk_load(sm.vals[b], in_v + lo + (size_t)i * TILE, TILE * sizeof(uint16_t), &sm.mbar[b]);
        }
    };
    if (tid == 0) {
        mbar_init(&sm.mbar[0], 1);
        mbar_init(&sm.mbar[1], 1);
        fence_mbar_init();
        issue(0, 0);
        issue(1, 1);
    }
    __syncthreads();
    uint32_t phase[2] = {0u, 0u};

    for (uint32_t i = 0; i < ntl; ++i) {
        const int b = i & 1;
        const uint32_t base = lo + i * TILE;
        const uint32_t valid = min(hi - base, (uint32_t)TILE);
        for (int x = tid; x < kSWarps * (kRadix / 2 + 1); x += kSThreads) (&sm.whist2[0][0])[x] = 0;
        bool expired = false;
        if (bulk_tile(i)) {
            uint32_t polls = 0;
            while (!mbar_try_wait(&sm.mbar[b], phase[b]))
                if (wait_expired(polls, spin_limit, status)) {
                    expired = true;
                    break;
                }
            phase[b] ^= 1u;
        } else {
            for (uint32_t s = tid; s < valid; s += kSThreads) {
                sm.keys[b][s] = ld_stream(in_k + base + s);
                sm.ptrs[b][s] = ld_stream(in_p + base + s);
                if (kCarry) sm.vals[b][s] = in_v[base + s];
            }
        }
        // a tile whose data never arrived is not scattered (its rows stay unwritten)
        const bool tile_ok = !__syncthreads_or(expired);

        // rows of this thread: warp w owns 32 * kSIpt consecutive rows
        uint64_t k[kSIpt];
        uint32_t p[kSIpt], dg[kSIpt], rank[kSIpt], cv[kSIpt];
        const uint32_t wofs = warp * 32 * kSIpt + lane;
        const bool full = valid == (uint32_t)TILE;
        if (kCarry) {
#pragma unroll
            for (int j = 0; j < kSIpt; ++j) cv[j] = sm.vals[b][wofs + j * 32];
        }
#pragma unroll
        for (int j = 0; j < kSIpt; ++j) {
            k[j] = sm.keys[b][wofs + j * 32];
            p[j] = sm.ptrs[b][wofs + j * 32];
            if (kCarry) dg[j] = (full || wofs + j * 32 < valid) ? (cv[j] >> (pos * kRadixBits)) & (kRadix - 1) : kRadix;
            else dg[j] = (full || wofs + j * 32 < valid) ? digit_of(k[j]) : kRadix;
        }
        // warp multisplit (see onesweep_kernel): the peers of a row come from
        // digit-bit ballots (a ninth bit when the tile has rows past the end);
        // the group leader's counter update is predicated, not branched
        const uint32_t lt = lanemask_lt();
        if (full) {
            // half the items find their peers with match.any, half with digit
            // ballots: the two run on different pipes, so neither saturates
#pragma unroll
            for (int j = 0; j < kSIpt; ++j) {
                const uint32_t peers =
                    (j & 1) ? __match_any_sync(0xffffffffu, dg[j]) : warp_peers<kRadixBits>(dg[j]);
                const int leader = __ffs(peers) - 1;
                const uint32_t sh = (dg[j] & 1u) * 16u;
                const uint32_t c = smem_atomic_add_if((int)lane == leader, &sm.whist2[warp][dg[j] >> 1],
                                                      (uint32_t)__popc(peers) << sh);
                rank[j] = __popc(peers & lt) + ((__shfl_sync(0xffffffffu, c, leader) >> sh) & 0xFFFFu);
            }
        } else {
#pragma unroll
            for (int j = 0; j < kSIpt; ++j) {
                const uint32_t peers = warp_peers<kRadixBits + 1>(dg[j]);
                const int leader = __ffs(peers) - 1;
                const uint32_t sh = (dg[j] & 1u) * 16u;
                const uint32_t c = smem_atomic_add_if((int)lane == leader, &sm.whist2[warp][dg[j] >> 1],
                                                      (uint32_t)__popc(peers) << sh);
                rank[j] = __popc(peers & lt) + ((__shfl_sync(0xffffffffu, c, leader) >> sh) & 0xFFFFu);
            }
        }
        __syncthreads();

        // per digit pair (threads 0..127): warp offsets, tile counts, local starts
        uint32_t c0 = 0, c1 = 0, x = 0;
        if (tid < kRadix / 2) {
#pragma unroll
            for (int w = 0; w < kSWarps; ++w) {
                const uint32_t word = sm.whist2[w][tid];
                sm.whist2[w][tid] = c0 | (c1 << 16);
                c0 += word & 0xFFFFu;
                c1 += word >> 16;
            }
            x = c0 + c1;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
                if (lane >= (uint32_t)o) x += y;
            }
            if (lane == 31) sm.scan_tmp[warp] = x;
        }
        __syncthreads();
        if (tid < kRadix / 2) {
            uint32_t before = 0;
#pragma unroll
            for (int w = 0; w < 4; ++w) before += (w < (int)warp) ? sm.scan_tmp[w] : 0u;
            const uint32_t l0 = before + x - c0 - c1, l1 = l0 + c0;
            sm.local_start[2 * tid] = l0;
            sm.local_start[2 * tid + 1] = l1;
            sm.gbase_rel[2 * tid] = run0 - l0;
            sm.gbase_rel[2 * tid + 1] = run1 - l1;
            run0 += c0;
            run1 += c1;
        }
        __syncthreads();

        if (full) {
#pragma unroll
            for (int j = 0; j < kSIpt; ++j) {
                const uint32_t wo = (sm.whist2[warp][dg[j] >> 1] >> ((dg[j] & 1u) * 16u)) & 0xFFFFu;
                const uint32_t slot = sm.local_start[dg[j]] + wo + rank[j];
                sm.keys[b][slot] = k[j];
                sm.ptrs[b][slot] = p[j];
                sm.dig[slot] = static_cast<typename ScatterSmem<TILE, kCarry>::Tag>(kCarry ? cv[j] : dg[j]);
            }
        } else {
#pragma unroll
            for (int j = 0; j < kSIpt; ++j) {
                if (dg[j] < kRadix) {
                    const uint32_t wo = (sm.whist2[warp][dg[j] >> 1] >> ((dg[j] & 1u) * 16u)) & 0xFFFFu;
                    const uint32_t slot = sm.local_start[dg[j]] + wo + rank[j];
                    sm.keys[b][slot] = k[j];
                    sm.ptrs[b][slot] = p[j];
                    sm.dig[slot] = static_cast<typename ScatterSmem<TILE, kCarry>::Tag>(kCarry ? cv[j] : dg[j]);
                }
            }
        }
        __syncthreads();
        auto digit_at = [&](uint32_t s) -> uint32_t {
            return kCarry ? (static_cast<uint32_t>(sm.dig[s]) >> (pos * kRadixBits)) & (kRadix - 1) : sm.dig[s];
        };
        if (tile_ok && full) {
#pragma unroll
            for (int j = 0; j < kSIpt; ++j) {
                const uint32_t s = tid + j * kSThreads;
                const uint32_t g = sm.gbase_rel[digit_at(s)] + s;
                out_k[g] = sm.keys[b][s];
                out_p[g] = sm.ptrs[b][s];
                if (kCarry) out_v[g] = sm.dig[s];
            }
        } else if (tile_ok) {
#pragma unroll
            for (int j = 0; j < kSIpt; ++j) {
                const uint32_t s = tid + j * kSThreads;
                if (s < valid) {
                    const uint32_t g = sm.gbase_rel[digit_at(s)] + s;
                    out_k[g] = sm.keys[b][s];
                    out_p[g] = sm.ptrs[b][s];
                    if (kCarry) out_v[g] = sm.dig[s];
                }
            }
        }
        __syncthreads();
        if (tid == 0) {
            fence_proxy_async_smem();
            issue(b, i + 2);
        }
    }
}

// ------------------------------------------------------------------ scratch and launch
struct SortScratch {
    uint64_t* tmp_k;
    uint32_t* tmp_p;
    uint32_t* gbase;       // kPositions * kRadix
    Plan* plan;
    uint32_t* chunk_hist;  // kMaxChunks * kRadix
    uint32_t* chunk_base;  // kMaxChunks * kRadix
    uint32_t* hist;        // kPositions * kRadix   (zeroed)
    uint32_t* counters;    // kPositions            (zeroed)
    uint64_t* lookback;    // ntiles * kRadix       (zeroed; onesweep only)
    char* zero_begin;
    size_t zero_bytes;
    size_t total;
};

inline SortScratch sort_carve(void* scratch, uint64_t n) {
    Carver c(scratch);
    SortScratch s;
    const bool chunked = n >= kChunkedMinRows;
    const uint64_t ntiles = (n + kTile - 1) / kTile;
    s.tmp_k = c.take<uint64_t>(n);
    s.tmp_p = c.take<uint32_t>(n);
    s.gbase = c.take<uint32_t>(kPositions * kRadix);
    s.plan = c.take<Plan>(1);
    s.chunk_hist = c.take<uint32_t>(kMaxChunks * kRadix);
    s.chunk_base = c.take<uint32_t>(kMaxChunks * kRadix);
    s.hist = c.take<uint32_t>(kPositions * kRadix);
    const size_t zb = c.off - kPositions * kRadix * sizeof(uint32_t);
    s.counters = c.take<uint32_t>(kPositions);
    s.lookback = chunked ? nullptr : c.take<uint64_t>(ntiles * kRadix);
    s.zero_begin = reinterpret_cast<char*>(s.hist);
    s.zero_bytes = c.off - zb;
    s.total = c.bytes();
    return s;
}

// Stable sort of (in_k, in_p) by value_of(key) into (out_k, out_p); the
// positions at or above npos of the value are treated as zero.
template <typename ValueFn>
int sort_by_value(const uint64_t* in_k, const uint32_t* in_p, uint64_t* out_k, uint32_t* out_p, uint64_t n,
                  void* scratch, cudaStream_t s, ValueFn value_of, int npos, const char* tag = "sort") {
    // profile names: <tag>_upsweep, <tag>_scatter, ...
    const std::string t(tag);
    const std::string n_up = t + "_upsweep", n_plan = t + "_plan", n_count = t + "_count", n_scan = t + "_chunk_scan",
                      n_scat = t + "_scatter", n_one = t + "_onesweep", n_copy = t + "_copy";
    if (n == 0) return SBH_OK;
    const int in_place = (in_k == out_k);
    if (in_place != (in_p == out_p)) {
        set_error("an in-place sort needs both keys and ptrs aliased");
        return SBH_EINVAL;
    }
    SortScratch sc = sort_carve(scratch, n);
    SBH_CUDA(cudaMemsetAsync(sc.zero_begin, 0, sc.zero_bytes, s));
    const int sms = num_sms();
    const uint32_t n32 = static_cast<uint32_t>(n);
    const unsigned up_blocks = (unsigned)min_u64((n + 1023) / 1024, (uint64_t)sms * 8);
    SBH_TIMED(n_up.c_str(), s, upsweep_kernel<ValueFn><<<up_blocks, 256, 0, s>>>(in_k, n32, sc.hist, value_of, npos));
    SBH_LAUNCHED();
    SBH_TIMED(n_plan.c_str(), s, plan_kernel<<<1, kRadix, 0, s>>>(sc.hist, n32, sc.gbase, sc.plan, in_place));
    SBH_LAUNCHED();
    Buffers b{in_k, in_p, sc.tmp_k, sc.tmp_p, out_k, out_p};
    const size_t smem = sizeof(SortSmem);
    const uint32_t limit = spin_limit();
    uint32_t* status = status_word();
    // bulk copies need 16-byte aligned tile starts in every buffer a pass may read
    const int bulk_ok = ((reinterpret_cast<uintptr_t>(in_k) | reinterpret_cast<uintptr_t>(in_p) |
                          reinterpret_cast<uintptr_t>(out_k) | reinterpret_cast<uintptr_t>(out_p)) & 15) == 0;
    const uint64_t ntiles = (n + kTile - 1) / kTile;
    if (n >= kChunkedMinRows) {
        // scatter tile: 4096 rows (two CTAs per SM) or, with SBH_SCATTER_TILE=8192, 8192 rows (one CTA per SM)
        static const int tile_rows = [] {
            const char* e = getenv("SBH_SCATTER_TILE");
            return (e && atoi(e) == 8192) ? 8192 : 4096;
        }();
        auto scat = tile_rows == 8192 ? chunk_scatter_kernel<ValueFn, 8192> : chunk_scatter_kernel<ValueFn, 4096>;
        const size_t ssmem = tile_rows == 8192 ? sizeof(ScatterSmem<8192, false>) : sizeof(ScatterSmem<4096, false>);
        SBH_CUDA(cudaFuncSetAttribute(scat, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ssmem));
        int per_sm = 0;
        SBH_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, scat, kSThreads, ssmem));
        if (per_sm < 1) per_sm = 1;
        const uint64_t want = min_u64(min_u64(ntiles, (uint64_t)sms * per_sm), kMaxChunks);
        const uint64_t ttiles = (n + tile_rows - 1) / tile_rows;
        const uint32_t chunk = (uint32_t)(((ttiles + want - 1) / want) * tile_rows);
        const uint32_t nchunks = (uint32_t)((n + chunk - 1) / chunk);
        for (int pos = 0; pos < kPositions; ++pos) {
            SBH_TIMED(n_count.c_str(), s,
                      chunk_count_kernel<ValueFn><<<nchunks, 1024, 0, s>>>(b, n32, pos, sc.plan, chunk, sc.chunk_hist,
                                                                          value_of));
            SBH_LAUNCHED();
            SBH_TIMED(n_scan.c_str(), s,
                      chunk_scan_kernel<<<1, 1024, 0, s>>>(sc.plan, pos, sc.chunk_hist, nchunks, sc.gbase,
                                                           sc.chunk_base));
            SBH_LAUNCHED();
            SBH_TIMED(n_scat.c_str(), s,
                      scat<<<nchunks, kSThreads, ssmem, s>>>(b, n32, pos, sc.plan, chunk, sc.chunk_base, value_of,
                                                           bulk_ok, limit, status));
            SBH_LAUNCHED();
        }
    } else {
        auto kern = onesweep_kernel<ValueFn>;
        SBH_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        int per_sm = 0;
        SBH_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kThreads, smem));
        if (per_sm < 1) per_sm = 1;
        const unsigned grid = (unsigned)min_u64(ntiles, (uint64_t)sms * per_sm);
        const int fault = take_fault();
        for (int pos = 0; pos < kPositions; ++pos) {
            SBH_TIMED(n_one.c_str(), s,
                      kern<<<grid, kThreads, smem, s>>>(b, n32, pos, sc.plan, sc.gbase, sc.lookback, sc.counters, limit,
                                                        fault == SBH_FAULT_SKIP_PUBLISH ? 1 : 0, status, value_of,
                                                        bulk_ok));
            SBH_LAUNCHED();
        }
    }
    const unsigned cblocks = (unsigned)min_u64((n + 255) / 256, (uint64_t)sms * 4);
    SBH_TIMED(n_copy.c_str(), s, copy_kernel<<<cblocks, 256, 0, s>>>(b, n32, sc.plan));
    SBH_LAUNCHED();
    return SBH_OK;
}

}  // namespace
}  // namespace sbh
