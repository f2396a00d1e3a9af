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
constexpr int kLookWidth = 4;  // look-back records read at once

struct Plan {
    int active[kPositions];
    int src[kPositions];  // 0 = input, 1 = temporary, 2 = output
    int dst[kPositions];
    int copy_src;         // -1 = no copy, else the buffer to copy to the output
    int npasses;
};

struct Buffers {
    const uint64_t* in_k;
    const uint32_t* in_p;  // null: input row i's ptr is i (a key column sorted without an extract)
    uint64_t* tmp_k;
    uint32_t* tmp_p;
    uint64_t* out_k;
    uint32_t* out_p;
    // the learned sort's 16-bit bucket ids of the input rows, and the bytes
    // carried with the rows between its two passes (the ids' high bytes);
    // null otherwise
    const uint16_t* in_ids = nullptr;
    const uint8_t* in_v = nullptr;
    uint8_t* tmp_v = nullptr;
    uint8_t* out_v = nullptr;
    // a plain key sort's chunked passes: each row's digit of the next active
    // pass, stored by a scatter pass at the row's output position so that the
    // next pass's chunk counts read one byte a row instead of the key; null
    // otherwise
    uint8_t* nd = nullptr;
    __device__ __forceinline__ const uint8_t* vals(int sel) const { return sel == 0 ? in_v : (sel == 1 ? tmp_v : out_v); }
    __device__ __forceinline__ uint8_t* wvals(int sel) const { return sel == 1 ? tmp_v : out_v; }
    __device__ __forceinline__ const uint64_t* keys(int sel) const { return sel == 0 ? in_k : (sel == 1 ? tmp_k : out_k); }
    __device__ __forceinline__ const uint32_t* ptrs(int sel) const { return sel == 0 ? in_p : (sel == 1 ? tmp_p : out_p); }
    __device__ __forceinline__ uint64_t* wkeys(int sel) const { return sel == 1 ? tmp_k : out_k; }
    __device__ __forceinline__ uint32_t* wptrs(int sel) const { return sel == 1 ? tmp_p : out_p; }
};

// A sort whose size is known only on the device (the learned sort's overflow
// rows): the chunked kernels read n from d_n and derive the chunk geometry
// from it, the same way the host does for a known size, with G the number of
// chunks launched for the largest size the caller allows.  d_n == nullptr:
// the size and geometry are the launch arguments.
// Both the onesweep and the chunked kernels are queued for such a sort; each
// returns at once unless the size selects its path (chunked from thr pairs).
struct DynN {
    const uint32_t* d_n = nullptr;
    uint32_t G = 0;
    uint32_t tile = 0;
    uint32_t thr = 0;
    __device__ __forceinline__ bool skip(bool chunked_path) const {
        return d_n && ((*d_n >= thr) != chunked_path);
    }
    __device__ __forceinline__ void apply(uint32_t& n, uint32_t& chunk, uint32_t& nchunks) const {
        if (!d_n) return;
        n = *d_n;
        const uint32_t ttiles = (n + tile - 1) / tile;
        const uint32_t want = min(ttiles, G);
        chunk = want ? ((ttiles + want - 1) / want) * tile : tile;
        nchunks = (n + chunk - 1) / chunk;
    }
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
                                                      uint32_t* __restrict__ ghist, ValueFn value_of, int npos,
                                                      DynN dn = DynN{}) {
    if (dn.skip(false)) return;
    if (dn.d_n) n = *dn.d_n;
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

// First pass of the chunked passes: CTA c counts the first digit of its
// chunk's values and folds the values into two words, the OR of the values
// and the OR of their complements (both zeroed beforehand): a digit position
// is constant when no bit of it is set in both.
template <typename ValueFn>
__global__ void __launch_bounds__(1024)
first_count_kernel(const uint64_t* __restrict__ keys, uint32_t n, uint32_t chunk, ValueFn value_of,
                   uint32_t* __restrict__ chunk_hist, unsigned long long* __restrict__ vbits, DynN dn = DynN{}) {
    if (dn.skip(true)) return;
    __shared__ uint32_t h[kRadix];
    uint32_t nchunks = gridDim.x;
    dn.apply(n, chunk, nchunks);
    if (blockIdx.x >= nchunks) return;
    __shared__ unsigned long long wor[32], wnot[32];
    for (int i = threadIdx.x; i < kRadix; i += blockDim.x) h[i] = 0;
    __syncthreads();
    const uint32_t lo = blockIdx.x * chunk, hi = min(n, lo + chunk);
    unsigned long long vor = 0, vnot = 0;
    uint32_t last = 0, run = 0;
    auto add = [&](uint64_t k) {
        const uint64_t v = value_of(k);
        vor |= v;
        vnot |= ~v;
        const uint32_t d = static_cast<uint32_t>(v) & (kRadix - 1);
        if (d == last) {
            ++run;
        } else {
            if (run) atomicAdd(&h[last], run);
            last = d;
            run = 1;
        }
    };
    uint32_t done = lo;
    if (lo < hi && (reinterpret_cast<uintptr_t>(keys + lo) & 15) == 0) {
        const uint32_t nq = (hi - lo) / 4;
        const ulonglong2* q = reinterpret_cast<const ulonglong2*>(keys + lo);
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
    for (uint32_t i = done + threadIdx.x; i < hi; i += blockDim.x) add(ld_stream(keys + i));
    if (run) atomicAdd(&h[last], run);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        vor |= __shfl_xor_sync(0xffffffffu, vor, o);
        vnot |= __shfl_xor_sync(0xffffffffu, vnot, o);
    }
    if (lane_id() == 0) {
        wor[threadIdx.x / 32] = vor;
        wnot[threadIdx.x / 32] = vnot;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < kRadix; i += blockDim.x) chunk_hist[blockIdx.x * kRadix + i] = h[i];
    if (threadIdx.x == 0) {
        for (uint32_t w = 1; w < blockDim.x / 32; ++w) {
            vor |= wor[w];
            vnot |= wnot[w];
        }
        atomicOr(&vbits[0], vor);
        atomicOr(&vbits[1], vnot);
    }
}

// The pass plan from the value bits: a pass is active when its digit is not
// constant (a bit of it set in some value and clear in another).
__device__ void fill_plan(const int* active, int in_place, Plan* __restrict__ plan) {
    Plan pl;
    int a = 0;
    for (int p = 0; p < kPositions; ++p) a += active[p];
    int i = 0, prev = 0;
    for (int p = 0; p < kPositions; ++p) {
        pl.active[p] = active[p];
        pl.src[p] = pl.dst[p] = 0;
        if (!active[p]) continue;
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

__global__ void plan_bits_kernel(const unsigned long long* __restrict__ vbits, int npos, Plan* __restrict__ plan,
                                 int in_place, DynN dn = DynN{}) {
    if (threadIdx.x != 0 || dn.skip(true)) return;
    const unsigned long long varying = vbits[0] & vbits[1];
    int active[kPositions];
    for (int p = 0; p < kPositions; ++p) active[p] = p < npos && ((varying >> (p * kRadixBits)) & (kRadix - 1)) != 0;
    fill_plan(active, in_place, plan);
}

// ------------------------------------------------------------------ plan
__global__ void __launch_bounds__(kRadix) plan_kernel(const uint32_t* __restrict__ ghist, uint32_t n,
                                                      uint32_t* __restrict__ gbase, Plan* __restrict__ plan,
                                                      int in_place, DynN dn = DynN{}) {
    if (dn.skip(false)) return;
    if (dn.d_n) n = *dn.d_n;
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
    if (d == 0) fill_plan(s_active, in_place, plan);
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
                int skip_publish_tile0, uint32_t* __restrict__ status, ValueFn value_of, int bulk_ok,
                DynN dn = DynN{}) {
    const DigitOf<ValueFn> digit_of{value_of, pos * kRadixBits};
    if (dn.skip(false)) return;
    if (dn.d_n) n = *dn.d_n;
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
            mbar_expect_tx(&sm.mbar[b], kTile * (sizeof(uint64_t) + (in_p ? sizeof(uint32_t) : 0)));
            bulk_load(sm.keys[b], in_k + (size_t)t * kTile, kTile * sizeof(uint64_t), &sm.mbar[b]);
            if (in_p) bulk_load(sm.ptrs[b], in_p + (size_t)t * kTile, kTile * sizeof(uint32_t), &sm.mbar[b]);
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
        bool expired = false;
        const uint32_t par = phase[b];
        if (bulk_ok && tile < nfull) {
            expired = !mbar_wait_bounded(&sm.mbar[b], par, spin_limit, status);
            phase[b] ^= 1u;
        } else {
            for (uint32_t s = tid; s < valid; s += kThreads) {
                sm.keys[b][s] = ld_stream(in_k + base + s);
                if (in_p) sm.ptrs[b][s] = ld_stream(in_p + base + s);
            }
        }
        if (__syncthreads_or(expired)) {
            // the tile's copy did not arrive within the budget: issue nothing
            // more, let both buffers' copies land, and leave (the tiles after
            // this one find no record and their bounded waits give up)
            mbar_drain(&sm.mbar[b], par);
            if (bulk_ok && sm.tile_of[b ^ 1] < nfull) mbar_drain(&sm.mbar[b ^ 1], phase[b ^ 1]);
            break;
        }

        // ---- registers (warp-striped: warp w owns 32*kIpt consecutive rows)
        uint64_t k[kIpt];
        uint32_t p[kIpt];
        const uint32_t wofs = warp * 32 * kIpt + lane;
#pragma unroll
        for (int j = 0; j < kIpt; ++j) {
            const uint32_t s = wofs + j * 32;
            k[j] = sm.keys[b][s];
            p[j] = in_p ? sm.ptrs[b][s] : base + s;
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

        // decoupled look-back over earlier tiles (bounded): the records of
        // four earlier tiles are read at once and taken in order, summing
        // aggregates until an inclusive prefix (tile 0 always publishes one);
        // a record not yet published is read again
        uint64_t excl = 0;
        if (tile > 0) {
            uint32_t t = tile - 1;
            uint32_t polls = 0;
            for (bool done = false; !done;) {
                uint64_t r[kLookWidth];
#pragma unroll
                for (int u = 0; u < kLookWidth; ++u)
                    r[u] = t >= (uint32_t)u ? ld_relaxed(lookback + (uint64_t)(t - u) * kRadix + d) : 0ull;
                int u = 0;
#pragma unroll
                for (; u < kLookWidth; ++u) {
                    if ((r[u] & (3ull << 62)) == 0 || (r[u] & (63ull << 56)) != epoch) break;
                    excl += r[u] & kValueMask;
                    if ((r[u] & (3ull << 62)) == kFlagPrefix || t == (uint32_t)u) {
                        done = true;
                        break;
                    }
                }
                if (done) break;
                t -= u;  // every record before t is an aggregate taken; t is not published yet
                if (u < kLookWidth && wait_expired(polls, spin_limit, status)) break;
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
__global__ void copy_kernel(Buffers buf, uint32_t n, const Plan* __restrict__ plan,
                            const uint32_t* __restrict__ d_n = nullptr) {
    const int sel = plan->copy_src;
    if (sel < 0) return;
    if (d_n) n = *d_n;
    const uint64_t* __restrict__ sk = buf.keys(sel);
    const uint32_t* __restrict__ sp = buf.ptrs(sel);
    const uint32_t stride = gridDim.x * blockDim.x;
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        buf.out_k[i] = sk[i];
        buf.out_p[i] = sp ? sp[i] : i;
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
// sorts of at least knob(SBH_KNOB_SORT_CHUNKED_MIN) pairs (default 2^23) take
// the chunked passes, smaller ones the onesweep kernel
inline bool use_chunked(uint64_t n) { return n >= knob(SBH_KNOB_SORT_CHUNKED_MIN); }

// Digit histogram of rows [lo, hi) from their digit bytes (1024 threads;
// the rows' data 16-byte aligned at lo), 32 bytes a thread per step.  Lane l
// adds to column l of a [digit][lane] table: the 32 atomics of a warp fall in
// 32 banks and never on one counter, whatever the digits (a run of one
// digit included).  For 256M rows of the mixed keys: 0.056 ms a pass, against
// 0.100 with runs of one digit counted in registers first (the lanes'
// branches diverge), 0.086 with a 256-bin table per warp and 0.140 with four
// tables shared by the warps.  kHi16: the rows hold 16-bit values and the
// digit is their high byte.
template <bool kHi16 = false>
__device__ __forceinline__ void nd_count(const void* __restrict__ src, uint32_t lo, uint32_t hi,
                                         uint32_t* __restrict__ out) {
    __shared__ uint32_t h[kRadix][32];
    for (int i = threadIdx.x; i < kRadix * 32; i += blockDim.x) (&h[0][0])[i] = 0;
    __syncthreads();
    const uint32_t lane = lane_id();
    auto add = [&](uint32_t d) { atomicAdd(&h[d][lane], 1u); };
    auto add4 = [&](uint32_t w) {  // the digits of the rows in one 32-bit word
        if constexpr (kHi16) {
            add((w >> 8) & 0xFFu);
            add(w >> 24);
        } else {
#pragma unroll
            for (int b = 0; b < 4; ++b) add((w >> (8 * b)) & 0xFFu);
        }
    };
    constexpr uint32_t kRowBytes = kHi16 ? 2 : 1;
    const char* __restrict__ base = static_cast<const char*>(src) + (size_t)lo * kRowBytes;
    const uint32_t nv = lo < hi ? (hi - lo) * kRowBytes / 32 : 0;
    const uint4* __restrict__ v = reinterpret_cast<const uint4*>(base);
    for (uint32_t i = threadIdx.x; i < nv; i += blockDim.x) {
        const uint4 a = __ldcs(v + 2 * i);
        const uint4 b = __ldcs(v + 2 * i + 1);
        add4(a.x); add4(a.y); add4(a.z); add4(a.w);
        add4(b.x); add4(b.y); add4(b.z); add4(b.w);
    }
    for (uint32_t i = lo + nv * 32 / kRowBytes + threadIdx.x; i < hi; i += blockDim.x) {
        if constexpr (kHi16) add(static_cast<const uint16_t*>(src)[i] >> 8);
        else add(static_cast<const uint8_t*>(src)[i]);
    }
    __syncthreads();
    // digit d's 32 columns: one warp per digit, a lane per column
    const uint32_t warp = threadIdx.x / 32;
    for (uint32_t d = warp; d < (uint32_t)kRadix; d += blockDim.x / 32) {
        uint32_t c = h[d][lane];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
        if (lane == 0) out[d] = c;
    }
}

// Digit histogram of each chunk.
template <typename ValueFn>
__global__ void __launch_bounds__(1024)
chunk_count_kernel(Buffers buf, uint32_t n, int pos, const Plan* __restrict__ plan, uint32_t chunk,
                   uint32_t* __restrict__ chunk_hist, ValueFn value_of, DynN dn = DynN{}) {
    if (dn.skip(true) || !plan->active[pos]) return;
    uint32_t nchunks = gridDim.x;
    dn.apply(n, chunk, nchunks);
    if (blockIdx.x >= nchunks) return;
    __shared__ uint32_t h[kRadix];
    const uint32_t lo = blockIdx.x * chunk;
    const uint32_t hi = min(n, lo + chunk);
    if constexpr (std::is_same<ValueFn, RadixValue>::value) {
        // an earlier pass ran: its scatter left this pass's digits in nd
        bool from_nd = false;
        if (buf.nd)
            for (int q = 0; q < pos; ++q) from_nd |= plan->active[q] != 0;
        if (from_nd) {
            nd_count(buf.nd, lo, hi, chunk_hist + (size_t)blockIdx.x * kRadix);
            return;
        }
    }
    const DigitOf<ValueFn> digit_of{value_of, pos * kRadixBits};
    const uint64_t* __restrict__ in_k = buf.keys(plan->src[pos]);
    for (int i = threadIdx.x; i < kRadix; i += blockDim.x) h[i] = 0;
    __syncthreads();
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
// one of four chunk groups = tid / 256.  The digit bases come from gbase, or,
// when it is null, from the chunk counts themselves (their digit totals,
// scanned).
__global__ void __launch_bounds__(1024)
chunk_scan_kernel(const Plan* __restrict__ plan, int pos, const uint32_t* __restrict__ chunk_hist, uint32_t nchunks,
                  const uint32_t* __restrict__ gbase, uint32_t* __restrict__ chunk_base, DynN dn = DynN{}) {
    if (dn.skip(true) || !plan->active[pos]) return;
    {
        uint32_t n = 0, chunk = 0;
        dn.apply(n, chunk, nchunks);
    }
    __shared__ uint32_t gsum[4][kRadix];
    __shared__ uint32_t base[kRadix];
    __shared__ uint32_t wsum[kRadix / 32];
    const uint32_t d = threadIdx.x & (kRadix - 1), g = threadIdx.x / kRadix;
    const uint32_t per = (nchunks + 3) / 4;
    const uint32_t c0 = min(nchunks, g * per), c1 = min(nchunks, c0 + per);
    uint32_t s = 0;
#pragma unroll 8
    for (uint32_t c = c0; c < c1; ++c) s += chunk_hist[c * kRadix + d];
    gsum[g][d] = s;
    __syncthreads();
    if (!gbase) {
        if (g == 0) {  // exclusive scan of the digit totals
            const uint32_t t = gsum[0][d] + gsum[1][d] + gsum[2][d] + gsum[3][d];
            uint32_t x = t;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
                if (lane_id() >= (uint32_t)o) x += y;
            }
            if (lane_id() == 31) wsum[d / 32] = x;
            base[d] = x - t;
        }
        __syncthreads();
    }
    uint32_t run;
    if (gbase) {
        run = gbase[pos * kRadix + d];
    } else {
        run = base[d];
        for (uint32_t w = 0; w < d / 32; ++w) run += wsum[w];
    }
    for (uint32_t gg = 0; gg < g; ++gg) run += gsum[gg][d];
#pragma unroll 8
    for (uint32_t c = c0; c < c1; ++c) {
        const uint32_t v = chunk_hist[c * kRadix + d];
        chunk_base[c * kRadix + d] = run;
        run += v;
    }
}

// Ranks and scatters one chunk, tile by tile, with running digit offsets.
// THREADS x (TILE / THREADS) rows per tile; five CTA barriers per tile:
//   B0  tile data present (bulk copy complete); the other buffer is free, so
//       the next tile's copy is issued
//   B1  ranked: per-warp digit counts final
//   B2  per warp group: exclusive counts over the group's warps, group totals
//   B3  per (group, digit): first staged slot; per digit: global offset
//   B4  staged in digit order; then the coalesced scatter (and the counters
//       are cleared for the next tile)
template <int TILE, int THREADS, bool kCarry, bool kDig, bool kIdx = false>
struct ScatterSmem {
    static constexpr int kW = THREADS / 32;
    static constexpr int kG = THREADS / 128;  // warp groups of the count scan
    uint64_t keys[2][TILE];  // double-buffered input tiles, reused to stage
    uint32_t ptrs[kIdx ? 1 : 2][kIdx ? 4 : TILE];  // the scatter in digit order
    uint16_t idx[kIdx ? TILE : 8];  // kIdx (ptr = row number): each staged row's place in its tile
    uint16_t vals[kCarry ? 2 : 1][kCarry ? TILE : 8];  // carried ids, staged the same way (the second
                                                       // pass's carried bytes arrive in the first TILE bytes)
    uint8_t dig[kDig ? TILE : 16];                     // digit of each staged row (derived values only)
    // per-warp digit counts, two 16-bit counters per word (digits 2w, 2w+1;
    // word 128 holds the sentinel digit of rows past the end)
    uint32_t whist2[kW][kRadix / 2 + 1];
    uint32_t gsum[kG][kRadix / 2];   // per warp group, packed digit-pair totals
    uint16_t gstart[kG][kRadix];     // first staged slot of each (group, digit)
    uint32_t run[kRadix];            // next output row of each digit in this chunk
    uint32_t gbase_rel[kRadix];      // output row minus staged slot, per digit
    uint32_t lw[kCarry ? 4 : 1];     // low-byte walk: digit so far, next digit start, tile's first digit,
                                     // digit starts inside the tile (listed in gsum until B1)
    uint64_t mbar[2];
};

// The digit of a staged row is re-derived from its key when the value is
// the key itself; other values keep it in shared memory.
template <typename ValueFn, bool kCarry>
struct ScatterDig {
    static constexpr bool value = !kCarry && !std::is_same<ValueFn, RadixValue>::value;
};

template <int TILE, int THREADS>
struct ScatterBlocks {  // CTAs per SM the launch bounds ask for (64 registers a thread at most)
    static constexpr int value = TILE * 12 * 2 > 120 * 1024 ? 1 : 65536 / (THREADS * 64);
};

// rows j of a thread (j % 8) whose peers come from match.any, the others from
// digit ballots: one in two measured fastest (the two run on different pipes)
constexpr uint32_t kMatchMask = 0xAA;
// kIdx: the pass reads the sort's input with no ptrs (ptrs_in NULL: a row's
// ptr is its row number), so no ptrs are loaded and the staging keeps each
// row's 16-bit place in its tile instead of a 4-byte ptr.  The learned sort
// launches it for its first carried-id pass over a key column, whose tiles
// then fit 4096 rows instead of 3584 (the two id passes at 256M rows 4.75 to
// 4.61 ms); for the plain sort's first pass it measured no faster.
template <typename ValueFn, int TILE, int THREADS, bool kCarry = false, bool kIdx = false>
__global__ void __launch_bounds__(THREADS, (ScatterBlocks<TILE, THREADS>::value))
chunk_scatter_kernel(Buffers buf, uint32_t n, int pos, const Plan* __restrict__ plan, uint32_t chunk,
                     const uint32_t* __restrict__ chunk_base, ValueFn value_of, int bulk_ok, uint32_t spin_limit,
                     uint32_t* __restrict__ status, uint32_t* __restrict__ first_row = nullptr,
                     const uint32_t* __restrict__ low_base = nullptr, DynN dn = DynN{}) {
    constexpr bool kDig = ScatterDig<ValueFn, kCarry>::value;
    constexpr bool kNext = !kCarry && std::is_same<ValueFn, RadixValue>::value;
    using Smem = ScatterSmem<TILE, THREADS, kCarry, kDig, kIdx>;
    constexpr int kW = Smem::kW, kG = Smem::kG, kWpg = kW / kG;
    constexpr int kIt = TILE / THREADS;
    static_assert(TILE % THREADS == 0 && THREADS % 128 == 0 && THREADS <= 1024, "tile geometry");
    static_assert(TILE < 65536, "16-bit counters");
    if (dn.skip(true) || !plan->active[pos]) return;
    const int shift = pos * kRadixBits;
    const DigitOf<ValueFn> digit_of{value_of, shift};
    const int src = plan->src[pos], dst = plan->dst[pos];
    const uint64_t* __restrict__ in_k = buf.keys(src);
    const uint32_t* __restrict__ in_p = kIdx ? nullptr : buf.ptrs(src);
    uint64_t* __restrict__ out_k = buf.wkeys(dst);
    uint32_t* __restrict__ out_p = buf.wptrs(dst);
    // Carried 16-bit ids (kCarry: two passes, low byte then high byte).  The
    // first pass reads each input row's id (in_ids) and writes the id's high
    // byte with the row.  The second orders by that byte and recovers the low
    // byte from the row's position: the first pass left the rows grouped by
    // low byte, rows [low_base[d], low_base[d + 1]) holding low byte d
    // (low_base = the first pass's digit bases).  A second pass after no
    // first one reads the input ids too.
    const bool full_ids = kCarry && (pos == 0 || !plan->active[0]);
    const bool walk = kCarry && !full_ids;
    // Last of the passes, first_row given: the ids are not written out;
    // instead every id's first output row is recorded (atomicMin into
    // first_row[id]).  A staged tile of the last pass is in id order, so a
    // row whose id differs from the staged row before it is the first of its
    // id in this tile.
    const bool rows_pass = kCarry && first_row != nullptr && (pos == 1 || !plan->active[1]);
    const uint16_t* __restrict__ in_ids = full_ids ? buf.in_ids : nullptr;
    const uint8_t* __restrict__ in_v = walk ? buf.vals(src) : nullptr;
    uint8_t* __restrict__ out_v = (kCarry && !rows_pass) ? buf.wvals(dst) : nullptr;
    // the next active pass, whose digit each row leaves in nd (none: -1)
    int nxt = -1;
    if constexpr (kNext) {
        if (buf.nd)
            for (int q = kPositions - 1; q > pos; --q)
                if (plan->active[q]) nxt = q;
    }
    {
        uint32_t nchunks = gridDim.x;
        dn.apply(n, chunk, nchunks);
    }
    const uint32_t lo = blockIdx.x * chunk;
    const uint32_t hi = min(n, lo + chunk);
    if (lo >= hi) return;
    const uint32_t ntl = (hi - lo + TILE - 1) / TILE;

    extern __shared__ __align__(128) unsigned char smem_raw[];
    Smem& sm = *reinterpret_cast<Smem*>(smem_raw);
    const uint32_t tid = threadIdx.x, lane = lane_id(), warp = tid / 32;

    auto bulk_tile = [&](uint32_t i) { return bulk_ok && lo + (i + 1) * TILE <= hi; };
    auto issue = [&](int b, uint32_t i) {  // thread 0 only
        if (i < ntl && bulk_tile(i)) {
            mbar_expect_tx(&sm.mbar[b], TILE * (sizeof(uint64_t) + (in_p ? sizeof(uint32_t) : 0)) +
                                            (full_ids ? TILE * sizeof(uint16_t) : (walk ? TILE : 0)));
            // a plain pass's tiles are read once: evict-first keeps the L2 for
            // the output runs whose last sector the next tile completes
            // (14.22 against 14.34 ms for eight passes at 256M rows); the
            // carried-id passes keep the default (evict-first was no faster)
            if constexpr (kCarry) {
                bulk_load(sm.keys[b], in_k + lo + (size_t)i * TILE, TILE * sizeof(uint64_t), &sm.mbar[b]);
                if constexpr (!kIdx)
                    if (in_p) bulk_load(sm.ptrs[b], in_p + lo + (size_t)i * TILE, TILE * sizeof(uint32_t), &sm.mbar[b]);
            } else {
                const uint64_t pol = l2_evict_first();
                bulk_load(sm.keys[b], in_k + lo + (size_t)i * TILE, TILE * sizeof(uint64_t), &sm.mbar[b], pol);
                if constexpr (!kIdx)
                    if (in_p)
                        bulk_load(sm.ptrs[b], in_p + lo + (size_t)i * TILE, TILE * sizeof(uint32_t), &sm.mbar[b], pol);
            }
            if (full_ids) bulk_load(sm.vals[b], in_ids + lo + (size_t)i * TILE, TILE * sizeof(uint16_t), &sm.mbar[b]);
            if (walk) bulk_load(sm.vals[b], in_v + lo + (size_t)i * TILE, TILE, &sm.mbar[b]);
        }
    };
    for (int x = tid; x < kW * (kRadix / 2 + 1); x += THREADS) (&sm.whist2[0][0])[x] = 0;
    for (int x = tid; x < kRadix; x += THREADS) sm.run[x] = chunk_base[blockIdx.x * kRadix + x];
    // buffers with a bulk copy in flight (bit b), the same in every thread
    uint32_t inflight = (bulk_tile(0) ? 1u : 0u) | ((ntl > 1 && bulk_tile(1)) ? 2u : 0u);
    if (tid == 0) {
        mbar_init(&sm.mbar[0], 1);
        mbar_init(&sm.mbar[1], 1);
        fence_mbar_init();
        issue(0, 0);
        issue(1, 1);
        if (walk) {
            sm.lw[0] = 0;  // low_base[0] = 0: every position is in digit 0 or later
            sm.lw[1] = low_base[1];
        }
    }
    __syncthreads();
    uint32_t phase[2] = {0u, 0u};

    for (uint32_t i = 0; i < ntl; ++i) {
        const int b = i & 1;
        const uint32_t base = lo + i * TILE;
        const uint32_t valid = min(hi - base, (uint32_t)TILE);
        if constexpr (kCarry) {
            // warp 0: the low byte of the tile's first row (d0) and the digit
            // starts inside the tile (m of them, ascending), walking on from
            // the previous tile; a start at or before base moves d0 on
            if (walk && warp == 0) {
                const uint32_t tend = base + valid - 1;
                const uint32_t c = sm.lw[0];
                uint32_t d0 = c, m = 0;
                if (sm.lw[1] <= tend) {
                    uint32_t* list = &sm.gsum[0][0];
                    uint32_t nb = 0, na = 0, after = 0xFFFFFFFFu;
                    for (uint32_t d = c + 1; d < (uint32_t)kRadix; d += 32) {
                        const uint32_t v = d + lane < (uint32_t)kRadix ? low_base[d + lane] : 0xFFFFFFFFu;
                        const uint32_t cb = __popc(__ballot_sync(0xffffffffu, v <= base));
                        const uint32_t ca = __popc(__ballot_sync(0xffffffffu, v <= tend));
                        nb += cb;  // final once a lane of this group starts past base
                        if (v > base && v <= tend) list[d - c - 1 + lane - nb] = v;
                        na += ca;
                        if (ca < 32) {
                            after = __shfl_sync(0xffffffffu, v, ca);
                            break;
                        }
                    }
                    d0 = c + nb;
                    m = na - nb;
                    if (lane == 0) {
                        sm.lw[0] = c + na;  // the digit of the tile's last row
                        sm.lw[1] = after;   // and where the next one starts
                    }
                }
                if (lane == 0) {
                    sm.lw[2] = d0;
                    sm.lw[3] = m;
                }
            }
        }
        bool expired = false;
        const uint32_t par = phase[b];
        if (bulk_tile(i)) {
            expired = !mbar_wait_bounded(&sm.mbar[b], par, spin_limit, status);
            phase[b] ^= 1u;
        } else {
            for (uint32_t s = tid; s < valid; s += THREADS) {
                sm.keys[b][s] = ld_stream(in_k + base + s);
                if constexpr (!kIdx)
                    if (in_p) sm.ptrs[b][s] = ld_stream(in_p + base + s);
                if (full_ids) sm.vals[b][s] = in_ids[base + s];
                if (walk) reinterpret_cast<uint8_t*>(sm.vals[b])[s] = in_v[base + s];
            }
        }
        // B0.  A tile whose data did not arrive within the budget ends the
        // chunk: no copy is issued any more, the copies in flight are let
        // land, and the rows not scattered stay unwritten (the call's output
        // is invalid and the timeout is recorded).  Otherwise tile i - 1 is
        // done with the other buffer, which takes tile i + 1.
        if (__syncthreads_or(expired)) {
            mbar_drain(&sm.mbar[b], par);
            if (inflight & (2u >> b)) mbar_drain(&sm.mbar[b ^ 1], phase[b ^ 1]);
            return;
        }
        inflight &= ~(1u << b);
        if (i >= 1 && i + 1 < ntl && bulk_tile(i + 1)) inflight |= 2u >> b;
        if (tid == 0 && i >= 1) {
            fence_proxy_async_smem();
            issue(b ^ 1, i + 1);
        }

        // the tile body, compiled separately for full tiles (no per-row
        // bounds) and for the ragged last tile
        auto tile = [&](auto full_tag) {
            constexpr bool full = decltype(full_tag)::value;
            uint64_t* __restrict__ kb = sm.keys[b];
            uint32_t* __restrict__ pb = sm.ptrs[kIdx ? 0 : b];
            uint16_t* __restrict__ vb = sm.vals[kCarry ? b : 0];
            // rows of this thread: warp w owns 32 * kIt consecutive rows
            uint64_t k[kIt];
            uint32_t p[kIt], dg[kIt], rank[kIt], cv[kIt];
            const uint32_t wofs = warp * 32 * kIt + lane;
#pragma unroll
            for (int j = 0; j < kIt; ++j) {
                k[j] = kb[wofs + j * 32];
                if constexpr (kIdx) p[j] = wofs + j * 32;  // the row's place in the tile
                else p[j] = in_p ? pb[wofs + j * 32] : base + wofs + j * 32;
                if (kCarry) cv[j] = walk ? reinterpret_cast<const uint8_t*>(vb)[wofs + j * 32] : vb[wofs + j * 32];
            }
            if constexpr (kCarry) {
                if (walk) {
                    const uint32_t d0 = sm.lw[2], m = sm.lw[3];
                    if (m == 0) {  // the usual case: one low byte for the whole tile
#pragma unroll
                        for (int j = 0; j < kIt; ++j) cv[j] = (cv[j] << 8) | d0;
                    } else {
                        const uint32_t* list = &sm.gsum[0][0];
#pragma unroll
                        for (int j = 0; j < kIt; ++j) {
                            if (full || wofs + j * 32 < valid) {  // low byte: d0 + the digit starts up to this row
                                const uint32_t row = base + wofs + j * 32;
                                uint32_t a = 0, z = m;
                                while (a < z) {
                                    const uint32_t mid = (a + z) >> 1;
                                    if (list[mid] <= row) a = mid + 1;
                                    else z = mid;
                                }
                                cv[j] = (cv[j] << 8) | (d0 + a);
                            }
                        }
                    }
                }
            }
#pragma unroll
            for (int j = 0; j < kIt; ++j) {
                const bool in = full || wofs + j * 32 < valid;
                if (kCarry) dg[j] = in ? (cv[j] >> shift) & (kRadix - 1) : kRadix;
                else dg[j] = in ? digit_of(k[j]) : kRadix;
            }
            // warp multisplit: the peers of a row (lanes with its digit) from
            // match.any or from digit-bit ballots (a ninth bit when the tile has
            // rows past the end); the group leader adds the group's size to the
            // warp's counter, predicated rather than branched, and the old value
            // is broadcast.  (Finding every row's peers first and then issuing
            // the counter atomics back to back measured slower: 15.31 against
            // 14.82 ms for the plain sort's eight passes at 256M rows.)
            const uint32_t lt = lanemask_lt();
#pragma unroll
            for (int j = 0; j < kIt; ++j) {
                uint32_t peers;
                if constexpr (full)  // alternate pipes: half match.any, half ballots
                    peers = ((kMatchMask >> (j & 7)) & 1) ? __match_any_sync(0xffffffffu, dg[j])
                                                          : warp_peers<kRadixBits>(dg[j]);
                else
                    peers = warp_peers<kRadixBits + 1>(dg[j]);
                const int leader = __ffs(peers) - 1;
                const uint32_t sh = (dg[j] & 1u) * 16u;
                const uint32_t old = smem_atomic_add_if_relaxed((int)lane == leader, &sm.whist2[warp][dg[j] >> 1],
                                                                (uint32_t)__popc(peers) << sh);
                rank[j] = __popc(peers & lt) + ((__shfl_sync(0xffffffffu, old, leader) >> sh) & 0xFFFFu);
            }
            __syncthreads();  // B1

            // exclusive counts over the warps of each group (all threads: digit
            // pair tid % 128, group tid / 128), and the group totals
            {
                const uint32_t pr = tid & (kRadix / 2 - 1), g = tid / (kRadix / 2);
                uint32_t acc = 0;
#pragma unroll
                for (int w = 0; w < kWpg; ++w) {
                    const uint32_t word = sm.whist2[g * kWpg + w][pr];
                    sm.whist2[g * kWpg + w][pr] = acc;
                    acc += word;
                }
                sm.gsum[g][pr] = acc;
            }
            __syncthreads();  // B2

            // warp g < kG: lane l takes digits 8l .. 8l + 7; the tile's exclusive
            // digit scan, plus the counts of earlier groups, gives each (group,
            // digit) its first staged slot; warp 0 also moves the digits' output
            // rows on
            if (warp < (uint32_t)kG) {
                // (gsum is read twice so that few registers are live next to the rows)
                uint32_t lsum = 0;
#pragma unroll
                for (int q = 0; q < 4; ++q)
#pragma unroll
                    for (int gg = 0; gg < kG; ++gg) {
                        const uint32_t v = sm.gsum[gg][4 * lane + q];
                        lsum += (v & 0xFFFFu) + (v >> 16);
                    }
                uint32_t x = lsum;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
                    if (lane >= (uint32_t)o) x += y;
                }
                uint32_t st = x - lsum;
#pragma unroll 1
                for (int q = 0; q < 4; ++q) {
                    uint32_t tot = 0, pre = 0;
#pragma unroll
                    for (int gg = 0; gg < kG; ++gg) {
                        const uint32_t v = sm.gsum[gg][4 * lane + q];
                        tot += v;
                        pre += (gg < (int)warp) ? v : 0u;
                    }
                    const uint32_t c0 = tot & 0xFFFFu, c1 = tot >> 16;
                    const uint32_t d0 = 8 * lane + 2 * q;
                    sm.gstart[warp][d0] = static_cast<uint16_t>(st + (pre & 0xFFFFu));
                    sm.gstart[warp][d0 + 1] = static_cast<uint16_t>(st + c0 + (pre >> 16));
                    if (warp == 0) {
                        const uint32_t r0 = sm.run[d0], r1 = sm.run[d0 + 1];
                        sm.gbase_rel[d0] = r0 - st;
                        sm.gbase_rel[d0 + 1] = r1 - (st + c0);
                        sm.run[d0] = r0 + c0;
                        sm.run[d0 + 1] = r1 + c1;
                    }
                    st += c0 + c1;
                }
            }
            __syncthreads();  // B3

            // stage the tile in digit order (in place: all rows are in registers)
            {
                const uint32_t grp = warp / kWpg;
#pragma unroll
                for (int j = 0; j < kIt; ++j) {
                    if (full || dg[j] < kRadix) {
                        const uint32_t wo = (sm.whist2[warp][dg[j] >> 1] >> ((dg[j] & 1u) * 16u)) & 0xFFFFu;
                        const uint32_t slot = sm.gstart[grp][dg[j]] + wo + rank[j];
                        kb[slot] = k[j];
                        if constexpr (kIdx) sm.idx[slot] = static_cast<uint16_t>(p[j]);
                        else pb[slot] = p[j];
                        if (kCarry) vb[slot] = static_cast<uint16_t>(cv[j]);
                        if (kDig) sm.dig[slot] = static_cast<uint8_t>(dg[j]);
                    }
                }
            }
            __syncthreads();  // B4

            {
#pragma unroll
                for (int j = 0; j < kIt; ++j) {
                    const uint32_t s = tid + j * THREADS;
                    if (full || s < valid) {
                        const uint64_t key = kb[s];
                        uint32_t d;
                        if (kCarry) d = (static_cast<uint32_t>(vb[s]) >> shift) & (kRadix - 1);
                        else if (kDig) d = sm.dig[s];
                        else d = static_cast<uint32_t>(key >> shift) & (kRadix - 1);
                        const uint32_t g = sm.gbase_rel[d] + s;
                        out_k[g] = key;
                        out_p[g] = kIdx ? base + sm.idx[s] : pb[s];
                        // (one byte a row, in runs under a sector: evict-last as for the carried ids)
                        if (kNext && nxt >= 0)
                            st_hint(buf.nd + g, static_cast<uint32_t>(key >> (nxt * kRadixBits)) & (kRadix - 1),
                                    l2_evict_last());
                        if (kCarry) {
                            if (rows_pass) {
                                const uint16_t v = vb[s];
                                if (s == 0 || vb[s - 1] != v) atomicMin(first_row + v, g);
                            } else {
                                // one byte a row lands in runs of ~14 bytes, under a
                                // 32-byte sector: evict-last keeps a run's partly
                                // written sector in L2 until the next tile fills it
                                // (4.79 against 4.98 ms for both passes at 256M rows)
                                st_hint(out_v + g, vb[s] >> 8, l2_evict_last());
                            }
                        }
                    }
                }
            }
        };
        if (valid == (uint32_t)TILE)
            tile(std::true_type{});
        else
            tile(std::false_type{});
        // counters of the next tile (B0 orders this before its ranking)
        for (int x = tid; x < kW * (kRadix / 2 + 1); x += THREADS) (&sm.whist2[0][0])[x] = 0;
    }
}

// Launch geometry of the chunked scatter: one chunk of whole tiles per
// resident CTA (at most kMaxChunks).
struct ChunkGeom {
    uint32_t chunk = 0, nchunks = 0;
    uint32_t want = 0;  // chunks for the largest n of this geometry (the launch grid of a device-sized sort)
    size_t smem = 0;
};

template <typename ValueFn, int TILE, int THREADS, bool kCarry, bool kIdx = false>
int chunk_geometry(uint64_t n, ChunkGeom* g) {
    auto kern = chunk_scatter_kernel<ValueFn, TILE, THREADS, kCarry, kIdx>;
    const size_t smem = sizeof(ScatterSmem<TILE, THREADS, kCarry, ScatterDig<ValueFn, kCarry>::value, kIdx>);
    SBH_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int per_sm = 0;
    SBH_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, THREADS, smem));
    if (per_sm < 1) per_sm = 1;
    const uint64_t ttiles = (n + TILE - 1) / TILE;
    const uint64_t want = min_u64(min_u64(ttiles, (uint64_t)num_sms() * per_sm), kMaxChunks);
    g->chunk = (uint32_t)(((ttiles + want - 1) / want) * TILE);
    g->nchunks = (uint32_t)((n + g->chunk - 1) / g->chunk);
    g->want = (uint32_t)want;
    g->smem = smem;
    return SBH_OK;
}


// ------------------------------------------------------------------ scratch and launch
struct SortScratch {
    uint64_t* tmp_k;
    uint32_t* tmp_p;
    uint8_t* nd;           // n: next-pass digits of the chunked passes (null: onesweep only)
    uint32_t* gbase;       // kPositions * kRadix
    Plan* plan;
    uint32_t* chunk_hist;  // kMaxChunks * kRadix
    uint32_t* chunk_base;  // kMaxChunks * kRadix
    uint32_t* hist;        // kPositions * kRadix   (zeroed)
    unsigned long long* vbits;  // 2: OR of the values, OR of their complements (zeroed)
    uint32_t* counters;    // kPositions            (zeroed)
    uint64_t* lookback;    // ntiles * kRadix       (zeroed; onesweep only)
    char* zero_begin;
    size_t zero_bytes;
    size_t total;
};

// dyn: a sort sized on the device (up to n pairs), whose onesweep path needs
// look-back records for sizes below the chunked threshold.
inline SortScratch sort_carve(void* scratch, uint64_t n, bool dyn = false) {
    Carver c(scratch);
    SortScratch s;
    const bool chunked = use_chunked(n) && !dyn;
    const uint64_t lb_rows = dyn ? min_u64(n, knob(SBH_KNOB_SORT_CHUNKED_MIN)) : n;
    const uint64_t ntiles = (lb_rows + kTile - 1) / kTile;
    s.tmp_k = c.take<uint64_t>(n);
    s.tmp_p = c.take<uint32_t>(n);
    s.nd = (chunked || dyn) ? c.take<uint8_t>(n) : nullptr;
    s.gbase = c.take<uint32_t>(kPositions * kRadix);
    s.plan = c.take<Plan>(1);
    s.chunk_hist = c.take<uint32_t>(kMaxChunks * kRadix);
    s.chunk_base = c.take<uint32_t>(kMaxChunks * kRadix);
    s.hist = c.take<uint32_t>(kPositions * kRadix);
    const size_t zb = c.off - kPositions * kRadix * sizeof(uint32_t);
    s.vbits = c.take<unsigned long long>(2);
    s.counters = c.take<uint32_t>(kPositions);
    s.lookback = chunked ? nullptr : c.take<uint64_t>(ntiles * kRadix);
    s.zero_begin = reinterpret_cast<char*>(s.hist);
    s.zero_bytes = c.off - zb;
    s.total = c.bytes();
    return s;
}

// The passes of a large sort: per pass, chunk digit counts -> chunk offsets
// -> scatter.
template <typename ValueFn, int TILE, int THREADS>
int chunked_passes(const Buffers& b, uint32_t n32, const SortScratch& sc, const ChunkGeom& g, ValueFn value_of,
                   int bulk_ok, cudaStream_t s, const std::string& n_count, const std::string& n_scan,
                   const std::string& n_scat, DynN dn = DynN{}) {
    const uint32_t limit = spin_limit();
    uint32_t* status = status_word();
    const uint32_t grid = dn.d_n ? g.want : g.nchunks;
    for (int pos = 0; pos < kPositions; ++pos) {
        if (pos > 0) {  // the first pass's chunk counts come from first_count_kernel (the same chunks, g)
            SBH_TIMED(n_count.c_str(), s,
                      chunk_count_kernel<ValueFn><<<grid, 1024, 0, s>>>(b, n32, pos, sc.plan, g.chunk,
                                                                       sc.chunk_hist, value_of, dn));
            SBH_LAUNCHED();
        }
        SBH_TIMED(n_scan.c_str(), s,
                  chunk_scan_kernel<<<1, 1024, 0, s>>>(sc.plan, pos, sc.chunk_hist, g.nchunks, nullptr,
                                                       sc.chunk_base, dn));
        SBH_LAUNCHED();
        SBH_TIMED(n_scat.c_str(), s,
                  (chunk_scatter_kernel<ValueFn, TILE, THREADS, false><<<grid, THREADS, g.smem, s>>>(
                      b, n32, pos, sc.plan, g.chunk, sc.chunk_base, value_of, bulk_ok, limit, status, nullptr,
                      nullptr, dn)));
        SBH_LAUNCHED();
    }
    return SBH_OK;
}

// The chunked passes of one sort with one scatter geometry (TILE rows per
// tile, THREADS threads per CTA): chunk geometry, first count with the
// values' bits, plan, then per pass count -> scan -> scatter.
template <typename ValueFn, int TILE, int THREADS>
int chunked_sort(const Buffers& b, uint32_t n32, const SortScratch& sc, ValueFn value_of, int npos, int in_place,
                 int bulk_ok, cudaStream_t s, const uint32_t* d_n, const std::string& n_up, const std::string& n_plan,
                 const std::string& n_count, const std::string& n_scan, const std::string& n_scat) {
    ChunkGeom g;
    int rc = chunk_geometry<ValueFn, TILE, THREADS, false>(n32, &g);
    if (rc) return rc;
    DynN dn{};
    if (d_n) dn = DynN{d_n, g.want, (uint32_t)TILE, (uint32_t)min_u64(knob(SBH_KNOB_SORT_CHUNKED_MIN), 0xFFFFFFFFull)};
    SBH_TIMED(n_up.c_str(), s,
              first_count_kernel<ValueFn><<<d_n ? g.want : g.nchunks, 1024, 0, s>>>(
                  b.in_k, n32, g.chunk, value_of, sc.chunk_hist, sc.vbits, dn));
    SBH_LAUNCHED();
    SBH_TIMED(n_plan.c_str(), s, plan_bits_kernel<<<1, 32, 0, s>>>(sc.vbits, npos, sc.plan, in_place, dn));
    SBH_LAUNCHED();
    return chunked_passes<ValueFn, TILE, THREADS>(b, n32, sc, g, value_of, bulk_ok, s, n_count, n_scan, n_scat, dn);
}

// Scatter geometries of the plain sort's chunked passes (the knob
// SBH_KNOB_SCATTER_GEOM): 0 = 4096-row tiles, 512 threads (two CTAs per SM);
// 1 = 2048 rows, 256 threads (four); 2 = 8192 rows, 1024 threads (one).
constexpr int kScatterGeoms = 3;

// Stable sort of (in_k, in_p) by value_of(key) into (out_k, out_p); the
// positions at or above npos of the value are treated as zero.  With d_n
// (device) the sort has *d_n <= n pairs, known only when it runs: both
// paths are queued (the onesweep kernels sized for the chunked threshold,
// the chunked ones for n pairs), every kernel reads the size, the chunked
// ones derive their chunk geometry from it, and the kernels of the path the
// size does not select return at once (no host synchronisation).
template <typename ValueFn>
int sort_by_value(const uint64_t* in_k, const uint32_t* in_p, uint64_t* out_k, uint32_t* out_p, uint64_t n,
                  void* scratch, cudaStream_t s, ValueFn value_of, int npos, const char* tag = "sort",
                  const uint32_t* d_n = nullptr) {
    // profile names: <tag>_upsweep, <tag>_scatter, ...
    const std::string t(tag);
    const std::string n_up = t + "_upsweep", n_plan = t + "_plan", n_count = t + "_count", n_scan = t + "_chunk_scan",
                      n_scat = t + "_scatter", n_one = t + "_onesweep", n_copy = t + "_copy";
    if (n == 0) return SBH_OK;
    const int in_place = (in_k == out_k);
    if (in_place != (in_p == out_p) || (in_place && !in_p)) {
        set_error("an in-place sort needs both keys and ptrs aliased");
        return SBH_EINVAL;
    }
    SortScratch sc = sort_carve(scratch, n, d_n != nullptr);
    SBH_CUDA(cudaMemsetAsync(sc.zero_begin, 0, sc.zero_bytes, s));
    const int sms = num_sms();
    const uint32_t n32 = static_cast<uint32_t>(n);
    // which kernels are queued: a known size takes one path; a size known
    // only on the device queues the onesweep kernels for sizes below the
    // chunked threshold and the chunked ones from it, and each returns at
    // once unless the size selects it
    const uint64_t thr = knob(SBH_KNOB_SORT_CHUNKED_MIN);
    const bool run_one = d_n ? thr > 0 : !use_chunked(n);
    const bool run_chunked = d_n ? n >= thr : use_chunked(n);
    const DynN dn_one = d_n ? DynN{d_n, 0, 0, (uint32_t)min_u64(thr, 0xFFFFFFFFull)} : DynN{};
    const uint64_t n_osw = d_n ? min_u64(n, thr) : n;  // the largest size the onesweep kernels see
    if (run_one) {
        const unsigned up_blocks = (unsigned)min_u64((n_osw + 1023) / 1024, (uint64_t)sms * 8);
        SBH_TIMED(n_up.c_str(), s,
                  upsweep_kernel<ValueFn><<<up_blocks, 256, 0, s>>>(in_k, n32, sc.hist, value_of, npos, dn_one));
        SBH_LAUNCHED();
        SBH_TIMED(n_plan.c_str(), s,
                  plan_kernel<<<1, kRadix, 0, s>>>(sc.hist, n32, sc.gbase, sc.plan, in_place, dn_one));
        SBH_LAUNCHED();
    }
    Buffers b{in_k, in_p, sc.tmp_k, sc.tmp_p, out_k, out_p};
    if (std::is_same<ValueFn, RadixValue>::value) b.nd = sc.nd;
    const size_t smem = sizeof(SortSmem);
    const uint32_t limit = spin_limit();
    uint32_t* status = status_word();
    // bulk copies need 16-byte aligned tile starts in every buffer a pass may read
    const int bulk_ok = ((reinterpret_cast<uintptr_t>(in_k) | reinterpret_cast<uintptr_t>(in_p) |
                          reinterpret_cast<uintptr_t>(out_k) | reinterpret_cast<uintptr_t>(out_p)) & 15) == 0;
    const uint64_t ntiles = (n_osw + kTile - 1) / kTile;
    if (run_chunked) {
        // the chunked passes find their digit bases in the chunk counts; the
        // plan needs only which digits vary: the first pass's counts and the
        // values' OR and AND in one read.  The plain sort's scatter geometry
        // is a knob; derived values keep the default.
        int rc;
        const uint64_t geom = std::is_same<ValueFn, RadixValue>::value ? knob(SBH_KNOB_SCATTER_GEOM) : 0;
        if constexpr (std::is_same<ValueFn, RadixValue>::value) {
            if (geom == 1)
                rc = chunked_sort<ValueFn, 2048, 256>(b, n32, sc, value_of, npos, in_place, bulk_ok, s, d_n, n_up,
                                                      n_plan, n_count, n_scan, n_scat);
            else if (geom == 2)
                rc = chunked_sort<ValueFn, 8192, 1024>(b, n32, sc, value_of, npos, in_place, bulk_ok, s, d_n, n_up,
                                                       n_plan, n_count, n_scan, n_scat);
            else
                rc = chunked_sort<ValueFn, 4096, 512>(b, n32, sc, value_of, npos, in_place, bulk_ok, s, d_n, n_up,
                                                      n_plan, n_count, n_scan, n_scat);
        } else {
            (void)geom;
            rc = chunked_sort<ValueFn, 4096, 512>(b, n32, sc, value_of, npos, in_place, bulk_ok, s, d_n, n_up, n_plan,
                                                  n_count, n_scan, n_scat);
        }
        if (rc) return rc;
    }
    if (run_one) {
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
                                                        bulk_ok, dn_one));
            SBH_LAUNCHED();
        }
    }
    const unsigned cblocks = (unsigned)min_u64((n + 255) / 256, (uint64_t)sms * 4);
    SBH_TIMED(n_copy.c_str(), s, copy_kernel<<<cblocks, 256, 0, s>>>(b, n32, sc.plan, d_n));
    SBH_LAUNCHED();
    return SBH_OK;
}

}  // namespace
}  // namespace sbh
