// A7 top-K per key, on a KPA sorted by key.
//
// One persistent kernel per call.  Each tile of 4096 rows is loaded with
// coalesced reads, transposed through shared memory so each thread owns 16
// consecutive rows, and reduced as a segmented scan whose element is
//     (number of segment heads, aggregate of the open segment).
// Combining (h1, a1) then (h2, a2) gives (h1 + h2, h2 ? a2 : a1 + a2).  Tiles
// chain their scan results with a decoupled look-back (bounded wait), so a
// key's rows may span any number of tiles.  A segment is written out by the
// thread that meets the next head (or holds the last row), at output index =
// number of heads before it.
#include "common.cuh"

namespace sbh {
namespace {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr int kIpt = 16;
constexpr int kTile = kThreads * kIpt;

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
        // shift down the entries that are worse than (val, ptr)
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
        TopK r;
        r.n = 0;
        uint32_t i = 0, j = 0;
#pragma unroll
        for (int s = 0; s < KMAX; ++s) {
            r.v[s] = 0;
            r.p[s] = 0xFFFFFFFFu;
            if (s < k) {
                const bool ha = i < n, hb = j < b.n;
                if (ha || hb) {
                    // read by dynamic index from the small arrays
                    uint64_t av = 0, bv = 0;
                    uint32_t ap = 0, bp = 0;
#pragma unroll
                    for (int q = 0; q < KMAX; ++q) {
                        if ((uint32_t)q == i) { av = v[q]; ap = p[q]; }
                        if ((uint32_t)q == j) { bv = b.v[q]; bp = b.p[q]; }
                    }
                    const bool take_a = ha && (!hb || better(av, ap, bv, bp));
                    r.v[s] = take_a ? av : bv;
                    r.p[s] = take_a ? ap : bp;
                    i += take_a;
                    j += !take_a;
                    r.n = s + 1;
                }
            }
        }
        *this = r;
    }
    __device__ __forceinline__ void shfl_up(const TopK& src, int o) {
        n = __shfl_up_sync(0xffffffffu, src.n, o);
#pragma unroll
        for (int s = 0; s < KMAX; ++s) {
            v[s] = __shfl_up_sync(0xffffffffu, src.v[s], o);
            p[s] = __shfl_up_sync(0xffffffffu, src.p[s], o);
        }
    }
};

// segmented-scan element
template <typename Agg>
struct Seg {
    uint32_t heads;
    Agg open;
};

template <typename Agg>
__device__ __forceinline__ Seg<Agg> seg_combine(const Seg<Agg>& a, const Seg<Agg>& b, int k) {
    Seg<Agg> r;
    r.heads = a.heads + b.heads;
    if (b.heads) {
        r.open = b.open;
    } else {
        r.open = a.open;
        r.open.absorb(b.open, k);
    }
    return r;
}

// look-back record of one tile: a flag word plus two immutable payloads
// (the tile's own aggregate, then its inclusive prefix).
template <typename Agg>
struct TileRec {
    Seg<Agg> agg;
    Seg<Agg> prefix;
};

constexpr uint32_t kRecAgg = 1, kRecPrefix = 2;

template <typename T>
__device__ __forceinline__ void store_volatile(T* dst, const T& v) {
    static_assert(sizeof(T) % 4 == 0, "word-sized payload");
    volatile uint32_t* d = reinterpret_cast<volatile uint32_t*>(dst);
    const uint32_t* s = reinterpret_cast<const uint32_t*>(&v);
#pragma unroll
    for (int i = 0; i < (int)(sizeof(T) / 4); ++i) d[i] = s[i];
}
template <typename T>
__device__ __forceinline__ T load_volatile(const T* src) {
    T v;
    const volatile uint32_t* s = reinterpret_cast<const volatile uint32_t*>(src);
    uint32_t* d = reinterpret_cast<uint32_t*>(&v);
#pragma unroll
    for (int i = 0; i < (int)(sizeof(T) / 4); ++i) d[i] = s[i];
    return v;
}

// ------------------------------------------------------------ output sinks
template <int KMAX>
struct TopKSink {
    uint64_t* keys;
    uint8_t* nvalid;
    uint64_t* vals;
    uint32_t* ptrs;
    uint64_t cap;
    int k;
    __device__ __forceinline__ void emit(uint64_t idx, uint64_t key, const TopK<KMAX>& a) const {
        if (idx >= cap) return;
        keys[idx] = key;
        nvalid[idx] = static_cast<uint8_t>(a.n);
#pragma unroll
        for (int s = 0; s < KMAX; ++s) {
            if (s < k) {
                vals[idx * k + s] = s < (int)a.n ? a.v[s] : 0ull;
                ptrs[idx * k + s] = s < (int)a.n ? a.p[s] : 0xFFFFFFFFu;
            }
        }
    }
};

template <typename Agg>
struct ReduceSmem {
    union {
        uint64_t keys[kTile];
        uint32_t ptrs[kTile];
    } stage;
    Seg<Agg> warp_tot[kWarps];
    Seg<Agg> tile_excl;
    uint64_t prev_key_of_tile;
    uint32_t tile;
};

// kVals: 0 = count only (no ptrs or values read), 4 or 8 = value bytes.
template <typename Agg, typename Sink, int kVals>
__global__ void __launch_bounds__(kThreads)
segreduce_kernel(const uint64_t* __restrict__ keys, const uint32_t* __restrict__ ptrs, uint64_t n,
                 const void* __restrict__ val_col, Sink sink, int k, uint64_t* __restrict__ nkeys_out,
                 uint32_t* __restrict__ flags, TileRec<Agg>* __restrict__ recs, uint32_t* __restrict__ tile_counter,
                 uint32_t spin_limit, uint32_t* __restrict__ status) {
    __shared__ ReduceSmem<Agg> sm;
    const uint32_t tid = threadIdx.x, lane = lane_id(), warp = tid / 32;
    const uint64_t ntiles = (n + kTile - 1) / kTile;

    for (;;) {
        if (tid == 0) sm.tile = atomicAdd(tile_counter, 1u);
        __syncthreads();
        const uint64_t tile = sm.tile;
        if (tile >= ntiles) break;
        const uint64_t base = tile * kTile;
        const uint32_t valid = (uint32_t)min_u64(n - base, kTile);
        if (tid == 0) sm.prev_key_of_tile = tile ? keys[base - 1] : 0ull;

        // ---- keys: coalesced load, then each thread reads 16 consecutive rows
#pragma unroll
        for (int j = 0; j < kIpt; ++j) {
            const uint32_t s = tid + j * kThreads;
            if (s < valid) sm.stage.keys[s] = ld_stream(keys + base + s);
        }
        __syncthreads();
        const uint32_t first = tid * kIpt;
        uint64_t kk[kIpt];
#pragma unroll
        for (int j = 0; j < kIpt; ++j) kk[j] = (first + j < valid) ? sm.stage.keys[first + j] : 0ull;
        uint64_t prev = first == 0 ? sm.prev_key_of_tile : (first - 1 < valid ? sm.stage.keys[first - 1] : 0ull);
        __syncthreads();

        uint32_t pp[kIpt];
        uint64_t vv[kIpt];
        if (kVals) {
#pragma unroll
            for (int j = 0; j < kIpt; ++j) {
                const uint32_t s = tid + j * kThreads;
                if (s < valid) sm.stage.ptrs[s] = ld_stream(ptrs + base + s);
            }
            __syncthreads();
#pragma unroll
            for (int j = 0; j < kIpt; ++j) pp[j] = (first + j < valid) ? sm.stage.ptrs[first + j] : 0u;
            // gather the nonresident value column through the pointers
#pragma unroll
            for (int j = 0; j < kIpt; ++j) {
                if (first + j < valid) {
                    if (kVals == 8) vv[j] = __ldg(static_cast<const unsigned long long*>(val_col) + pp[j]);
                    else vv[j] = __ldg(static_cast<const unsigned int*>(val_col) + pp[j]);
                } else {
                    vv[j] = 0;
                }
            }
        } else {
#pragma unroll
            for (int j = 0; j < kIpt; ++j) { pp[j] = 0; vv[j] = 0; }
        }

        // ---- thread summary
        uint32_t headmask = 0;
        Seg<Agg> x;
        x.heads = 0;
        x.open = Agg::identity();
        {
            uint64_t pk = prev;
#pragma unroll
            for (int j = 0; j < kIpt; ++j) {
                if (first + j < valid) {
                    const bool h = (base + first + j == 0) || kk[j] != pk;
                    if (h) {
                        headmask |= 1u << j;
                        x.heads += 1;
                        x.open = Agg::identity();
                    }
                    x.open.add_row(vv[j], pp[j], k);
                    pk = kk[j];
                }
            }
        }

        // ---- warp inclusive scan of the summaries
        Seg<Agg> inc = x;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            Seg<Agg> y;
            y.heads = __shfl_up_sync(0xffffffffu, inc.heads, o);
            y.open.shfl_up(inc.open, o);
            if (lane >= (uint32_t)o) inc = seg_combine(y, inc, k);
        }
        if (lane == 31) sm.warp_tot[warp] = inc;
        // exclusive within the warp
        Seg<Agg> wexcl;
        wexcl.heads = __shfl_up_sync(0xffffffffu, inc.heads, 1);
        wexcl.open.shfl_up(inc.open, 1);
        if (lane == 0) { wexcl.heads = 0; wexcl.open = Agg::identity(); }
        __syncthreads();

        // ---- tile aggregate, publish, look back (thread 0)
        if (tid == 0) {
            Seg<Agg> t = sm.warp_tot[0];
            for (int w = 1; w < kWarps; ++w) t = seg_combine(t, sm.warp_tot[w], k);
            Seg<Agg> excl;
            excl.heads = 0;
            excl.open = Agg::identity();
            if (tile == 0) {
                store_volatile(&recs[0].prefix, t);
                __threadfence();
                st_release(flags, kRecPrefix);
            } else {
                store_volatile(&recs[tile].agg, t);
                __threadfence();
                st_release(flags + tile, kRecAgg);
                // walk back, accumulating excl = rec[j] (+) excl
                uint64_t j = tile - 1;
                uint32_t polls = 0;
                bool have = false;
                for (;;) {
                    const uint32_t f = ld_acquire(flags + j);
                    if (f == 0) {
                        if (wait_expired(polls, spin_limit, status)) break;
                        continue;
                    }
                    const Seg<Agg> r = load_volatile(f == kRecPrefix ? &recs[j].prefix : &recs[j].agg);
                    excl = have ? seg_combine(r, excl, k) : r;
                    have = true;
                    if (f == kRecPrefix || j == 0) break;
                    --j;
                }
                const Seg<Agg> incl = seg_combine(excl, t, k);
                store_volatile(&recs[tile].prefix, incl);
                __threadfence();
                st_release(flags + tile, kRecPrefix);
            }
            sm.tile_excl = excl;
        }
        __syncthreads();

        // ---- this thread's exclusive prefix, then walk its rows and emit
        Seg<Agg> pre = sm.tile_excl;
        for (uint32_t w = 0; w < warp; ++w) pre = seg_combine(pre, sm.warp_tot[w], k);
        pre = seg_combine(pre, wexcl, k);

        Agg cur = pre.open;
        int64_t seg = (int64_t)pre.heads - 1;
        uint64_t pk = prev;
#pragma unroll
        for (int j = 0; j < kIpt; ++j) {
            if (first + j < valid) {
                if (headmask & (1u << j)) {
                    if (seg >= 0) sink.emit((uint64_t)seg, pk, cur);
                    ++seg;
                    cur = Agg::identity();
                }
                cur.add_row(vv[j], pp[j], k);
                pk = kk[j];
                if (base + first + j == n - 1) {
                    sink.emit((uint64_t)seg, pk, cur);
                    *nkeys_out = (uint64_t)(seg + 1);
                }
            }
        }
        __syncthreads();
    }
}

template <typename Agg>
size_t seg_scratch(uint64_t n, size_t* flags_off, size_t* recs_off, size_t* counter_off) {
    Carver c(nullptr);
    const uint64_t ntiles = (n + kTile - 1) / kTile;
    c.take<uint32_t>(1);
    *counter_off = 0;
    *flags_off = c.off;
    c.take<uint32_t>(ntiles);
    const size_t zero_end = c.off;
    (void)zero_end;
    c.take<TileRec<Agg>>(ntiles);
    *recs_off = c.off - ntiles * sizeof(TileRec<Agg>);
    return c.bytes();
}

template <typename Agg, typename Sink, int kVals>
int launch_segreduce(const uint64_t* keys, const uint32_t* ptrs, uint64_t n, const void* vals, Sink sink, int k,
                     uint64_t* nkeys, void* scratch, cudaStream_t s) {
    size_t flags_off, recs_off, counter_off;
    seg_scratch<Agg>(n, &flags_off, &recs_off, &counter_off);
    char* base = static_cast<char*>(scratch);
    const uint64_t ntiles = (n + kTile - 1) / kTile;
    // zero the tile counter and the flags
    SBH_CUDA(cudaMemsetAsync(base, 0, flags_off + ntiles * sizeof(uint32_t), s));
    int per_sm = 0;
    SBH_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, segreduce_kernel<Agg, Sink, kVals>, kThreads, 0));
    if (per_sm < 1) per_sm = 1;
    const unsigned grid = (unsigned)min_u64(ntiles, (uint64_t)num_sms() * per_sm);
    SBH_TIMED("segreduce", s, segreduce_kernel<Agg, Sink, kVals><<<grid, kThreads, 0, s>>>(
        keys, ptrs, n, vals, sink, k, nkeys, reinterpret_cast<uint32_t*>(base + flags_off),
        reinterpret_cast<TileRec<Agg>*>(base + recs_off), reinterpret_cast<uint32_t*>(base + counter_off),
        spin_limit(), status_word()));
    SBH_LAUNCHED();
    return SBH_OK;
}

template <int KMAX>
int topk_dispatch(const uint64_t* keys, const uint32_t* ptrs, uint64_t n, const void* vals, int vb, int K,
                  uint64_t* ok, uint8_t* onv, uint64_t* ov, uint32_t* op, uint64_t cap, uint64_t* nkeys,
                  void* scratch, cudaStream_t s) {
    TopKSink<KMAX> sink{ok, onv, ov, op, cap, K};
    if (vb == 8) return launch_segreduce<TopK<KMAX>, TopKSink<KMAX>, 8>(keys, ptrs, n, vals, sink, K, nkeys, scratch, s);
    return launch_segreduce<TopK<KMAX>, TopKSink<KMAX>, 4>(keys, ptrs, n, vals, sink, K, nkeys, scratch, s);
}

size_t topk_scratch(uint64_t n) {
    size_t a, b, c;
    return seg_scratch<TopK<8>>(n, &a, &b, &c);
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
    bool done = false;
    int rc = scratch_check(d_scratch, scratch_bytes, topk_scratch(n), &done);
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
    if (K == 1) return topk_dispatch<1>(d_keys, d_ptrs, n, d_val_col, val_bytes, K, d_out_keys, d_out_nvalid, d_out_vals, d_out_ptrs, cap, d_nkeys, d_scratch, s);
    if (K == 2) return topk_dispatch<2>(d_keys, d_ptrs, n, d_val_col, val_bytes, K, d_out_keys, d_out_nvalid, d_out_vals, d_out_ptrs, cap, d_nkeys, d_scratch, s);
    if (K == 3) return topk_dispatch<3>(d_keys, d_ptrs, n, d_val_col, val_bytes, K, d_out_keys, d_out_nvalid, d_out_vals, d_out_ptrs, cap, d_nkeys, d_scratch, s);
    if (K == 4) return topk_dispatch<4>(d_keys, d_ptrs, n, d_val_col, val_bytes, K, d_out_keys, d_out_nvalid, d_out_vals, d_out_ptrs, cap, d_nkeys, d_scratch, s);
    return topk_dispatch<8>(d_keys, d_ptrs, n, d_val_col, val_bytes, K, d_out_keys, d_out_nvalid, d_out_vals, d_out_ptrs, cap, d_nkeys, d_scratch, s);
}

}  // extern "C"
