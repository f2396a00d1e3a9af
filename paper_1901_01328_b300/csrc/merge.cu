// A5 Merge: merge-path merge of sorted KPAs in (key, ptr) order.
//
// Two runs A and B are merged by output tiles of 2048 pairs.  For large
// merges one small kernel first finds where every tile's first output
// diagonal cuts A and B (a binary search on the merge path per tile, all
// tiles in parallel; small merges let each CTA search its own); each CTA of
// the merge then stages its two slices in shared memory, and each thread
// merges 8 outputs from its own co-rank and stores them from registers.  More than two runs are merged in rounds of
// pairwise merges through a scratch ping-pong buffer.
#include <vector>

#include "common.cuh"

namespace sbh {
namespace {

constexpr int kThreads = 256;
constexpr int kIpt = 8;
constexpr int kTile = kThreads * kIpt;

__device__ __forceinline__ bool kp_less(uint64_t ka, uint32_t pa, uint64_t kb, uint32_t pb) {
    return ka < kb || (ka == kb && pa < pb);
}

// Number of A elements among the first d outputs of merge(A, B).
template <typename KA, typename PA, typename KB, typename PB>
__device__ __forceinline__ uint32_t corank(uint32_t d, const KA ak, const PA ap, uint32_t na, const KB bk,
                                           const PB bp, uint32_t nb) {
    uint32_t lo = d > nb ? d - nb : 0;
    uint32_t hi = d < na ? d : na;
    while (lo < hi) {
        const uint32_t mid = (lo + hi) / 2;
        const uint32_t j = d - mid - 1;
        if (kp_less(bk[j], bp[j], ak[mid], ap[mid])) hi = mid;
        else lo = mid + 1;
    }
    return lo;
}

// cuts[t] = co-rank of diagonal min(t * kTile, na + nb), t <= ntiles.
__global__ void __launch_bounds__(256)
merge_cuts_kernel(const uint64_t* __restrict__ ak, const uint32_t* __restrict__ ap, uint32_t na,
                  const uint64_t* __restrict__ bk, const uint32_t* __restrict__ bp, uint32_t nb, uint32_t ntiles,
                  uint32_t* __restrict__ cuts) {
    const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t > ntiles) return;
    const uint32_t d = (uint32_t)min_u64((uint64_t)t * kTile, (uint64_t)na + nb);
    cuts[t] = corank(d, ak, ap, na, bk, bp, nb);
}

// Merges the tile of outputs made of A rows [a0, a0 + la) and B rows [b0,
// b0 + lb) (a merge-path slice) into ok[0 .. la + lb), op[...].  vec_ok: ok
// and op are 16-byte aligned at the tile start.
__device__ __forceinline__ void merge_tile(const uint64_t* __restrict__ ak, const uint32_t* __restrict__ ap,
                                           uint32_t a0, uint32_t la, const uint64_t* __restrict__ bk,
                                           const uint32_t* __restrict__ bp, uint32_t b0, uint32_t lb,
                                           uint64_t* __restrict__ ok, uint32_t* __restrict__ op, int vec_ok,
                                           uint64_t* sk, uint32_t* sp) {
    const uint32_t len = la + lb;
    // stage A slice then B slice; element x sits at slot x ^ ((x >> 4) & 15),
    // so that threads reading a few elements apart (the merge below) hit
    // different banks
    auto sw = [](uint32_t x) { return x ^ ((x >> 4) & 15u); };
    for (uint32_t i = threadIdx.x; i < len; i += kThreads) {
        if (i < la) { sk[sw(i)] = ak[a0 + i]; sp[sw(i)] = ap[a0 + i]; }
        else { sk[sw(i)] = bk[b0 + i - la]; sp[sw(i)] = bp[b0 + i - la]; }
    }
    __syncthreads();
    // each thread merges kIpt outputs starting at its own diagonal (the
    // co-rank by binary search; the two heads kept in registers)
    const uint32_t my = min(threadIdx.x * kIpt, len);
    uint32_t i, j;
    {
        uint32_t lo = my > lb ? my - lb : 0, hi = my < la ? my : la;
        while (lo < hi) {
            const uint32_t mid = (lo + hi) / 2;
            const uint32_t q = la + (my - mid - 1);
            if (kp_less(sk[sw(q)], sp[sw(q)], sk[sw(mid)], sp[sw(mid)])) hi = mid;
            else lo = mid + 1;
        }
        i = lo;
        j = my - lo;
    }
    uint64_t ka = i < la ? sk[sw(i)] : 0, kb = j < lb ? sk[sw(la + j)] : 0;
    uint32_t pa = i < la ? sp[sw(i)] : 0, pb = j < lb ? sp[sw(la + j)] : 0;
    uint64_t rk[kIpt];
    uint32_t rp[kIpt];
#pragma unroll
    for (int t = 0; t < kIpt; ++t) {
        const bool ha = i < la, hb = j < lb;
        const bool take_a = ha && (!hb || !kp_less(kb, pb, ka, pa));
        rk[t] = take_a ? ka : (hb ? kb : 0);
        rp[t] = take_a ? pa : (hb ? pb : 0);
        if (take_a) {
            ++i;
            if (i < la) {
                ka = sk[sw(i)];
                pa = sp[sw(i)];
            }
        } else if (hb) {
            ++j;
            if (j < lb) {
                kb = sk[sw(la + j)];
                pb = sp[sw(la + j)];
            }
        }
    }
    // this thread's kIpt outputs are consecutive: 16-byte stores straight
    // from registers (a staging round trip through shared memory would hit
    // the same banks from every eighth thread)
    const uint32_t o0 = threadIdx.x * kIpt;
    if (vec_ok && o0 + kIpt <= len) {
        uint4* kq = reinterpret_cast<uint4*>(ok + o0);
#pragma unroll
        for (int t = 0; t < kIpt; t += 2)
            __stcs(kq + t / 2, make_uint4(static_cast<uint32_t>(rk[t]), static_cast<uint32_t>(rk[t] >> 32),
                                          static_cast<uint32_t>(rk[t + 1]), static_cast<uint32_t>(rk[t + 1] >> 32)));
        uint4* pq = reinterpret_cast<uint4*>(op + o0);
#pragma unroll
        for (int t = 0; t < kIpt; t += 4) __stcs(pq + t / 4, make_uint4(rp[t], rp[t + 1], rp[t + 2], rp[t + 3]));
    } else {
#pragma unroll
        for (int t = 0; t < kIpt; ++t) {
            if (o0 + t < len) {
                st_stream(ok + o0 + t, rk[t]);
                st_stream(op + o0 + t, rp[t]);
            }
        }
    }
}

__global__ void __launch_bounds__(kThreads)
merge_pair_kernel(const uint64_t* __restrict__ ak, const uint32_t* __restrict__ ap, uint32_t na,
                  const uint64_t* __restrict__ bk, const uint32_t* __restrict__ bp, uint32_t nb,
                  const uint32_t* __restrict__ cuts, uint64_t* __restrict__ ok, uint32_t* __restrict__ op, int vec_ok) {
    __shared__ uint64_t sk[kTile];
    __shared__ uint32_t sp[kTile];
    __shared__ uint32_t cut[2];
    const uint32_t total = na + nb;
    const uint32_t d0 = blockIdx.x * kTile;
    const uint32_t d1 = min(d0 + kTile, total);
    if (!cuts) {  // small merges find their own cuts (one launch fewer)
        if (threadIdx.x < 2) cut[threadIdx.x] = corank(threadIdx.x ? d1 : d0, ak, ap, na, bk, bp, nb);
        __syncthreads();
    }
    const uint32_t a0 = cuts ? cuts[blockIdx.x] : cut[0], a1 = cuts ? cuts[blockIdx.x + 1] : cut[1];
    const uint32_t b0 = d0 - a0, b1 = d1 - a1;
    merge_tile(ak, ap, a0, a1 - a0, bk, bp, b0, b1 - b0, ok + d0, op + d0, vec_ok, sk, sp);
}

// ---------------------------------------------------------------- many independent merges
// Segment s merges A rows [a_start, a_start + a_len) with B rows [b_start,
// b_start + b_len) into out rows [out_start, out_start + a_len + b_len); its
// output tiles are the global tiles [tile0, tile0 + ceil(len / kTile)).
struct MergeSeg {
    uint64_t a_start, a_len, b_start, b_len, out_start, tile0;
};

__device__ __forceinline__ uint32_t seg_of_tile(const MergeSeg* __restrict__ segs, uint32_t nseg, uint32_t t) {
    uint32_t lo = 0, hi = nseg;  // last segment whose first tile is <= t
    while (hi - lo > 1) {
        const uint32_t mid = (lo + hi) / 2;
        if (segs[mid].tile0 <= t) lo = mid;
        else hi = mid;
    }
    return lo;
}

// cuts[t] = co-rank of global tile t's first output diagonal in its segment.
__global__ void __launch_bounds__(256)
merge_seg_cuts_kernel(const uint64_t* __restrict__ ak, const uint32_t* __restrict__ ap,
                      const uint64_t* __restrict__ bk, const uint32_t* __restrict__ bp,
                      const MergeSeg* __restrict__ segs, uint32_t nseg, uint32_t ntiles, uint32_t* __restrict__ cuts) {
    const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= ntiles) return;
    const MergeSeg g = segs[seg_of_tile(segs, nseg, t)];
    const uint32_t d = (uint32_t)((t - g.tile0) * (uint64_t)kTile);
    cuts[t] = corank(d, ak + g.a_start, ap + g.a_start, (uint32_t)g.a_len, bk + g.b_start, bp + g.b_start,
                     (uint32_t)g.b_len);
}

__global__ void __launch_bounds__(kThreads)
merge_seg_kernel(const uint64_t* __restrict__ ak, const uint32_t* __restrict__ ap, const uint64_t* __restrict__ bk,
                 const uint32_t* __restrict__ bp, const MergeSeg* __restrict__ segs, uint32_t nseg,
                 const uint32_t* __restrict__ cuts, uint64_t* __restrict__ ok, uint32_t* __restrict__ op, int vec_ok) {
    __shared__ uint64_t sk[kTile];
    __shared__ uint32_t sp[kTile];
    const uint32_t t = blockIdx.x;
    const MergeSeg g = segs[seg_of_tile(segs, nseg, t)];
    const uint32_t total = (uint32_t)(g.a_len + g.b_len);
    const uint32_t d0 = (uint32_t)((t - g.tile0) * (uint64_t)kTile);
    const uint32_t d1 = min(d0 + (uint32_t)kTile, total);
    const uint32_t a0 = cuts[t];
    const uint32_t a1 = d1 < total ? cuts[t + 1] : (uint32_t)g.a_len;  // the next tile is in this segment
    const uint32_t b0 = d0 - a0, b1 = d1 - a1;
    const int vec = vec_ok && (g.out_start % 4) == 0;
    merge_tile(ak + g.a_start, ap + g.a_start, a0, a1 - a0, bk + g.b_start, bp + g.b_start, b0, b1 - b0,
               ok + g.out_start + d0, op + g.out_start + d0, vec, sk, sp);
}

__global__ void copy_run_kernel(const uint64_t* __restrict__ k, const uint32_t* __restrict__ p, uint32_t n,
                                uint64_t* __restrict__ ok, uint32_t* __restrict__ op) {
    const uint32_t stride = gridDim.x * blockDim.x;
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        ok[i] = k[i];
        op[i] = p[i];
    }
}

struct Run {
    const uint64_t* k;
    const uint32_t* p;
    uint64_t n;
};

int merge_two(const Run& a, const Run& b, uint64_t* ok, uint32_t* op, uint32_t* cuts, cudaStream_t s) {
    const uint64_t total = a.n + b.n;
    if (total == 0) return SBH_OK;
    const uint32_t ntiles = (uint32_t)((total + kTile - 1) / kTile);
    if (ntiles > knob(SBH_KNOB_MERGE_SEARCH_MIN_TILES)) {  // default 2047 tiles (4M outputs)
        SBH_TIMED("merge_cuts", s,
                  merge_cuts_kernel<<<(ntiles + 256) / 256, 256, 0, s>>>(a.k, a.p, (uint32_t)a.n, b.k, b.p,
                                                                       (uint32_t)b.n, ntiles, cuts));
        SBH_LAUNCHED();
    } else {
        cuts = nullptr;
    }
    const int vec_ok = ((reinterpret_cast<uintptr_t>(ok) | reinterpret_cast<uintptr_t>(op)) & 15) == 0;
    SBH_TIMED("merge_path", s,
              merge_pair_kernel<<<ntiles, kThreads, 0, s>>>(a.k, a.p, (uint32_t)a.n, b.k, b.p, (uint32_t)b.n, cuts,
                                                            ok, op, vec_ok));
    SBH_LAUNCHED();
    return SBH_OK;
}

int copy_run(const Run& a, uint64_t* ok, uint32_t* op, cudaStream_t s) {
    if (a.n == 0 || a.k == ok) return SBH_OK;
    const unsigned grid = (unsigned)min_u64((a.n + 255) / 256, (uint64_t)num_sms() * 8);
    SBH_TIMED("merge_copy", s, copy_run_kernel<<<grid, 256, 0, s>>>(a.k, a.p, (uint32_t)a.n, ok, op));
    SBH_LAUNCHED();
    return SBH_OK;
}

}  // namespace
}  // namespace sbh

extern "C" int sbh_kpa_merge(int nruns, const uint64_t* const* d_run_keys, const uint32_t* const* d_run_ptrs,
                             const uint64_t* run_lens, uint64_t* d_keys_out, uint32_t* d_ptrs_out, void* d_scratch,
                             size_t* scratch_bytes, void* stream) {
    using namespace sbh;
    clear_error();
    if (nruns < 0 || (nruns > 0 && (!d_run_keys || !d_run_ptrs || !run_lens))) {
        set_error("bad run arrays");
        return SBH_EINVAL;
    }
    uint64_t total = 0;
    for (int r = 0; r < nruns; ++r) total += run_lens[r];
    if (total > 0xFFFFFFFFull) { set_error("total length must be < 2^32"); return SBH_EINVAL; }
    Carver c(nullptr);
    c.take<uint32_t>(total / kTile + 2);  // tile cuts
    if (nruns > 2) { c.take<uint64_t>(total); c.take<uint32_t>(total); c.take<uint64_t>(total); c.take<uint32_t>(total); }
    bool done = false;
    int rc = scratch_check(d_scratch, scratch_bytes, c.bytes(), &done);
    if (rc || done) return rc;
    if (total == 0) return SBH_OK;
    if (!d_keys_out || !d_ptrs_out) { set_error("null output"); return SBH_EINVAL; }
    for (int r = 0; r < nruns; ++r)
        if (run_lens[r] && (!d_run_keys[r] || !d_run_ptrs[r])) { set_error("null run pointer"); return SBH_EINVAL; }
    cudaStream_t s = as_stream(stream);
    std::vector<Run> runs;
    for (int r = 0; r < nruns; ++r)
        if (run_lens[r]) runs.push_back({d_run_keys[r], d_run_ptrs[r], run_lens[r]});
    Carver w(d_scratch);
    uint32_t* cuts = w.take<uint32_t>(total / kTile + 2);
    if (runs.size() == 1) return copy_run(runs[0], d_keys_out, d_ptrs_out, s);
    if (runs.size() == 2) return merge_two(runs[0], runs[1], d_keys_out, d_ptrs_out, cuts, s);
    // rounds of pairwise merges; each round writes one of two scratch buffers,
    // the last round writes the output
    uint64_t* bk[2];
    uint32_t* bp[2];
    bk[0] = w.take<uint64_t>(total);
    bp[0] = w.take<uint32_t>(total);
    bk[1] = w.take<uint64_t>(total);
    bp[1] = w.take<uint32_t>(total);
    int cur = 0;
    while (runs.size() > 1) {
        const bool last = runs.size() == 2;
        uint64_t* ok = last ? d_keys_out : bk[cur];
        uint32_t* op = last ? d_ptrs_out : bp[cur];
        std::vector<Run> next;
        uint64_t off = 0;
        for (size_t r = 0; r + 1 < runs.size(); r += 2) {
            rc = merge_two(runs[r], runs[r + 1], ok + off, op + off, cuts, s);
            if (rc) return rc;
            next.push_back({ok + off, op + off, runs[r].n + runs[r + 1].n});
            off += runs[r].n + runs[r + 1].n;
        }
        if (runs.size() % 2) {
            const Run& odd = runs.back();
            rc = copy_run(odd, ok + off, op + off, s);
            if (rc) return rc;
            next.push_back({ok + off, op + off, odd.n});
        }
        runs.swap(next);
        cur ^= 1;
    }
    return SBH_OK;
}

extern "C" int sbh_kpa_merge_segments(int nseg, const uint64_t* d_a_keys, const uint32_t* d_a_ptrs,
                                      const uint64_t* d_b_keys, const uint32_t* d_b_ptrs, const uint64_t* a_start,
                                      const uint64_t* a_len, const uint64_t* b_start, const uint64_t* b_len,
                                      uint64_t* d_keys_out, uint32_t* d_ptrs_out, void* d_scratch,
                                      size_t* scratch_bytes, void* stream) {
    using namespace sbh;
    clear_error();
    if (nseg < 0 || (nseg > 0 && (!a_start || !a_len || !b_start || !b_len))) {
        set_error("bad segment arrays");
        return SBH_EINVAL;
    }
    // the segments' outputs lie end to end; every index stays below 2^32
    std::vector<MergeSeg> segs;
    uint64_t out = 0, tiles = 0;
    for (int g = 0; g < nseg; ++g) {
        const uint64_t len = a_len[g] + b_len[g];
        if (a_start[g] + a_len[g] > 0xFFFFFFFFull || b_start[g] + b_len[g] > 0xFFFFFFFFull) {
            set_error("segment %d reaches past 2^32 rows", g);
            return SBH_EINVAL;
        }
        if (len == 0) continue;
        segs.push_back({a_start[g], a_len[g], b_start[g], b_len[g], out, tiles});
        out += len;
        tiles += (len + kTile - 1) / kTile;
    }
    if (out > 0xFFFFFFFFull) { set_error("total output must be < 2^32 rows"); return SBH_EINVAL; }
    Carver c(nullptr);
    c.take<MergeSeg>(segs.size() + 1);
    c.take<uint32_t>(tiles + 1);
    bool done = false;
    int rc = scratch_check(d_scratch, scratch_bytes, c.bytes(), &done);
    if (rc || done) return rc;
    if (segs.empty()) return SBH_OK;
    if (!d_a_keys || !d_a_ptrs || !d_b_keys || !d_b_ptrs || !d_keys_out || !d_ptrs_out) {
        set_error("null pointer");
        return SBH_EINVAL;
    }
    cudaStream_t s = as_stream(stream);
    Carver w(d_scratch);
    MergeSeg* d_segs = w.take<MergeSeg>(segs.size() + 1);
    uint32_t* cuts = w.take<uint32_t>(tiles + 1);
    SBH_CUDA(cudaMemcpyAsync(d_segs, segs.data(), segs.size() * sizeof(MergeSeg), cudaMemcpyHostToDevice, s));
    const uint32_t nt = (uint32_t)tiles, ns = (uint32_t)segs.size();
    SBH_TIMED("merge_seg_cuts", s,
              merge_seg_cuts_kernel<<<(nt + 255) / 256, 256, 0, s>>>(d_a_keys, d_a_ptrs, d_b_keys, d_b_ptrs, d_segs,
                                                                    ns, nt, cuts));
    SBH_LAUNCHED();
    const int vec_ok = ((reinterpret_cast<uintptr_t>(d_keys_out) | reinterpret_cast<uintptr_t>(d_ptrs_out)) & 15) == 0;
    SBH_TIMED("merge_seg", s,
              merge_seg_kernel<<<nt, kThreads, 0, s>>>(d_a_keys, d_a_ptrs, d_b_keys, d_b_ptrs, d_segs, ns, cuts,
                                                       d_keys_out, d_ptrs_out, vec_ok));
    SBH_LAUNCHED();
    return SBH_OK;
}
