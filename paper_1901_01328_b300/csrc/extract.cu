// A1 window ranges and A2 Extract.
#include "common.cuh"

namespace sbh {
namespace {

// ---------------------------------------------------------------- Extract
// keys[i] = src[i]; ptrs[i] = row_begin + i.  Four rows per thread step with
// 16-byte loads and stores when src, keys and ptrs are 16-byte aligned.
template <bool kVec>
__global__ void __launch_bounds__(256) extract_kernel(const uint64_t* __restrict__ src, uint32_t row_begin,
                                                       uint32_t n, uint64_t* __restrict__ keys,
                                                       uint32_t* __restrict__ ptrs, uint64_t* __restrict__ key_or,
                                                       uint64_t* __restrict__ samples, uint32_t stride) {
    uint64_t acc = 0;
    const uint32_t nthreads = gridDim.x * blockDim.x;
    const uint32_t tid = blockIdx.x * blockDim.x + threadIdx.x;
    if (kVec) {
        // two groups of four rows in flight per thread; rem = (first row of
        // the group) mod stride, advanced without dividing
        const uint32_t nq = n / 4;
        const uint32_t step_mod = samples ? (4u * nthreads) % stride : 0u;
        uint32_t rem = samples ? (4u * tid) % stride : 0u;
        auto group = [&](uint32_t q, const ulonglong2& a, const ulonglong2& b) {
            const uint32_t i = q * 4;
            __stcs(reinterpret_cast<ulonglong2*>(keys + i), a);
            __stcs(reinterpret_cast<ulonglong2*>(keys + i + 2), b);
            const uint4 p = make_uint4(row_begin + i, row_begin + i + 1, row_begin + i + 2, row_begin + i + 3);
            __stcs(reinterpret_cast<uint4*>(ptrs + i), p);
            acc |= a.x | a.y | b.x | b.y;
            if (samples) {
                const uint32_t off = rem ? stride - rem : 0u;  // first sampled row is i + off
                if (off < 4) {
                    const uint64_t v[4] = {a.x, a.y, b.x, b.y};
                    for (uint64_t o = off; o < 4; o += stride) samples[(i + o) / stride] = v[o];
                }
                rem += step_mod;
                if (rem >= stride) rem -= stride;
            }
        };
        for (uint32_t q = tid; q < nq; q += 2 * nthreads) {
            const uint32_t q2 = q + nthreads;
            const ulonglong2 a = __ldcs(reinterpret_cast<const ulonglong2*>(src + 4 * q));
            const ulonglong2 b = __ldcs(reinterpret_cast<const ulonglong2*>(src + 4 * q + 2));
            ulonglong2 c = make_ulonglong2(0, 0), d = make_ulonglong2(0, 0);
            if (q2 < nq) {
                c = __ldcs(reinterpret_cast<const ulonglong2*>(src + 4 * q2));
                d = __ldcs(reinterpret_cast<const ulonglong2*>(src + 4 * q2 + 2));
            }
            group(q, a, b);
            if (q2 < nq) group(q2, c, d);
        }
        for (uint32_t i = nq * 4 + tid; i < n; i += nthreads) {
            uint64_t k = src[i];
            keys[i] = k;
            ptrs[i] = row_begin + i;
            acc |= k;
            if (samples && i % stride == 0) samples[i / stride] = k;
        }
    } else {
        for (uint32_t i = tid; i < n; i += nthreads) {
            uint64_t k = src[i];
            keys[i] = k;
            ptrs[i] = row_begin + i;
            acc |= k;
            if (samples && i % stride == 0) samples[i / stride] = k;
        }
    }
    if (key_or) {
        for (int o = 16; o > 0; o >>= 1) acc |= __shfl_xor_sync(0xffffffffu, acc, o);
        if (lane_id() == 0 && acc) atomicOr(reinterpret_cast<unsigned long long*>(key_or), (unsigned long long)acc);
    }
}

// Only the sample: samples[j] = src[j * stride].
__global__ void __launch_bounds__(256) sample_kernel(const uint64_t* __restrict__ src, uint32_t m, uint32_t stride,
                                                      uint64_t* __restrict__ samples) {
    const uint32_t j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j < m) samples[j] = __ldg(reinterpret_cast<const unsigned long long*>(src) + (uint64_t)j * stride);
}

// ---------------------------------------------------------------- Extract of many windows
// Row r of window w (offsets[w] <= r < offsets[w + 1]) becomes the pair
// ((w << wshift) | key_col[r], r).  The window of a row is found by binary
// search over the offsets (a few KB, cached).
__global__ void __launch_bounds__(256) extract_windows_kernel(const uint64_t* __restrict__ col,
                                                              const uint64_t* __restrict__ offsets, uint32_t nwin,
                                                              uint32_t row_begin, uint32_t n, int wshift,
                                                              uint64_t* __restrict__ keys, uint32_t* __restrict__ ptrs,
                                                              uint64_t* __restrict__ key_or) {
    uint64_t acc = 0;
    const uint32_t nthreads = gridDim.x * blockDim.x;
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += nthreads) {
        const uint64_t r = (uint64_t)row_begin + i;
        // last w with offsets[w] <= r
        uint32_t lo = 0, hi = nwin;
        while (hi - lo > 1) {
            const uint32_t mid = (lo + hi) / 2;
            if (__ldg(offsets + mid) <= r) lo = mid;
            else hi = mid;
        }
        const uint64_t k = __ldcs(reinterpret_cast<const unsigned long long*>(col + r));
        acc |= k;
        __stcs(reinterpret_cast<unsigned long long*>(keys + i), (unsigned long long)((static_cast<uint64_t>(lo) << wshift) | k));
        __stcs(reinterpret_cast<unsigned int*>(ptrs + i), static_cast<unsigned int>(r));
    }
    if (key_or) {
        for (int o = 16; o > 0; o >>= 1) acc |= __shfl_xor_sync(0xffffffffu, acc, o);
        if (lane_id() == 0 && acc) atomicOr(reinterpret_cast<unsigned long long*>(key_or), (unsigned long long)acc);
    }
}

// ---------------------------------------------------------------- bundle split by timestamp
// A bundle's rows go to the window slots of their timestamps: window w =
// (ts_base + ts_rel[r]) / win_len; w == first_win or first_win + 1 goes to
// slot w & 1, anything else is dropped (counted).  Stable within each slot:
// per tile counts -> one-CTA scan that also moves the slots' fill counters
// -> emit at the tile's offset plus the row's rank among its tile's rows of
// the same slot.
constexpr int kSplitThreads = 256;
constexpr int kSplitIpt = 16;
constexpr int kSplitTile = kSplitThreads * kSplitIpt;

__device__ __forceinline__ uint32_t split_tag(int64_t ts, uint64_t win_len, uint64_t first_win) {
    if (ts < 0) return 2u;
    const uint64_t w = static_cast<uint64_t>(ts) / win_len;
    if (w == first_win || w == first_win + 1) return static_cast<uint32_t>(w & 1u);
    return 2u;
}

__global__ void __launch_bounds__(kSplitThreads) split_count_kernel(const int64_t* __restrict__ ts_rel, uint32_t n,
                                                                    int64_t ts_base, uint64_t win_len,
                                                                    uint64_t first_win, uint32_t* __restrict__ cnt) {
    __shared__ uint32_t c[3];
    if (threadIdx.x < 3) c[threadIdx.x] = 0;
    __syncthreads();
    const uint32_t base = blockIdx.x * kSplitTile;
    uint32_t mine[3] = {0, 0, 0};
#pragma unroll
    for (int j = 0; j < kSplitIpt; ++j) {
        const uint32_t r = base + j * kSplitThreads + threadIdx.x;
        if (r < n) ++mine[split_tag(ts_base + ts_rel[r], win_len, first_win)];
    }
#pragma unroll
    for (int t = 0; t < 3; ++t) {
        const uint32_t x = __reduce_add_sync(0xffffffffu, mine[t]);
        if (lane_id() == 0 && x) atomicAdd(&c[t], x);
    }
    __syncthreads();
    if (threadIdx.x < 3) cnt[blockIdx.x * 3 + threadIdx.x] = c[threadIdx.x];
}

// One CTA: tile offsets per slot (starting at the slot's fill), new fills,
// dropped rows, and the overflow flag when a slot would pass its capacity.
__global__ void __launch_bounds__(1024) split_scan_kernel(uint32_t* __restrict__ cnt, uint32_t ntiles,
                                                          uint64_t* __restrict__ fill, uint64_t cap0, uint64_t cap1,
                                                          uint64_t* __restrict__ dropped,
                                                          uint32_t* __restrict__ overflow) {
    __shared__ uint64_t wt[3][32];
    __shared__ uint64_t carry[3];
    const uint32_t lane = lane_id(), warp = threadIdx.x / 32;
    if (threadIdx.x < 3) carry[threadIdx.x] = threadIdx.x < 2 ? fill[threadIdx.x] : 0ull;
    __syncthreads();
    for (uint32_t c0 = 0; c0 < ntiles; c0 += blockDim.x) {
        const uint32_t i = c0 + threadIdx.x;
        uint64_t v[3], x[3];
#pragma unroll
        for (int t = 0; t < 3; ++t) {
            v[t] = i < ntiles ? cnt[i * 3 + t] : 0u;
            x[t] = v[t];
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint64_t y = __shfl_up_sync(0xffffffffu, x[t], o);
                if (lane >= (uint32_t)o) x[t] += y;
            }
            if (lane == 31) wt[t][warp] = x[t];
        }
        __syncthreads();
#pragma unroll
        for (int t = 0; t < 3; ++t) {
            uint64_t before = carry[t];
            for (uint32_t w = 0; w < warp; ++w) before += wt[t][w];
            if (i < ntiles) cnt[i * 3 + t] = static_cast<uint32_t>(before + x[t] - v[t]);  // offset into the slot
            x[t] += before;
        }
        __syncthreads();
        if (threadIdx.x == blockDim.x - 1)
            for (int t = 0; t < 3; ++t) carry[t] = x[t];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const uint64_t f0 = carry[0], f1 = carry[1];
        if (f0 > cap0 || f1 > cap1) *overflow = 1u;
        fill[0] = f0 < cap0 ? f0 : cap0;
        fill[1] = f1 < cap1 ? f1 : cap1;
        *dropped += carry[2];
    }
}

__global__ void __launch_bounds__(kSplitThreads) split_emit_kernel(const uint64_t* __restrict__ col,
                                                                   const int64_t* __restrict__ ts_rel, uint32_t n,
                                                                   int64_t ts_base, uint64_t win_len,
                                                                   uint64_t first_win, uint32_t ptr_base,
                                                                   const uint32_t* __restrict__ off,
                                                                   uint64_t* __restrict__ k0, uint32_t* __restrict__ p0,
                                                                   uint64_t cap0, uint64_t* __restrict__ k1,
                                                                   uint32_t* __restrict__ p1, uint64_t cap1) {
    __shared__ uint32_t wc[2][kSplitThreads / 32];
    const uint32_t lane = lane_id(), warp = threadIdx.x / 32;
    const uint32_t first = blockIdx.x * kSplitTile + warp * 32 * kSplitIpt;  // warp-striped rows
    uint32_t tag[kSplitIpt];
    uint32_t c0 = 0, c1 = 0;
#pragma unroll
    for (int j = 0; j < kSplitIpt; ++j) {
        const uint32_t r = first + j * 32 + lane;
        tag[j] = r < n ? split_tag(ts_base + ts_rel[r], win_len, first_win) : 3u;
        c0 += __popc(__ballot_sync(0xffffffffu, tag[j] == 0));
        c1 += __popc(__ballot_sync(0xffffffffu, tag[j] == 1));
    }
    if (lane == 0) {
        wc[0][warp] = c0;
        wc[1][warp] = c1;
    }
    __syncthreads();
    uint64_t o0 = off[blockIdx.x * 3], o1 = off[blockIdx.x * 3 + 1];
    for (uint32_t w = 0; w < warp; ++w) {
        o0 += wc[0][w];
        o1 += wc[1][w];
    }
    const uint32_t lt = lanemask_lt();
#pragma unroll
    for (int j = 0; j < kSplitIpt; ++j) {
        const uint32_t r = first + j * 32 + lane;
        const uint32_t m0 = __ballot_sync(0xffffffffu, tag[j] == 0), m1 = __ballot_sync(0xffffffffu, tag[j] == 1);
        if (tag[j] == 0) {
            const uint64_t g = o0 + __popc(m0 & lt);
            if (g < cap0) {
                k0[g] = col[r];
                p0[g] = ptr_base + r;
            }
        } else if (tag[j] == 1) {
            const uint64_t g = o1 + __popc(m1 & lt);
            if (g < cap1) {
                k1[g] = col[r];
                p1[g] = ptr_base + r;
            }
        }
        o0 += __popc(m0);
        o1 += __popc(m1);
    }
}

// ---------------------------------------------------------------- windows
template <typename T>
__device__ __forceinline__ uint64_t lower_bound_ts(const T* ts, uint64_t n, uint64_t v) {
    uint64_t lo = 0, hi = n;
    while (lo < hi) {
        uint64_t mid = lo + (hi - lo) / 2;
        if (static_cast<uint64_t>(ts[mid]) < v) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

template <typename T>
__global__ void window_kernel(const T* __restrict__ ts, uint64_t n, const uint64_t* __restrict__ starts,
                              uint64_t len, uint64_t nwin, uint64_t* __restrict__ rb, uint64_t* __restrict__ re) {
    uint64_t w = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
    if (w >= nwin) return;
    const uint64_t s = starts[w];
    rb[w] = lower_bound_ts(ts, n, s);
    re[w] = lower_bound_ts(ts, n, s + len);  // the caller keeps s + len below 2^64
}

// Resolves a key column that may live in page-locked host memory.
int device_view(const uint64_t* p, const uint64_t** out) {
    cudaPointerAttributes a;
    cudaError_t e = cudaPointerGetAttributes(&a, p);
    if (e != cudaSuccess) {
        cudaGetLastError();
        set_error("key_col: cudaPointerGetAttributes failed: %s", cudaGetErrorString(e));
        return SBH_EINVAL;
    }
    if (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged) {
        *out = p;
        return SBH_OK;
    }
    if (a.type == cudaMemoryTypeHost && a.devicePointer) {
        *out = static_cast<const uint64_t*>(a.devicePointer);
        return SBH_OK;
    }
    set_error("key_col must be device memory or page-locked, mapped host memory");
    return SBH_EINVAL;
}

}  // namespace
}  // namespace sbh

extern "C" {

int sbh_kpa_extract(const uint64_t* key_col, uint64_t row_begin, uint64_t n, uint64_t* d_keys, uint32_t* d_ptrs,
                    uint64_t* d_key_or, uint64_t* d_samples, uint64_t sample_stride, void* stream) {
    using namespace sbh;
    clear_error();
    if (n == 0) {
        if (d_key_or) SBH_CUDA(cudaMemsetAsync(d_key_or, 0, sizeof(uint64_t), as_stream(stream)));
        return SBH_OK;
    }
    const bool sample_only = !d_keys && !d_ptrs;
    if (!key_col || (!sample_only && (!d_keys || !d_ptrs)) || (sample_only && (!d_samples || d_key_or))) {
        set_error("null pointer");
        return SBH_EINVAL;
    }
    if (row_begin + n > 0xFFFFFFFFull || row_begin + n < row_begin) {
        set_error("row_begin + n must be < 2^32 with 32-bit pointers");
        return SBH_EINVAL;
    }
    if (d_samples && sample_stride == 0) { set_error("sample_stride must be > 0"); return SBH_EINVAL; }
    const uint64_t* col = nullptr;
    int rc = device_view(key_col, &col);
    if (rc) return rc;
    const uint64_t* src = col + row_begin;
    cudaStream_t s = as_stream(stream);
    if (sample_only) {
        const uint64_t m = (n + sample_stride - 1) / sample_stride;
        SBH_TIMED("extract_sample", s,
                  sample_kernel<<<(unsigned)((m + 255) / 256), 256, 0, s>>>(src, (uint32_t)m, (uint32_t)sample_stride,
                                                                          d_samples));
        SBH_LAUNCHED();
        return SBH_OK;
    }
    if (d_key_or) SBH_CUDA(cudaMemsetAsync(d_key_or, 0, sizeof(uint64_t), s));
    const bool vec = ((reinterpret_cast<uintptr_t>(src) | reinterpret_cast<uintptr_t>(d_keys) |
                       reinterpret_cast<uintptr_t>(d_ptrs)) & 15) == 0;
    const uint64_t work = vec ? (n + 3) / 4 : n;
    const uint64_t max_blocks = (uint64_t)num_sms() * 8;
    uint64_t blocks = (work + 255) / 256;
    if (blocks > max_blocks) blocks = max_blocks;
    uint32_t stride = d_samples ? static_cast<uint32_t>(sample_stride > 0xFFFFFFFFull ? 0xFFFFFFFFull : sample_stride) : 1;
    if (vec)
        SBH_TIMED("extract", s, extract_kernel<true><<<(unsigned)blocks, 256, 0, s>>>(src, (uint32_t)row_begin, (uint32_t)n, d_keys, d_ptrs,
                                                             d_key_or, d_samples, stride));
    else
        SBH_TIMED("extract", s, extract_kernel<false><<<(unsigned)blocks, 256, 0, s>>>(src, (uint32_t)row_begin, (uint32_t)n, d_keys, d_ptrs,
                                                              d_key_or, d_samples, stride));
    SBH_LAUNCHED();
    return SBH_OK;
}

int sbh_kpa_extract_windows(const uint64_t* key_col, const uint64_t* d_offsets, uint64_t nwin, uint64_t row_begin,
                            uint64_t n, uint64_t* d_keys, uint32_t* d_ptrs, uint64_t* d_key_or, void* stream) {
    using namespace sbh;
    clear_error();
    cudaStream_t s = as_stream(stream);
    if (nwin == 0 || nwin > 0xFFFFFFFFull) { set_error("nwin must be in 1 .. 2^32 - 1"); return SBH_EINVAL; }
    if (row_begin + n > 0xFFFFFFFFull || row_begin + n < row_begin) {
        set_error("row_begin + n must be < 2^32 with 32-bit pointers");
        return SBH_EINVAL;
    }
    if (n && (!key_col || !d_offsets || !d_keys || !d_ptrs)) { set_error("null pointer"); return SBH_EINVAL; }
    if (d_key_or) SBH_CUDA(cudaMemsetAsync(d_key_or, 0, sizeof(uint64_t), s));
    if (n == 0) return SBH_OK;
    const uint64_t* col = nullptr;
    int rc = device_view(key_col, &col);
    if (rc) return rc;
    const int wshift = 64 - sbh_window_bits(nwin);
    const uint64_t max_blocks = (uint64_t)num_sms() * 8;
    uint64_t blocks = (n + 255) / 256;
    if (blocks > max_blocks) blocks = max_blocks;
    SBH_TIMED("extract_windows", s,
              extract_windows_kernel<<<(unsigned)blocks, 256, 0, s>>>(col, d_offsets, (uint32_t)nwin, (uint32_t)row_begin,
                                                                      (uint32_t)n, wshift, d_keys, d_ptrs, d_key_or));
    SBH_LAUNCHED();
    return SBH_OK;
}

int sbh_kpa_split_ts(const uint64_t* key_col, const int64_t* ts_rel, uint64_t n, int64_t ts_base, uint64_t win_len,
                     uint64_t first_win, uint32_t ptr_base, uint64_t* d_keys0, uint32_t* d_ptrs0, uint64_t cap0,
                     uint64_t* d_keys1, uint32_t* d_ptrs1, uint64_t cap1, uint64_t* d_fill, uint64_t* d_dropped,
                     uint32_t* d_overflow, void* d_scratch, size_t* scratch_bytes, void* stream) {
    using namespace sbh;
    clear_error();
    const uint64_t ntiles = (n + kSplitTile - 1) / kSplitTile;
    bool done = false;
    int rc = scratch_check(d_scratch, scratch_bytes, (ntiles ? ntiles : 1) * 3 * sizeof(uint32_t), &done);
    if (rc || done) return rc;
    if (n == 0) return SBH_OK;
    if (win_len == 0) { set_error("win_len must be > 0"); return SBH_EINVAL; }
    if ((uint64_t)ptr_base + n > 0xFFFFFFFFull) { set_error("ptr_base + n must be < 2^32"); return SBH_EINVAL; }
    if (!key_col || !ts_rel || !d_fill || !d_dropped || !d_overflow || (cap0 && (!d_keys0 || !d_ptrs0)) ||
        (cap1 && (!d_keys1 || !d_ptrs1))) {
        set_error("null pointer");
        return SBH_EINVAL;
    }
    cudaStream_t s = as_stream(stream);
    uint32_t* cnt = static_cast<uint32_t*>(d_scratch);
    const uint32_t n32 = static_cast<uint32_t>(n);
    SBH_TIMED("split_count", s, split_count_kernel<<<(unsigned)ntiles, kSplitThreads, 0, s>>>(ts_rel, n32, ts_base, win_len,
                                                                                          first_win, cnt));
    SBH_LAUNCHED();
    SBH_TIMED("split_scan", s, split_scan_kernel<<<1, 1024, 0, s>>>(cnt, (uint32_t)ntiles, d_fill, cap0, cap1, d_dropped,
                                                                    d_overflow));
    SBH_LAUNCHED();
    SBH_TIMED("split_emit", s,
              split_emit_kernel<<<(unsigned)ntiles, kSplitThreads, 0, s>>>(key_col, ts_rel, n32, ts_base, win_len,
                                                                           first_win, ptr_base, cnt, d_keys0, d_ptrs0,
                                                                           cap0, d_keys1, d_ptrs1, cap1));
    SBH_LAUNCHED();
    return SBH_OK;
}

int sbh_window_bits(uint64_t nwin) { return nwin ? 64 - __builtin_clzll(nwin) : 0; }

int sbh_window_ranges(const void* d_ts, int ts_bytes, uint64_t n, const uint64_t* d_starts, uint64_t len,
                      uint64_t nwin, uint64_t* d_row_begin, uint64_t* d_row_end, void* stream) {
    using namespace sbh;
    clear_error();
    if (nwin == 0) return SBH_OK;
    if ((!d_ts && n) || !d_starts || !d_row_begin || !d_row_end) { set_error("null pointer"); return SBH_EINVAL; }
    if (ts_bytes != 4 && ts_bytes != 8) { set_error("ts_bytes must be 4 or 8"); return SBH_EINVAL; }
    cudaStream_t s = as_stream(stream);
    unsigned blocks = (unsigned)((nwin + 255) / 256);
    if (ts_bytes == 4)
        SBH_TIMED("window_ranges", s, window_kernel<uint32_t><<<blocks, 256, 0, s>>>(static_cast<const uint32_t*>(d_ts), n, d_starts, len, nwin,
                                                       d_row_begin, d_row_end));
    else
        SBH_TIMED("window_ranges", s, window_kernel<uint64_t><<<blocks, 256, 0, s>>>(static_cast<const uint64_t*>(d_ts), n, d_starts, len, nwin,
                                                       d_row_begin, d_row_end));
    SBH_LAUNCHED();
    return SBH_OK;
}

}  // extern "C"
