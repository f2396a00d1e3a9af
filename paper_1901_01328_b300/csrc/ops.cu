// Record-level primitives of Table 2 on a KPA: Materialize (and KeySwap,
// the same gather of another key column) and Select.
#include "common.cuh"

namespace sbh {
namespace {

// ---------------------------------------------------------------- Materialize
// out[i] = col[ptrs[i]]: four rows per thread step, their pointer loads and
// then their gathers in flight together.
template <typename T>
__global__ void __launch_bounds__(256) gather_kernel(const uint32_t* __restrict__ ptrs, uint32_t n,
                                                     const T* __restrict__ col, T* __restrict__ out) {
    const uint32_t stride = gridDim.x * blockDim.x;
    for (uint32_t i0 = blockIdx.x * blockDim.x + threadIdx.x; i0 < n; i0 += 4 * stride) {
        uint32_t p[4];
        T v[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) p[u] = i0 + u * stride < n ? ld_stream(ptrs + i0 + u * stride) : 0u;
#pragma unroll
        for (int u = 0; u < 4; ++u) v[u] = i0 + u * stride < n ? __ldg(col + p[u]) : T(0);
#pragma unroll
        for (int u = 0; u < 4; ++u)
            if (i0 + u * stride < n) out[i0 + u * stride] = v[u];
    }
}

// ---------------------------------------------------------------- counted copy
// dst[i] = src[i] for i < min(*count, cap) * per, the count read on the
// device; dst may be page-locked host memory (written over the host link);
// D narrower than T keeps the low bytes.
template <typename T, typename D>
__global__ void __launch_bounds__(256) copy_counted_kernel(const T* __restrict__ src, D* __restrict__ dst,
                                                           const uint64_t* __restrict__ count, uint64_t per,
                                                           uint64_t cap) {
    const uint64_t m = min_u64(*count, cap) * per;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < m; i += stride)
        dst[i] = static_cast<D>(src[i]);
}

// ---------------------------------------------------------------- KeySwap through a lookup
// keys_out[i] = table[col[ptrs[i]]] (Materialize of col fused with the
// Extract of a new key by a lookup table); a value past the table gives ~0
// and is counted.
__global__ void __launch_bounds__(256) lookup_kernel(const uint32_t* __restrict__ ptrs, uint32_t n,
                                                     const uint64_t* __restrict__ col,
                                                     const uint64_t* __restrict__ table, uint64_t table_len,
                                                     uint64_t* __restrict__ out, unsigned long long* __restrict__ misses) {
    const uint32_t stride = gridDim.x * blockDim.x;
    uint32_t miss = 0;
    for (uint32_t i0 = blockIdx.x * blockDim.x + threadIdx.x; i0 < n; i0 += 4 * stride) {
        uint32_t p[4];
        uint64_t c[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) p[u] = i0 + u * stride < n ? ld_stream(ptrs + i0 + u * stride) : 0u;
#pragma unroll
        for (int u = 0; u < 4; ++u) c[u] = i0 + u * stride < n ? __ldg(col + p[u]) : 0ull;
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            if (i0 + u * stride < n) {
                const bool ok = c[u] < table_len;
                out[i0 + u * stride] = ok ? __ldg(table + c[u]) : ~0ull;
                miss += ok ? 0u : 1u;
            }
        }
    }
    if (misses) {
        miss = __reduce_add_sync(0xffffffffu, miss);
        if (lane_id() == 0 && miss) atomicAdd(misses, (unsigned long long)miss);
    }
}

// ---------------------------------------------------------------- Select
// Stable compaction of the rows whose value col[ptr] lies in [lo, hi):
// per-tile counts -> one-CTA scan -> emit at the tile's offset plus the
// row's rank among its tile's kept rows.
constexpr int kSelThreads = 256;
constexpr int kSelIpt = 16;
constexpr int kSelTile = kSelThreads * kSelIpt;

template <typename T>
__device__ __forceinline__ uint32_t keep_bits(const uint32_t* __restrict__ ptrs, uint32_t n, const T* __restrict__ col,
                                              uint64_t lo, uint64_t hi, uint32_t first, uint32_t lane,
                                              uint32_t (&p)[kSelIpt]) {
#pragma unroll
    for (int j = 0; j < kSelIpt; ++j) {
        const uint32_t r = first + j * 32 + lane;
        p[j] = r < n ? ld_stream(ptrs + r) : 0u;
    }
    uint32_t m = 0;
#pragma unroll
    for (int j = 0; j < kSelIpt; ++j) {
        const uint32_t r = first + j * 32 + lane;
        if (r < n) {
            const uint64_t v = static_cast<uint64_t>(__ldg(col + p[j]));
            if (v >= lo && v < hi) m |= 1u << j;
        }
    }
    return m;
}

template <typename T>
__global__ void __launch_bounds__(kSelThreads) select_count_kernel(const uint32_t* __restrict__ ptrs, uint32_t n,
                                                                   const T* __restrict__ col, uint64_t lo, uint64_t hi,
                                                                   uint32_t* __restrict__ cnt) {
    __shared__ uint32_t wc[kSelThreads / 32];
    const uint32_t lane = lane_id(), warp = threadIdx.x / 32;
    const uint32_t first = blockIdx.x * kSelTile + warp * 32 * kSelIpt;
    uint32_t p[kSelIpt];
    const uint32_t m = keep_bits(ptrs, n, col, lo, hi, first, lane, p);
    const uint32_t c = __reduce_add_sync(0xffffffffu, __popc(m));
    if (lane == 0) wc[warp] = c;
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t t = 0;
        for (int w = 0; w < kSelThreads / 32; ++w) t += wc[w];
        cnt[blockIdx.x] = t;
    }
}

__global__ void __launch_bounds__(1024) select_scan_kernel(uint32_t* __restrict__ cnt, uint32_t ntiles,
                                                           uint64_t* __restrict__ total) {
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
    if (threadIdx.x == 0) *total = carry;
}

template <typename T>
__global__ void __launch_bounds__(kSelThreads) select_emit_kernel(const uint64_t* __restrict__ keys,
                                                                  const uint32_t* __restrict__ ptrs, uint32_t n,
                                                                  const T* __restrict__ col, uint64_t lo, uint64_t hi,
                                                                  const uint32_t* __restrict__ off,
                                                                  uint64_t* __restrict__ out_keys,
                                                                  uint32_t* __restrict__ out_ptrs, uint64_t cap) {
    __shared__ uint32_t wc[kSelThreads / 32];
    const uint32_t lane = lane_id(), warp = threadIdx.x / 32;
    const uint32_t first = blockIdx.x * kSelTile + warp * 32 * kSelIpt;
    uint32_t p[kSelIpt];
    const uint32_t m = keep_bits(ptrs, n, col, lo, hi, first, lane, p);
    const uint32_t c = __reduce_add_sync(0xffffffffu, __popc(m));
    if (lane == 0) wc[warp] = c;
    __syncthreads();
    uint64_t g = off[blockIdx.x];
    for (uint32_t w = 0; w < warp; ++w) g += wc[w];
    const uint32_t lt = lanemask_lt();
#pragma unroll
    for (int j = 0; j < kSelIpt; ++j) {
        const uint32_t b = __ballot_sync(0xffffffffu, (m >> j) & 1u);
        if ((m >> j) & 1u) {
            const uint64_t gi = g + __popc(b & lt);
            if (gi < cap) {
                out_keys[gi] = keys[first + j * 32 + lane];
                out_ptrs[gi] = p[j];
            }
        }
        g += __popc(b);
    }
}

template <typename T>
int select_run(const uint64_t* keys, const uint32_t* ptrs, uint32_t n, const void* col, uint64_t lo, uint64_t hi,
               uint64_t* ok, uint32_t* op, uint64_t cap, uint64_t* count, uint32_t* cnt, cudaStream_t s) {
    const uint32_t ntiles = (n + kSelTile - 1) / kSelTile;
    const T* c = static_cast<const T*>(col);
    SBH_TIMED("select_count", s, select_count_kernel<T><<<ntiles, kSelThreads, 0, s>>>(ptrs, n, c, lo, hi, cnt));
    SBH_LAUNCHED();
    SBH_TIMED("select_scan", s, select_scan_kernel<<<1, 1024, 0, s>>>(cnt, ntiles, count));
    SBH_LAUNCHED();
    SBH_TIMED("select_emit", s, select_emit_kernel<T><<<ntiles, kSelThreads, 0, s>>>(keys, ptrs, n, c, lo, hi, cnt, ok,
                                                                                   op, cap));
    SBH_LAUNCHED();
    return SBH_OK;
}

}  // namespace
}  // namespace sbh

extern "C" {

int sbh_kpa_materialize(const uint32_t* d_ptrs, uint64_t n, const void* d_col, int col_bytes, void* d_out,
                        void* stream) {
    using namespace sbh;
    clear_error();
    if (n == 0) return SBH_OK;
    if (!d_ptrs || !d_col || !d_out) { set_error("null pointer"); return SBH_EINVAL; }
    if (col_bytes != 4 && col_bytes != 8) { set_error("col_bytes must be 4 or 8"); return SBH_EINVAL; }
    if (n > 0xFFFFFFFFull) { set_error("n must be < 2^32"); return SBH_EINVAL; }
    cudaStream_t s = as_stream(stream);
    const unsigned grid = (unsigned)min_u64((n + 1023) / 1024, (uint64_t)num_sms() * 8);
    if (col_bytes == 8)
        SBH_TIMED("materialize", s, gather_kernel<uint64_t><<<grid, 256, 0, s>>>(
                                        d_ptrs, (uint32_t)n, static_cast<const uint64_t*>(d_col),
                                        static_cast<uint64_t*>(d_out)));
    else
        SBH_TIMED("materialize", s, gather_kernel<uint32_t><<<grid, 256, 0, s>>>(
                                        d_ptrs, (uint32_t)n, static_cast<const uint32_t*>(d_col),
                                        static_cast<uint32_t*>(d_out)));
    SBH_LAUNCHED();
    return SBH_OK;
}

int sbh_copy_counted(const void* d_src, void* dst, int elem_bytes, int dst_bytes, const uint64_t* d_count,
                     uint64_t per, uint64_t cap, void* stream) {
    using namespace sbh;
    clear_error();
    if (!d_src || !dst || !d_count) { set_error("null pointer"); return SBH_EINVAL; }
    if (elem_bytes != 1 && elem_bytes != 4 && elem_bytes != 8) { set_error("elem_bytes must be 1, 4 or 8"); return SBH_EINVAL; }
    if (dst_bytes != elem_bytes && !(elem_bytes == 8 && dst_bytes == 4)) {
        set_error("dst_bytes must equal elem_bytes, or be 4 when elem_bytes is 8");
        return SBH_EINVAL;
    }
    if (per == 0 || cap == 0) return SBH_OK;
    cudaStream_t s = as_stream(stream);
    const unsigned grid = (unsigned)min_u64((cap * per + 255) / 256, (uint64_t)num_sms() * 8);
    if (elem_bytes == 8 && dst_bytes == 4)
        SBH_TIMED("copy_counted", s, (copy_counted_kernel<uint64_t, uint32_t><<<grid, 256, 0, s>>>(
                                         static_cast<const uint64_t*>(d_src), static_cast<uint32_t*>(dst), d_count,
                                         per, cap)));
    else if (elem_bytes == 8)
        SBH_TIMED("copy_counted", s, (copy_counted_kernel<uint64_t, uint64_t><<<grid, 256, 0, s>>>(
                                         static_cast<const uint64_t*>(d_src), static_cast<uint64_t*>(dst), d_count,
                                         per, cap)));
    else if (elem_bytes == 4)
        SBH_TIMED("copy_counted", s, (copy_counted_kernel<uint32_t, uint32_t><<<grid, 256, 0, s>>>(
                                         static_cast<const uint32_t*>(d_src), static_cast<uint32_t*>(dst), d_count,
                                         per, cap)));
    else
        SBH_TIMED("copy_counted", s, (copy_counted_kernel<uint8_t, uint8_t><<<grid, 256, 0, s>>>(
                                         static_cast<const uint8_t*>(d_src), static_cast<uint8_t*>(dst), d_count,
                                         per, cap)));
    SBH_LAUNCHED();
    return SBH_OK;
}

int sbh_kpa_keyswap(const uint32_t* d_ptrs, uint64_t n, const uint64_t* d_key_col, uint64_t* d_keys_out,
                    void* stream) {
    return sbh_kpa_materialize(d_ptrs, n, d_key_col, 8, d_keys_out, stream);
}

int sbh_kpa_keyswap_lookup(const uint32_t* d_ptrs, uint64_t n, const uint64_t* d_col, const uint64_t* d_table,
                           uint64_t table_len, uint64_t* d_keys_out, uint64_t* d_misses, void* stream) {
    using namespace sbh;
    clear_error();
    if (n == 0) return SBH_OK;
    if (!d_ptrs || !d_col || !d_keys_out || (table_len && !d_table)) { set_error("null pointer"); return SBH_EINVAL; }
    if (n > 0xFFFFFFFFull) { set_error("n must be < 2^32"); return SBH_EINVAL; }
    cudaStream_t s = as_stream(stream);
    const unsigned grid = (unsigned)min_u64((n + 1023) / 1024, (uint64_t)num_sms() * 8);
    SBH_TIMED("keyswap_lookup", s,
              lookup_kernel<<<grid, 256, 0, s>>>(d_ptrs, (uint32_t)n, d_col, d_table, table_len, d_keys_out,
                                                 reinterpret_cast<unsigned long long*>(d_misses)));
    SBH_LAUNCHED();
    return SBH_OK;
}

int sbh_kpa_select(const uint64_t* d_keys, const uint32_t* d_ptrs, uint64_t n, const void* d_col, int col_bytes,
                   uint64_t lo, uint64_t hi, uint64_t* d_out_keys, uint32_t* d_out_ptrs, uint64_t cap,
                   uint64_t* d_count, void* d_scratch, size_t* scratch_bytes, void* stream) {
    using namespace sbh;
    clear_error();
    if (n > 0xFFFFFFFFull) { set_error("n must be < 2^32"); return SBH_EINVAL; }
    const uint64_t ntiles = (n + kSelTile - 1) / kSelTile;
    bool done = false;
    int rc = scratch_check(d_scratch, scratch_bytes, (ntiles ? ntiles : 1) * sizeof(uint32_t), &done);
    if (rc || done) return rc;
    if (!d_count) { set_error("d_count is NULL"); return SBH_EINVAL; }
    cudaStream_t s = as_stream(stream);
    if (n == 0) {
        SBH_CUDA(cudaMemsetAsync(d_count, 0, sizeof(uint64_t), s));
        return SBH_OK;
    }
    if (!d_keys || !d_ptrs || !d_col || (cap && (!d_out_keys || !d_out_ptrs))) {
        set_error("null pointer");
        return SBH_EINVAL;
    }
    if (col_bytes != 4 && col_bytes != 8) { set_error("col_bytes must be 4 or 8"); return SBH_EINVAL; }
    uint32_t* cnt = static_cast<uint32_t*>(d_scratch);
    if (col_bytes == 8)
        return select_run<uint64_t>(d_keys, d_ptrs, (uint32_t)n, d_col, lo, hi, d_out_keys, d_out_ptrs, cap, d_count,
                                    cnt, s);
    return select_run<uint32_t>(d_keys, d_ptrs, (uint32_t)n, d_col, lo, hi, d_out_keys, d_out_ptrs, cap, d_count, cnt,
                                s);
}

}  // extern "C"
