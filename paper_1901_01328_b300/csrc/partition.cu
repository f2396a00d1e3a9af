// Partition (Table 2: split a KPA into sub-KPAs by ranges of its resident
// keys).  The part of a key is the number of range bounds not above it, so a
// stable sort of the KPA by that part number is the partition: the parts lie
// end to end, each in the input order.  The sort is the radix machinery of
// radix_core.cuh with the part number as the value (one 8-bit pass for up to
// 256 parts, two for up to 65536, ...), and a last pass over the output keys
// records where each part starts.
#include "radix_core.cuh"

namespace sbh {
namespace {

// Number of bounds <= k (binary search over the non-decreasing bounds; they
// are few and stay in L1).
struct PartOf {
    const uint64_t* bounds;
    uint32_t nb;
    __device__ __forceinline__ uint64_t operator()(uint64_t k) const {
        uint32_t lo = 0, hi = nb;
        while (lo < hi) {
            const uint32_t mid = (lo + hi) / 2;
            if (__ldg(bounds + mid) <= k) lo = mid + 1;
            else hi = mid;
        }
        return lo;
    }
};

// offsets[j] = first output row of part j (j <= nb + 1, offsets[nb + 1] = n):
// row i writes the offsets of the parts after the previous row's part up to
// its own; the thread past the last row fills the rest with n.
__global__ void __launch_bounds__(256) part_offsets_kernel(const uint64_t* __restrict__ keys, uint32_t n, PartOf fn,
                                                           uint64_t* __restrict__ offsets) {
    const uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
    if (i > n) return;
    const uint64_t cur = i < n ? fn(keys[i]) : (uint64_t)fn.nb + 1;
    const uint64_t first = i > 0 ? fn(keys[i - 1]) + 1 : 0;
    for (uint64_t p = first; p <= cur; ++p) offsets[p] = i;
}

int part_digits(uint64_t nb) {  // 8-bit digits of the largest part number, nb
    int d = 0;
    for (uint64_t v = nb; v; v >>= 8) ++d;
    return d;
}

}  // namespace
}  // namespace sbh

extern "C" int sbh_kpa_partition(const uint64_t* d_keys, const uint32_t* d_ptrs, uint64_t n,
                                 const uint64_t* d_bounds, uint64_t nb, uint64_t* d_keys_out, uint32_t* d_ptrs_out,
                                 uint64_t* d_offsets, void* d_scratch, size_t* scratch_bytes, void* stream) {
    using namespace sbh;
    clear_error();
    if (n > 0xFFFFFFFFull) { set_error("n must be < 2^32"); return SBH_EINVAL; }
    if (nb >= 0xFFFFFFFFull) { set_error("at most 2^32 - 2 bounds"); return SBH_EINVAL; }
    bool done = false;
    int rc = scratch_check(d_scratch, scratch_bytes, sort_carve(nullptr, n).total, &done);
    if (rc || done) return rc;
    if (!d_offsets || (nb && !d_bounds)) { set_error("null pointer"); return SBH_EINVAL; }
    if (n && (!d_keys || !d_ptrs || !d_keys_out || !d_ptrs_out)) { set_error("null pointer"); return SBH_EINVAL; }
    cudaStream_t s = as_stream(stream);
    const PartOf fn{d_bounds, static_cast<uint32_t>(nb)};
    if (n) {
        const int npos = part_digits(nb);
        if (npos == 0) {  // one part: the KPA itself
            if (d_keys_out != d_keys)
                SBH_CUDA(cudaMemcpyAsync(d_keys_out, d_keys, n * sizeof(uint64_t), cudaMemcpyDeviceToDevice, s));
            if (d_ptrs_out != d_ptrs)
                SBH_CUDA(cudaMemcpyAsync(d_ptrs_out, d_ptrs, n * sizeof(uint32_t), cudaMemcpyDeviceToDevice, s));
        } else {
            rc = sort_by_value(d_keys, d_ptrs, d_keys_out, d_ptrs_out, n, d_scratch, s, fn, npos, "partition");
            if (rc) return rc;
        }
    }
    SBH_TIMED("partition_offsets", s,
              part_offsets_kernel<<<(unsigned)(n / 256 + 1), 256, 0, s>>>(d_keys_out, (uint32_t)n, fn, d_offsets));
    SBH_LAUNCHED();
    return SBH_OK;
}
