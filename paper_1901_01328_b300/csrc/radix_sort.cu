// A3 Sort: stable LSD radix sort of a KPA (uint64 key, uint32 ptr) by the
// key, 8-bit digits; the passes are described in radix_core.cuh.
#include "radix_core.cuh"

namespace sbh {

size_t radix_sort_scratch(uint64_t n) { return sort_carve(nullptr, n).total; }

}  // namespace sbh

extern "C" int sbh_kpa_sort(const uint64_t* d_keys_in, const uint32_t* d_ptrs_in, uint64_t* d_keys_out,
                            uint32_t* d_ptrs_out, uint64_t n, void* d_scratch, size_t* scratch_bytes, void* stream) {
    using namespace sbh;
    clear_error();
    if (n > 0xFFFFFFFFull) { set_error("n must be < 2^32"); return SBH_EINVAL; }
    bool done = false;
    int rc = scratch_check(d_scratch, scratch_bytes, radix_sort_scratch(n), &done);
    if (rc || done) return rc;
    if (n == 0) return SBH_OK;
    if (!d_keys_in || !d_keys_out || !d_ptrs_out) { set_error("null pointer"); return SBH_EINVAL; }
    if (!d_ptrs_in && d_keys_in == d_keys_out) { set_error("row-number ptrs need a separate output"); return SBH_EINVAL; }
    return sort_by_value(d_keys_in, d_ptrs_in, d_keys_out, d_ptrs_out, n, d_scratch, as_stream(stream), RadixValue{},
                         kPositions);
}
