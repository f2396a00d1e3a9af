// Shared host and device helpers of the KPA grouping library (sm_103a).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <cstdarg>
#include <cstddef>

#include "sbh.h"

namespace sbh {

// ------------------------------------------------------------------ host side
void set_error(const char* fmt, ...);
void clear_error();

// Device pointer of this library's per-device status word (bit 0: a bounded
// device wait expired).  Looked up once per device.
uint32_t* status_word();
// Current number of polls a device-side wait makes before giving up.
uint32_t spin_limit();
// Returns the pending fault hook and clears it.
int take_fault();
// Number of SMs of the current device.
int num_sms();
// Current value of a tuning knob (SBH_KNOB_*).
uint64_t knob(int k);

// Optional per-launch timing (sbh_profile_enable): a scope records a CUDA
// event pair around the launches it encloses, on their stream.
struct ProfScope {
    int slot = -1;
    cudaStream_t stream;
    ProfScope(const char* name, cudaStream_t s);
    ~ProfScope();
};

__host__ __device__ __forceinline__ uint64_t min_u64(uint64_t a, uint64_t b) { return a < b ? a : b; }

inline cudaStream_t as_stream(void* s) { return reinterpret_cast<cudaStream_t>(s); }

// Checks a CUDA call; records the error text and returns SBH_ECUDA on failure.
#define SBH_CUDA(call)                                                                       \
    do {                                                                                     \
        cudaError_t e_ = (call);                                                             \
        if (e_ != cudaSuccess) {                                                             \
            ::sbh::set_error("%s: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__, __LINE__); \
            return SBH_ECUDA;                                                                \
        }                                                                                    \
    } while (0)

// Runs a kernel launch inside a profiling scope named `name`.
#define SBH_TIMED(name, stream, ...)             \
    do {                                         \
        ::sbh::ProfScope ps_((name), (stream));  \
        __VA_ARGS__;                             \
    } while (0)

// Checks the last launch.
#define SBH_LAUNCHED() SBH_CUDA(cudaGetLastError())

// Carves 256-byte aligned pieces out of one scratch buffer.  With base ==
// nullptr it only measures.
struct Carver {
    char* base;
    size_t off = 0;
    explicit Carver(void* b) : base(static_cast<char*>(b)) {}
    template <typename T>
    T* take(size_t count) {
        off = (off + 255) & ~size_t(255);
        T* p = base ? reinterpret_cast<T*>(base + off) : nullptr;
        off += count * sizeof(T);
        return p;
    }
    size_t bytes() const { return (off + 255) & ~size_t(255); }
};

// Common scratch-protocol check.  Returns SBH_OK and sets *done when the call
// was only a size query.
inline int scratch_check(void* scratch, size_t* scratch_bytes, size_t need, bool* done) {
    *done = false;
    if (!scratch_bytes) {
        set_error("scratch_bytes is NULL");
        return SBH_EINVAL;
    }
    if (!scratch) {
        *scratch_bytes = need;
        *done = true;
        return SBH_OK;
    }
    if (*scratch_bytes < need) {
        set_error("scratch too small: %zu < %zu bytes", *scratch_bytes, need);
        return SBH_ENOSPACE;
    }
    if (reinterpret_cast<uintptr_t>(scratch) & 255) {
        set_error("scratch is not 256-byte aligned");
        return SBH_EINVAL;
    }
    return SBH_OK;
}

// ---------------------------------------------------------------- device side
constexpr uint32_t kStatusTimeout = 1u;

__device__ __forceinline__ uint64_t ld_acquire(const uint64_t* p) {
    uint64_t v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ uint32_t ld_acquire(const uint32_t* p) {
    uint32_t v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release(uint64_t* p, uint64_t v) {
    asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ void st_release(uint32_t* p, uint32_t v) {
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ void st_relaxed(uint64_t* p, uint64_t v) {
    asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ uint64_t ld_relaxed(const uint64_t* p) {
    uint64_t v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ uint32_t ld_relaxed(const uint32_t* p) {
    uint32_t v;
    asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void record_timeout(uint32_t* status) {
    if (status) atomicOr(status, kStatusTimeout);
}

// One poll of a bounded wait.  Returns true when the wait must give up: its
// own budget is spent, or (checked every 256 polls) another wait of this
// library already gave up, so that one stuck tile cannot make every later
// tile wait out a full budget.
__device__ __forceinline__ bool wait_expired(uint32_t& polls, uint32_t limit, uint32_t* status) {
    ++polls;
    if (polls > limit) {
        record_timeout(status);
        return true;
    }
    if ((polls & 255u) == 0 && status && (ld_relaxed(status) & kStatusTimeout)) return true;
    if (polls > 8) __nanosleep(32);
    return false;
}

__device__ __forceinline__ uint32_t lane_id() { return threadIdx.x & 31u; }
__device__ __forceinline__ uint32_t lanemask_lt() {
    uint32_t m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

// ---- shared-memory barriers and bulk (TMA) copies
__device__ __forceinline__ uint32_t smem_addr(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
// Orders earlier generic-proxy accesses to shared memory before later
// async-proxy (bulk copy) writes to it.
__device__ __forceinline__ void fence_proxy_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes) : "memory");
}
// 1-D bulk copy global -> shared, completing `bytes` on the barrier.  dst,
// src and bytes must be multiples of 16.
__device__ __forceinline__ void bulk_load(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_addr(dst)),
                 "l"(src), "r"(bytes), "r"(smem_addr(bar))
                 : "memory");
}
// L2 eviction-priority policies (createpolicy) for the cache_hint forms below.
__device__ __forceinline__ uint64_t l2_evict_first() {
    uint64_t pol;
    asm("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
    return pol;
}
__device__ __forceinline__ uint64_t l2_evict_last() {
    uint64_t pol;
    asm("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(pol));
    return pol;
}
// bulk_load with an L2 policy for the source lines.
__device__ __forceinline__ void bulk_load(void* dst, const void* src, uint32_t bytes, uint64_t* bar, uint64_t pol) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1], %2, [%3], %4;" ::"r"(
            smem_addr(dst)),
        "l"(src), "r"(bytes), "r"(smem_addr(bar)), "l"(pol)
        : "memory");
}
// One-byte global store with an L2 policy for its line.
__device__ __forceinline__ void st_hint(uint8_t* p, uint32_t v, uint64_t pol) {
    asm volatile("st.global.L2::cache_hint.u8 [%0], %1, %2;" ::"l"(p), "r"(v), "l"(pol));
}
// Per-thread asynchronous copies global -> shared of 4 or 8 bytes (both
// addresses aligned to the size); complete for the issuing thread after
// cp_async_wait_all.
__device__ __forceinline__ void cp_async8(void* dst, const void* src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(smem_addr(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async4(void* dst, const void* src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(smem_addr(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Waits for the bulk copies completing the given phase of a barrier in this
// CTA's shared memory.  A copy from this GPU's memory always lands, so unlike
// the waits on other CTAs this one never gives up because another wait of the
// library did: only its own poll budget bounds it.  Returns false (and records
// a timeout) when that budget ran out; the copy may then still be in flight,
// and the CTA must drain it (mbar_drain) before it leaves.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity, uint32_t limit, uint32_t* status) {
    uint32_t polls = 0;
    while (!mbar_try_wait(bar, parity)) {
        if (++polls > limit) {
            record_timeout(status);
            return false;
        }
        if (polls > 8) __nanosleep(32);
    }
    return true;
}

// Lets a bulk copy that an expired wait left behind land before the CTA
// leaves, so that it cannot write into shared memory that the SM has given to
// the next CTA.  Bounded by its own budget (about a second), independent of
// the test hook that shortens the other waits.
constexpr uint32_t kDrainPolls = 1u << 24;
__device__ __forceinline__ void mbar_drain(uint64_t* bar, uint32_t parity) {
    for (uint32_t polls = 0; !mbar_try_wait(bar, parity) && polls < kDrainPolls; ++polls)
        if (polls > 8) __nanosleep(64);
}

// Shared-memory atomic add done only where pred holds, without a branch
// (returns the old value there, 0 elsewhere).
__device__ __forceinline__ uint32_t smem_atomic_add_if(bool pred, uint32_t* addr, uint32_t v) {
    uint32_t old = 0;
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.u32 p, %2, 0;\n @p atom.shared.add.u32 %0, [%1], %3;\n}\n"
        : "+r"(old)
        : "r"(smem_addr(addr)), "r"(static_cast<uint32_t>(pred)), "r"(v)
        : "memory");
    return old;
}

// The same without a compiler memory barrier, so that independent loads and
// arithmetic may be scheduled around it; the counters it updates must be
// read only after a CTA barrier.
__device__ __forceinline__ uint32_t smem_atomic_add_if_relaxed(bool pred, uint32_t* addr, uint32_t v) {
    uint32_t old = 0;
    asm volatile("{\n .reg .pred p;\n setp.ne.u32 p, %2, 0;\n @p atom.shared.add.u32 %0, [%1], %3;\n}\n"
                 : "+r"(old)
                 : "r"(smem_addr(addr)), "r"(static_cast<uint32_t>(pred)), "r"(v));
    return old;
}

// Streaming (evict-first) loads and stores for data touched once.
__device__ __forceinline__ uint64_t ld_stream(const uint64_t* p) { return __ldcs(reinterpret_cast<const unsigned long long*>(p)); }
__device__ __forceinline__ uint32_t ld_stream(const uint32_t* p) { return __ldcs(reinterpret_cast<const unsigned int*>(p)); }
__device__ __forceinline__ void st_stream(uint64_t* p, uint64_t v) { __stcs(reinterpret_cast<unsigned long long*>(p), (unsigned long long)v); }
__device__ __forceinline__ void st_stream(uint32_t* p, uint32_t v) { __stcs(reinterpret_cast<unsigned int*>(p), v); }

}  // namespace sbh
