// Library-wide state: error text, the per-device status word, test hooks.
#include <atomic>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "common.cuh"

namespace {

thread_local char g_err[512] = {0};

// Bit 0: a bounded device-side wait expired.  One word per device (a
// __device__ variable exists once in every context that loads the library).
__device__ uint32_t g_status_word = 0;

constexpr int kMaxDevices = 64;
std::mutex g_mu;
uint32_t* g_status_ptr[kMaxDevices] = {nullptr};
int g_sms[kMaxDevices] = {0};

constexpr uint32_t kDefaultSpinLimit = 1u << 22;  // a few seconds of polls
std::atomic<uint32_t> g_spin_limit{kDefaultSpinLimit};
// tuning knobs (sbh_set_knob): the sorts' chunked-pass threshold and the
// merges' separate cut-search threshold
std::atomic<uint64_t> g_knob[SBH_KNOB_COUNT] = {{1ull << 23}, {2047}, {0}};  // measured on B300
std::atomic<int> g_fault{SBH_FAULT_NONE};

struct ProfRecord {
    std::string name;
    cudaEvent_t start, stop;
};
std::mutex g_prof_mu;
std::atomic<int> g_prof_on{0};
std::vector<ProfRecord> g_prof;

int current_device() {
    int d = 0;
    if (cudaGetDevice(&d) != cudaSuccess || d < 0 || d >= kMaxDevices) return -1;
    return d;
}

}  // namespace

namespace sbh {

void set_error(const char* fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
}

void clear_error() { g_err[0] = 0; }

uint32_t* status_word() {
    int d = current_device();
    if (d < 0) return nullptr;
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_status_ptr[d]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_status_word) != cudaSuccess) return nullptr;
        g_status_ptr[d] = static_cast<uint32_t*>(p);
    }
    return g_status_ptr[d];
}

uint32_t spin_limit() { return g_spin_limit.load(); }

uint64_t knob(int k) { return (k >= 0 && k < SBH_KNOB_COUNT) ? g_knob[k].load() : 0; }

int take_fault() { return g_fault.exchange(SBH_FAULT_NONE); }

int num_sms() {
    int d = current_device();
    if (d < 0) return 148;
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_sms[d]) {
        int v = 0;
        if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, d) != cudaSuccess || v <= 0) v = 148;
        g_sms[d] = v;
    }
    return g_sms[d];
}

ProfScope::ProfScope(const char* name, cudaStream_t s) : stream(s) {
    if (!g_prof_on.load()) return;
    ProfRecord r;
    r.name = name;
    if (cudaEventCreate(&r.start) != cudaSuccess) return;
    if (cudaEventCreate(&r.stop) != cudaSuccess) { cudaEventDestroy(r.start); return; }
    cudaEventRecord(r.start, s);
    std::lock_guard<std::mutex> lk(g_prof_mu);
    slot = static_cast<int>(g_prof.size());
    g_prof.push_back(r);
}

ProfScope::~ProfScope() {
    if (slot < 0) return;
    std::lock_guard<std::mutex> lk(g_prof_mu);
    cudaEventRecord(g_prof[slot].stop, stream);
}

}  // namespace sbh

extern "C" {

int sbh_set_knob(int k, uint64_t value) {
    using namespace sbh;
    clear_error();
    if (k < 0 || k >= SBH_KNOB_COUNT) { set_error("unknown knob %d", k); return SBH_EINVAL; }
    if (k == SBH_KNOB_SCATTER_GEOM && value > 2) { set_error("scatter geometry must be 0, 1 or 2"); return SBH_EINVAL; }
    g_knob[k].store(value);
    return SBH_OK;
}

uint64_t sbh_get_knob(int k) { return sbh::knob(k); }

void sbh_profile_enable(int on) {
    std::lock_guard<std::mutex> lk(g_prof_mu);
    for (auto& r : g_prof) { cudaEventDestroy(r.start); cudaEventDestroy(r.stop); }
    g_prof.clear();
    g_prof_on.store(on ? 1 : 0);
}

int sbh_profile_collect(int max_records, char* names, int name_len, double* ms) {
    std::lock_guard<std::mutex> lk(g_prof_mu);
    const int n = static_cast<int>(g_prof.size());
    for (int i = 0; i < n && i < max_records; ++i) {
        float t = 0.f;
        cudaEventSynchronize(g_prof[i].stop);
        if (cudaEventElapsedTime(&t, g_prof[i].start, g_prof[i].stop) != cudaSuccess) t = -1.f;
        if (ms) ms[i] = t;
        if (names && name_len > 0) {
            std::strncpy(names + (size_t)i * name_len, g_prof[i].name.c_str(), name_len - 1);
            names[(size_t)i * name_len + name_len - 1] = 0;
        }
    }
    return n;
}

const char* sbh_version(void) { return "sbh 0.1 (sm_103a)"; }

const char* sbh_last_error(void) { return g_err; }

void sbh_set_spin_limit(uint32_t polls) { g_spin_limit.store(polls ? polls : kDefaultSpinLimit); }

void sbh_set_fault(int fault) { g_fault.store(fault); }

int sbh_sync_status(void* stream) {
    sbh::clear_error();
    uint32_t* w = sbh::status_word();
    if (!w) {
        sbh::set_error("cannot resolve the device status word");
        return SBH_ECUDA;
    }
    cudaStream_t s = sbh::as_stream(stream);
    uint32_t host = 0;
    SBH_CUDA(cudaMemcpyAsync(&host, w, sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
    SBH_CUDA(cudaMemsetAsync(w, 0, sizeof(uint32_t), s));
    SBH_CUDA(cudaStreamSynchronize(s));
    if (host & sbh::kStatusTimeout) {
        sbh::set_error("a device-side wait expired; the output of the affected call is invalid");
        return SBH_ETIMEOUT;
    }
    return SBH_OK;
}

}  // extern "C"
