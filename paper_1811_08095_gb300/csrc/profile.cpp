// Per-kernel timing registry behind odwf_profile_enable / odwf_profile_read.
#include "profile.h"

#include <cstring>
#include <mutex>
#include <vector>

#include "../../include/odwf.h"
#include "kernels.h"

namespace odwf {

int fail(int code, const std::string& msg);

namespace {

constexpr int kMaxClasses = 64;

struct ClassInfo {
    std::string name;
    double bytes_per_system = 0, bytes_per_launch = 0;
    long long launches = 0;
    double total_ms = 0;
};

struct Pending {
    int cls;
    cudaEvent_t a, b;
};

struct Registry {
    std::mutex mu;
    bool enabled = false;
    std::vector<ClassInfo> classes;
    std::vector<Pending> pending;
    std::vector<cudaEvent_t> free_events;
    unsigned long long* dev_counts = nullptr;  // [kMaxClasses]
};

Registry& reg() {
    static Registry r;
    return r;
}

cudaEvent_t get_event(Registry& R) {
    if (!R.free_events.empty()) {
        cudaEvent_t e = R.free_events.back();
        R.free_events.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

void collect_locked(Registry& R) {
    for (auto& p : R.pending) {
        cudaEventSynchronize(p.b);
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, p.a, p.b) == cudaSuccess && p.cls >= 0 && p.cls < (int)R.classes.size()) {
            R.classes[p.cls].launches += 1;
            R.classes[p.cls].total_ms += ms;
        }
        R.free_events.push_back(p.a);
        R.free_events.push_back(p.b);
    }
    R.pending.clear();
}

}  // namespace

bool prof_enabled() { return reg().enabled; }

int prof_class(const std::string& name, double bytes_per_system, double bytes_per_launch) {
    Registry& R = reg();
    std::lock_guard<std::mutex> g(R.mu);
    for (size_t i = 0; i < R.classes.size(); ++i)
        if (R.classes[i].name == name) return (int)i;
    if ((int)R.classes.size() >= kMaxClasses) return -1;
    ClassInfo c;
    c.name = name;
    c.bytes_per_system = bytes_per_system;
    c.bytes_per_launch = bytes_per_launch;
    R.classes.push_back(c);
    return (int)R.classes.size() - 1;
}

ProfSlot prof_begin(int cls, cudaStream_t s) {
    ProfSlot slot;
    Registry& R = reg();
    if (!R.enabled || cls < 0) return slot;
    std::lock_guard<std::mutex> g(R.mu);
    slot.cls = cls;
    slot.start = get_event(R);
    slot.stop = get_event(R);
    slot.dev_count = R.dev_counts ? R.dev_counts + cls : nullptr;
    cudaEventRecord(slot.start, s);
    return slot;
}

void prof_end(const ProfSlot& slot, cudaStream_t s) {
    if (slot.cls < 0) return;
    Registry& R = reg();
    std::lock_guard<std::mutex> g(R.mu);
    cudaEventRecord(slot.stop, s);
    R.pending.push_back({slot.cls, slot.start, slot.stop});
}

void prof_collect() {
    Registry& R = reg();
    if (!R.enabled) return;
    std::lock_guard<std::mutex> g(R.mu);
    collect_locked(R);
}

}  // namespace odwf

using odwf::fail;

extern "C" {

int odwf_profile_enable(int on) {
    auto& R = odwf::reg();
    std::lock_guard<std::mutex> g(R.mu);
    odwf::collect_locked(R);
    if (on) {
        if (!R.dev_counts) {
            if (cudaMalloc(&R.dev_counts, sizeof(unsigned long long) * odwf::kMaxClasses) != cudaSuccess) {
                cudaGetLastError();
                R.dev_counts = nullptr;
                return fail(ODWF_ENOMEM, "odwf_profile_enable: device allocation failed");
            }
        }
        if (cudaMemset(R.dev_counts, 0, sizeof(unsigned long long) * odwf::kMaxClasses) != cudaSuccess)
            return fail(ODWF_ECUDA, "odwf_profile_enable: memset failed");
        for (auto& c : R.classes) {
            c.launches = 0;
            c.total_ms = 0;
        }
    }
    R.enabled = on != 0;
    return ODWF_OK;
}

long long odwf_launch_count(void) { return odwf::launch_count(); }

int odwf_profile_read(odwf_kernel_prof* out, int max_entries, int* n_out) {
    if (!out || !n_out || max_entries < 0) return fail(ODWF_EINVAL, "odwf_profile_read: bad arguments");
    auto& R = odwf::reg();
    std::lock_guard<std::mutex> g(R.mu);
    if (cudaDeviceSynchronize() != cudaSuccess) return fail(ODWF_ECUDA, "odwf_profile_read: device error");
    odwf::collect_locked(R);
    unsigned long long counts[odwf::kMaxClasses] = {0};
    if (R.dev_counts &&
        cudaMemcpy(counts, R.dev_counts, sizeof(counts), cudaMemcpyDeviceToHost) != cudaSuccess)
        return fail(ODWF_ECUDA, "odwf_profile_read: copy failed");
    int n = 0;
    for (size_t i = 0; i < R.classes.size() && n < max_entries; ++i) {
        const auto& c = R.classes[i];
        if (c.launches == 0) continue;
        odwf_kernel_prof& o = out[n++];
        std::memset(&o, 0, sizeof(o));
        std::strncpy(o.name, c.name.c_str(), sizeof(o.name) - 1);
        o.launches = c.launches;
        o.system_launches = (int64_t)counts[i];
        o.total_ms = c.total_ms;
        o.bytes_per_system = c.bytes_per_system;
        o.bytes_per_launch = c.bytes_per_launch;
    }
    *n_out = n;
    return ODWF_OK;
}

}  // extern "C"
