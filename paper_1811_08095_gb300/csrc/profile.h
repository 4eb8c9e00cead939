// Optional per-kernel timing of the solver's launches (off by default).
//
// When enabled, every profiled launch is bracketed by two CUDA events recorded on the
// launching stream; elapsed times are collected after the stream synchronizes.  Each
// profiled kernel also counts, on the device, how many (system, launch) pairs actually
// ran (a gated system exits before the counter), so algorithmic bytes can be computed
// exactly for batched launches.
#pragma once

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <string>

namespace odwf {

struct ProfSlot {
    int cls = -1;                          // kernel class index (-1: profiling off)
    cudaEvent_t start = nullptr, stop = nullptr;
    unsigned long long* dev_count = nullptr;  // device counter of running systems
};

bool prof_enabled();
// Register (or find) a kernel class with its algorithmic bytes per running system and per
// launch (shared data such as links); returns its index.
int prof_class(const std::string& name, double bytes_per_system, double bytes_per_launch);
ProfSlot prof_begin(int cls, cudaStream_t s);
void prof_end(const ProfSlot& slot, cudaStream_t s);
void prof_collect();  // after a stream synchronize: accumulate finished event pairs

// Scoped per-launch timing of one kernel class with its algorithmic bytes per launch (a no-op
// when profiling is off); the launcher counts the launch itself.
struct ProfScope {
    ProfSlot slot;
    cudaStream_t st;
    ProfScope(const char* name, double bytes_per_launch, cudaStream_t s) : st(s) {
        slot = prof_begin(prof_enabled() ? prof_class(name, 0.0, bytes_per_launch) : -1, s);
    }
    ~ProfScope() { prof_end(slot, st); }
    ProfScope(const ProfScope&) = delete;
    ProfScope& operator=(const ProfScope&) = delete;
};

// NVTX range for the solver's host-side phases (iteration chunks, reliable updates, admission,
// finalization, serving passes): visible in Nsight tools, a no-op without one.
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange&) = delete;
    NvtxRange& operator=(const NvtxRange&) = delete;
};

}  // namespace odwf
