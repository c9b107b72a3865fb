// Per-phase device timing with CUDA events recorded on the launch stream
// (disabled unless fds_timing_enable(1) was called).  A ProfScope brackets
// one launch or a short group of launches under a name; work counts (flops or
// bytes of the algorithm) may be attached for roofline reporting.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

bool prof_enabled();
// timing is suspended on the calling thread while it captures a CUDA graph
// (the events would belong to the graph, not to this launch)
void prof_set_capturing(bool on);
struct ProfCaptureScope {
    ProfCaptureScope() { prof_set_capturing(true); }
    ~ProfCaptureScope() { prof_set_capturing(false); }
};
void prof_begin(const char *name, cudaStream_t s);
void prof_end(cudaStream_t s, double flops, double bytes, double units);
// work of a phase known only after its launches ran (e.g. from the ranks the
// ID found): added to the phase's totals without a launch or a time
void prof_add_work(const char *name, double flops, double bytes, double units);

struct ProfScope {
    cudaStream_t s;
    double flops = 0, bytes = 0, units = 0;
    bool on;
    ProfScope(const char *name, cudaStream_t st) : s(st), on(prof_enabled()) {
        if (on) prof_begin(name, s);
    }
    ~ProfScope() {
        if (on) prof_end(s, flops, bytes, units);
    }
};
