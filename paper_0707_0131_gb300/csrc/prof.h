// Kernel instrumentation: every launch of the library's kernels is counted under
// a name together with its algorithmic bytes (the minimum HBM traffic of that
// launch); when timing is enabled, each launch is also bracketed by CUDA events
// recorded on its own stream.
#pragma once
#include <cuda_runtime.h>

namespace eig {

struct ProfScope {
    ProfScope(const char *name, double bytes, cudaStream_t s);
    ~ProfScope();
    int slot;
    int ev;
    cudaStream_t stream;
};

struct KernelStat {
    char name[40];
    long launches;
    double ms;
    double bytes;
};

void prof_enable(bool on);
void prof_reset();
// Synchronises the device, folds pending event pairs into the totals.
int prof_read(KernelStat *out, int max);

}  // namespace eig
