// Kernel instrumentation: every launch of the library's kernels is counted under
// a name together with its algorithmic bytes (the minimum HBM traffic of that
// launch); when timing is enabled, each launch is also bracketed by CUDA events
// recorded on its own stream.
#pragma once
#include <cuda_runtime.h>

#include <utility>
#include <vector>

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

// Launches recorded while a stream is captured into a CUDA graph: the capture does
// not run them, each replay of the graph does.
struct ProfRecord {
    std::vector<std::pair<int, double>> items;  // (entry, bytes) per captured launch
};
// While active on this thread, ProfScope appends to *rec instead of counting.
void prof_record_begin(ProfRecord *rec);
void prof_record_end();
// Counts one replay of a recorded block.
void prof_replay(const ProfRecord &rec);
bool prof_timing();

void prof_enable(bool on);
// While timing is on (and not while capturing a graph): a device counter, in bytes, for the
// entry `name`, which kernels whose traffic depends on device state (RHS that have stopped
// move nothing) add to; prof_read folds it into the entry's bytes.  nullptr otherwise: the
// caller then charges its host-side estimate.
unsigned long long *prof_device_bytes(const char *name);
void prof_reset();
// Synchronises the device, folds pending event pairs into the totals.
int prof_read(KernelStat *out, int max);
// Measured FMA throughput (TFLOP/s) in FP64 (prec 64) or FP32 (prec 32); synchronises s.
cudaError_t alu_peak(int prec, double *tflops, cudaStream_t s);

}  // namespace eig
