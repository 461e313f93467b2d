#include "prof.h"

#include <cstring>
#include <mutex>
#include <string>
#include <vector>

namespace eig {

namespace {
struct Entry {
    std::string name;
    long launches = 0;
    double ms = 0.0;
    double bytes = 0.0;
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> pending;
};
std::mutex g_mu;
std::vector<Entry> g_entries;
std::vector<cudaEvent_t> g_pool;
bool g_timing = false;
thread_local ProfRecord *g_rec = nullptr;
// bytes counted on the device by kernels whose traffic depends on device state (one
// counter per entry slot); allocated when timing is first enabled
constexpr int MAX_DEV = 64;
unsigned long long *g_dev = nullptr;

int slot_of(const char *name) {
    for (size_t i = 0; i < g_entries.size(); i++)
        if (g_entries[i].name == name) return (int)i;
    g_entries.push_back(Entry());
    g_entries.back().name = name;
    return (int)g_entries.size() - 1;
}

cudaEvent_t get_event() {
    if (!g_pool.empty()) {
        cudaEvent_t e = g_pool.back();
        g_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}
}  // namespace

ProfScope::ProfScope(const char *name, double bytes, cudaStream_t s) : slot(-1), ev(-1), stream(s) {
    std::lock_guard<std::mutex> lk(g_mu);
    slot = slot_of(name);
    if (g_rec) {
        g_rec->items.push_back({slot, bytes});
        return;
    }
    Entry &e = g_entries[slot];
    e.launches++;
    e.bytes += bytes;
    if (g_timing) {
        cudaEvent_t a = get_event(), b = get_event();
        cudaEventRecord(a, s);
        e.pending.push_back({a, b});
        ev = (int)e.pending.size() - 1;
    }
}

ProfScope::~ProfScope() {
    if (ev < 0) return;
    std::lock_guard<std::mutex> lk(g_mu);
    cudaEventRecord(g_entries[slot].pending[ev].second, stream);
}

void prof_record_begin(ProfRecord *rec) { g_rec = rec; }
void prof_record_end() { g_rec = nullptr; }

void prof_replay(const ProfRecord &rec) {
    std::lock_guard<std::mutex> lk(g_mu);
    for (const auto &it : rec.items) {
        if (it.first < 0 || it.first >= (int)g_entries.size()) continue;
        g_entries[it.first].launches++;
        g_entries[it.first].bytes += it.second;
    }
}

bool prof_timing() {
    std::lock_guard<std::mutex> lk(g_mu);
    return g_timing;
}

void prof_enable(bool on) {
    std::lock_guard<std::mutex> lk(g_mu);
    g_timing = on;
    if (on && !g_dev) {
        if (cudaMalloc(&g_dev, MAX_DEV * sizeof(unsigned long long)) != cudaSuccess) {
            g_dev = nullptr;
            cudaGetLastError();
        } else {
            cudaMemset(g_dev, 0, MAX_DEV * sizeof(unsigned long long));
        }
    }
}

unsigned long long *prof_device_bytes(const char *name) {
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_timing || !g_dev || g_rec) return nullptr;
    const int sl = slot_of(name);
    return sl < MAX_DEV ? g_dev + sl : nullptr;
}

void prof_reset() {
    cudaDeviceSynchronize();
    if (g_dev) cudaMemset(g_dev, 0, MAX_DEV * sizeof(unsigned long long));
    std::lock_guard<std::mutex> lk(g_mu);
    for (auto &e : g_entries) {
        for (auto &pr : e.pending) {
            g_pool.push_back(pr.first);
            g_pool.push_back(pr.second);
        }
        e.pending.clear();
        e.launches = 0;
        e.ms = 0.0;
        e.bytes = 0.0;
    }
}

int prof_read(KernelStat *out, int max) {
    cudaDeviceSynchronize();
    unsigned long long dev[MAX_DEV] = {0};
    if (g_dev) {
        cudaMemcpy(dev, g_dev, sizeof(dev), cudaMemcpyDeviceToHost);
        cudaMemset(g_dev, 0, sizeof(dev));
    }
    std::lock_guard<std::mutex> lk(g_mu);
    int n = 0;
    for (size_t i = 0; i < g_entries.size(); i++) {
        auto &e = g_entries[i];
        if (i < (size_t)MAX_DEV) e.bytes += (double)dev[i];
        for (auto &pr : e.pending) {
            float ms = 0.f;
            if (cudaEventElapsedTime(&ms, pr.first, pr.second) == cudaSuccess) e.ms += ms;
            g_pool.push_back(pr.first);
            g_pool.push_back(pr.second);
        }
        cudaGetLastError();
        e.pending.clear();
        if (n < max && out) {
            memset(&out[n], 0, sizeof(KernelStat));
            strncpy(out[n].name, e.name.c_str(), sizeof(out[n].name) - 1);
            out[n].launches = e.launches;
            out[n].ms = e.ms;
            out[n].bytes = e.bytes;
        }
        n++;
    }
    return n;
}

// ------------------------------------------------------------------------------------
// Arithmetic roofs: FP64 and FP32 fused multiply-add throughput of this GPU, measured
// with independent FMA chains (8 per thread, FP32 as packed pairs) over a grid that
// fills every SM; the reference for kernels bound by arithmetic rather than HBM.
// ------------------------------------------------------------------------------------
namespace {
__global__ void k_fma64_probe(double *out, int iters, double a, double b) {
    double x[8];
#pragma unroll
    for (int j = 0; j < 8; j++) x[j] = threadIdx.x * 1e-3 + j;
    for (int i = 0; i < iters; i++)
#pragma unroll
        for (int j = 0; j < 8; j++) x[j] = fma(x[j], a, b);
    double sm = 0.0;
#pragma unroll
    for (int j = 0; j < 8; j++) sm += x[j];
    if (sm == 1234.5) out[0] = sm;  // never true: keeps the chains alive
}
__global__ void k_fma32_probe(float *out, int iters, float a, float b) {
    float2 x[8];
    const float2 a2 = make_float2(a, a), b2 = make_float2(b, b);
#pragma unroll
    for (int j = 0; j < 8; j++) x[j] = make_float2(threadIdx.x * 1e-3f + j, j * 0.5f);
    for (int i = 0; i < iters; i++)
#pragma unroll
        for (int j = 0; j < 8; j++) x[j] = __ffma2_rn(x[j], a2, b2);
    float sm = 0.f;
#pragma unroll
    for (int j = 0; j < 8; j++) sm += x[j].x + x[j].y;
    if (sm == 1234.5f) out[0] = sm;
}
}  // namespace

cudaError_t alu_peak(int prec, double *tflops, cudaStream_t s) {
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    const int threads = 256, blocks = sms * 8;
    const int iters = prec == 64 ? 512 : 16384;
    void *buf = nullptr;
    e = cudaMallocAsync(&buf, 16, s);
    if (e != cudaSuccess) return e;
    cudaEvent_t a = nullptr, b = nullptr;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    float best = 0.f;
    for (int rep = 0; rep < 3; rep++) {
        cudaEventRecord(a, s);
        if (prec == 64) k_fma64_probe<<<blocks, threads, 0, s>>>((double *)buf, iters, 0.999999, 1e-7);
        else k_fma32_probe<<<blocks, threads, 0, s>>>((float *)buf, iters, 0.999f, 1e-4f);
        cudaEventRecord(b, s);
        e = cudaEventSynchronize(b);
        if (e != cudaSuccess) break;
        float ms = 0.f;
        cudaEventElapsedTime(&ms, a, b);
        if (rep > 0 && (best == 0.f || ms < best)) best = ms;
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    cudaFreeAsync(buf, s);
    if (e != cudaSuccess) return e;
    // FMAs: threads * iters * 8 chains (x 2 lanes for the packed FP32 pairs); 2 flops each
    const double fmas = (double)blocks * threads * iters * 8.0 * (prec == 64 ? 1.0 : 2.0);
    *tflops = 2.0 * fmas / (best * 1e-3) / 1e12;
    return cudaGetLastError();
}

}  // namespace eig
