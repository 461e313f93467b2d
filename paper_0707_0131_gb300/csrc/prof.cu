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
}

void prof_reset() {
    cudaDeviceSynchronize();
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
    std::lock_guard<std::mutex> lk(g_mu);
    int n = 0;
    for (auto &e : g_entries) {
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

}  // namespace eig
