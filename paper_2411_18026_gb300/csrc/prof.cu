// Timing registry behind fds_timing_enable / fds_timing_report.
#include <atomic>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <vector>
#include <cstdio>
#include <cstring>

#include "common.cuh"
#include "prof.cuh"

namespace {
struct Rec {
    std::string name;
    std::thread::id tid;     // scopes nest per thread (concurrent batched builds)
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    double flops = 0, bytes = 0, units = 0;
};
struct Acc {
    long launches = 0;
    double ms = 0, flops = 0, bytes = 0, units = 0;
};
std::mutex g_mu;
bool g_on = false;
std::vector<Rec> g_open;     // recorded, not yet resolved
std::map<std::string, Acc> g_acc;

void resolve_locked() {
    for (auto &r : g_open) {
        if (r.e1) {
            cudaEventSynchronize(r.e1);
            float ms = 0;
            if (cudaEventElapsedTime(&ms, r.e0, r.e1) == cudaSuccess) {
                Acc &a = g_acc[r.name];
                a.launches += 1;
                a.ms += ms;
                a.flops += r.flops;
                a.bytes += r.bytes;
                a.units += r.units;
            }
            cudaEventDestroy(r.e1);
        }
        if (r.e0) cudaEventDestroy(r.e0);
    }
    g_open.clear();
}
}  // namespace

thread_local bool g_capturing = false;
void prof_set_capturing(bool on) { g_capturing = on; }
bool prof_enabled() { return g_on && !g_capturing; }

static std::atomic<long long> g_launches{0};
void fds_count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
extern "C" int64_t fds_launch_count(void) { return (int64_t)g_launches.load(); }

void prof_begin(const char *name, cudaStream_t s) {
    std::lock_guard<std::mutex> lk(g_mu);
    Rec r;
    r.name = name;
    r.tid = std::this_thread::get_id();
    cudaEventCreate(&r.e0);
    cudaEventRecord(r.e0, s);
    g_open.push_back(r);
}

void prof_end(cudaStream_t s, double flops, double bytes, double units) {
    std::lock_guard<std::mutex> lk(g_mu);
    const std::thread::id me = std::this_thread::get_id();
    for (auto it = g_open.rbegin(); it != g_open.rend(); ++it)
        if (!it->e1 && it->tid == me) {
            cudaEventCreate(&it->e1);
            cudaEventRecord(it->e1, s);
            it->flops = flops;
            it->bytes = bytes;
            it->units = units;
            break;
        }
    if (g_open.size() > 4096) resolve_locked();
}

void prof_add_work(const char *name, double flops, double bytes, double units) {
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_on) return;
    Acc &a = g_acc[name];
    a.flops += flops;
    a.bytes += bytes;
    a.units += units;
}

extern "C" void fds_timing_enable(int32_t on) {
    std::lock_guard<std::mutex> lk(g_mu);
    g_on = on != 0;
}

extern "C" void fds_timing_reset(void) {
    std::lock_guard<std::mutex> lk(g_mu);
    resolve_locked();
    g_acc.clear();
}

extern "C" int fds_timing_report(char *buf, int32_t cap) {
    std::lock_guard<std::mutex> lk(g_mu);
    resolve_locked();
    std::string out;
    char line[256];
    for (auto &kv : g_acc) {
        snprintf(line, sizeof(line), "%s %ld %.6f %.6e %.6e %.6e\n", kv.first.c_str(), kv.second.launches,
                 kv.second.ms, kv.second.flops, kv.second.bytes, kv.second.units);
        out += line;
    }
    if (buf && cap > 0) {
        size_t n = out.size() < (size_t)(cap - 1) ? out.size() : (size_t)(cap - 1);
        memcpy(buf, out.data(), n);
        buf[n] = 0;
    }
    return (int)out.size() + 1;
}

namespace {
thread_local char g_err[256] = "";
}

void fds_note_cuda_error(cudaError_t e, const char *file, int line) {
    const char *f = strrchr(file, '/');
    snprintf(g_err, sizeof(g_err), "%s (%s) at %s:%d", cudaGetErrorName(e), cudaGetErrorString(e), f ? f + 1 : file,
             line);
}

extern "C" const char *fds_last_error_detail(void) { return g_err; }

void fds_set_error_detail(const char *msg) { snprintf(g_err, sizeof(g_err), "%s", msg ? msg : ""); }

std::mutex &dyn_smem_mutex() {
    static std::mutex m;
    return m;
}

size_t &dyn_smem_slot(const void *kernel) {
    static std::map<const void *, size_t> cur;   // default limit 48 KB until raised
    auto it = cur.find(kernel);
    if (it == cur.end()) it = cur.emplace(kernel, (size_t)48 * 1024).first;
    return it->second;
}
