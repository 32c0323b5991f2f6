// Kernel tracing: launch counts (always on) and, when enabled, per-launch
// device durations from CUDA events recorded on the launching stream, with
// the algorithmic bytes each launch must move (the byte model of each kernel
// family is computed by its launcher from the problem sizes).
#include <cstring>
#include <map>
#include <mutex>

#include "ms_internal.h"

namespace msgb {

namespace {

struct Pending {
    const char *name;
    cudaEvent_t a, b;
    double bytes;
};

struct Stat {
    int64_t launches = 0;
    int64_t timed = 0;
    double ms = 0.0;
    double bytes = 0.0;
};

struct Profiler {
    std::mutex mu;
    bool enabled = false;
    std::map<std::string, Stat> stats;
    std::vector<Pending> pending;
    std::vector<cudaEvent_t> pool;
    int64_t total_launches = 0;

    cudaEvent_t get_event() {
        if (!pool.empty()) {
            cudaEvent_t e = pool.back();
            pool.pop_back();
            return e;
        }
        cudaEvent_t e = nullptr;
        if (cudaEventCreate(&e) != cudaSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        return e;
    }

    void resolve() {
        for (Pending &p : pending) {
            float t = 0.f;
            if (p.a && p.b && cudaEventSynchronize(p.b) == cudaSuccess && cudaEventElapsedTime(&t, p.a, p.b) == cudaSuccess) {
                Stat &s = stats[p.name];
                s.timed++;
                s.ms += t;
                s.bytes += p.bytes;
            } else {
                cudaGetLastError();
            }
            if (p.a) pool.push_back(p.a);
            if (p.b) pool.push_back(p.b);
        }
        pending.clear();
    }
};

// launches captured into a graph on this thread are listed, not timed
thread_local bool t_recording = false;
thread_local std::vector<std::string> t_recorded;

Profiler &prof() {
    static Profiler *p = new Profiler();   // never destroyed: events may outlive the CUDA context at exit
    return *p;
}

}  // namespace

KernelScope::KernelScope(cudaStream_t st, const char *name, double bytes) : st_(st), name_(name), bytes_(bytes) {
    Profiler &p = prof();
    std::lock_guard<std::mutex> g(p.mu);
    p.total_launches++;
    p.stats[name].launches++;
    if (t_recording) {   // captured into a graph: counted per replay, never timed with events
        t_recorded.emplace_back(name);
        return;
    }
    if (p.enabled) {
        a_ = p.get_event();
        if (a_) cudaEventRecord(a_, st_);
    }
}

KernelScope::~KernelScope() {
    if (!a_) return;
    Profiler &p = prof();
    std::lock_guard<std::mutex> g(p.mu);
    cudaEvent_t b = p.get_event();
    if (b) cudaEventRecord(b, st_);
    p.pending.push_back({name_, a_, b, bytes_});
}

void profile_add_bytes(const char *name, double bytes) {
    Profiler &p = prof();
    std::lock_guard<std::mutex> g(p.mu);
    for (auto it = p.pending.rbegin(); it != p.pending.rend(); ++it)
        if (std::strcmp(it->name, name) == 0) {
            it->bytes += bytes;
            return;
        }
}

std::mutex &attr_mutex() {
    static std::mutex m;
    return m;
}

bool profile_enabled() {
    Profiler &p = prof();
    std::lock_guard<std::mutex> g(p.mu);
    return p.enabled;
}

void profile_record_begin() {
    t_recording = true;
    t_recorded.clear();
}

std::vector<std::string> profile_record_end() {
    t_recording = false;
    return std::move(t_recorded);
}

void profile_add_launches(const std::vector<std::string> &names, int64_t times) {
    Profiler &p = prof();
    std::lock_guard<std::mutex> g(p.mu);
    for (const std::string &n : names) {
        p.stats[n].launches += times;
        p.total_launches += times;
    }
}

void profile_enable(bool on) {
    Profiler &p = prof();
    std::lock_guard<std::mutex> g(p.mu);
    p.enabled = on;
}

void profile_reset() {
    Profiler &p = prof();
    std::lock_guard<std::mutex> g(p.mu);
    p.resolve();
    p.stats.clear();
    p.total_launches = 0;
}

int profile_read(ms_kernel_stat *out, int cap, int64_t *total) {
    Profiler &p = prof();
    std::lock_guard<std::mutex> g(p.mu);
    p.resolve();
    int k = 0;
    for (auto &kv : p.stats) {
        if (out && k < cap) {
            ms_kernel_stat &o = out[k];
            std::memset(&o, 0, sizeof(o));
            std::strncpy(o.name, kv.first.c_str(), sizeof(o.name) - 1);
            o.launches = kv.second.launches;
            o.timed_launches = kv.second.timed;
            o.total_ms = kv.second.ms;
            o.bytes = kv.second.bytes;
        }
        ++k;
    }
    if (total) *total = p.total_launches;
    return k;
}

}  // namespace msgb
