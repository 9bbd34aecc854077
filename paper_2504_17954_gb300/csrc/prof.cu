// Opt-in per-kernel timing: when enabled, every kernel launch of the library is bracketed by
// two CUDA events recorded on the launching stream; ivrgs_prof_report() sums them per kernel.
// Off by default (and it must stay off during CUDA-graph capture).
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "prof.cuh"

namespace ivrgs {

namespace {
struct Rec {
    const char* name;
    cudaEvent_t a, b;
};
std::mutex g_mu;
bool g_on = false;
std::vector<Rec> g_recs;
std::vector<cudaEvent_t> g_pool;
struct Acc {
    std::string name;
    long long count;
    double ms;
};
std::vector<Acc> g_acc;

cudaEvent_t take_event() {
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

ProfScope::ProfScope(const char* name, cudaStream_t s) : name_(name), s_(s), a_(nullptr) {
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_on) return;
    a_ = take_event();
    cudaEventRecord(a_, s_);
}

ProfScope::~ProfScope() {
    if (!a_) return;
    std::lock_guard<std::mutex> lk(g_mu);
    cudaEvent_t b = take_event();
    cudaEventRecord(b, s_);
    g_recs.push_back({name_, a_, b});
}

}  // namespace ivrgs

using namespace ivrgs;

extern "C" {

void ivrgs_prof_enable(int32_t on) {
    std::lock_guard<std::mutex> lk(g_mu);
    g_on = on != 0;
}

int64_t ivrgs_prof_report(char* buf, int64_t len) {
    std::lock_guard<std::mutex> lk(g_mu);
    // drain finished records into the per-kernel totals
    for (const Rec& r : g_recs) {
        cudaEventSynchronize(r.b);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, r.a, r.b);
        bool found = false;
        for (auto& x : g_acc)
            if (x.name == r.name) {
                x.count += 1;
                x.ms += ms;
                found = true;
                break;
            }
        if (!found) g_acc.push_back({r.name, 1, (double)ms});
        g_pool.push_back(r.a);
        g_pool.push_back(r.b);
    }
    g_recs.clear();
    std::string out;
    for (auto& x : g_acc) {
        char line[256];
        snprintf(line, sizeof line, "%s %lld %.6f\n", x.name.c_str(), x.count, x.ms);
        out += line;
    }
    // the totals are handed out (and reset) only to a caller whose buffer holds them
    if (buf && len > (int64_t)out.size()) {
        memcpy(buf, out.data(), out.size());
        buf[out.size()] = 0;
        g_acc.clear();
    }
    return (int64_t)out.size();
}

}  // extern "C"
