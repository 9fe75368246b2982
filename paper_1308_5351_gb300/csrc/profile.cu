// Optional per-launch device timing (CUDA events on the launching stream).
// Off by default; while on, every instrumented launch records an event pair
// and the amount of algorithmic work it was asked to do, so that a caller
// can form achieved rates for each kernel over exactly the region it timed.
#include <mutex>
#include <vector>

#include "gnk_internal.h"

namespace gnk {
namespace {

struct Rec {
    cudaEvent_t a, b;
    int kind;
    double work;
    double instr;
    double bytes;
    bool skipped;
};

std::mutex g_mu;
bool g_on = false;
unsigned g_mask = ~0u;
thread_local bool t_collect = false;
thread_local std::vector<long> t_ids;
std::vector<Rec> g_recs;
std::vector<cudaEvent_t> g_pool;

cudaEvent_t take_event() {
    if (!g_pool.empty()) {
        cudaEvent_t e = g_pool.back();
        g_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return e;
}

void recycle_all() {
    for (Rec& r : g_recs) {
        if (r.a) g_pool.push_back(r.a);
        if (r.b) g_pool.push_back(r.b);
    }
    g_recs.clear();
}

}  // namespace

ProfToken prof_begin(cudaStream_t st, int kind) {
    ProfToken t;
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_on) return t;
    if (kind >= 0 && kind < 32 && !((g_mask >> kind) & 1u)) return t;
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &cap) != cudaSuccess) {
        cudaGetLastError();
        return t;
    }
    if (cap != cudaStreamCaptureStatusNone) return t;  // no event timing inside captured graphs
    t.ev = take_event();
    if (t.ev) cudaEventRecord(static_cast<cudaEvent_t>(t.ev), st);
    return t;
}

long prof_end(const ProfToken& t, int kind, double work, cudaStream_t st, double instr, double bytes) {
    if (!t.ev) return -1;
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_on) {
        g_pool.push_back(static_cast<cudaEvent_t>(t.ev));
        return -1;
    }
    cudaEvent_t b = take_event();
    if (!b) return -1;
    cudaEventRecord(b, st);
    g_recs.push_back(Rec{static_cast<cudaEvent_t>(t.ev), b, kind, work, instr, bytes, false});
    const long id = (long)g_recs.size() - 1;
    if (t_collect) t_ids.push_back(id);
    return id;
}

void prof_collect_begin() {
    t_collect = true;
    t_ids.clear();
}

void prof_collect_end(std::vector<long>* out) {
    t_collect = false;
    out->swap(t_ids);
    t_ids.clear();
}

void prof_skip(long idx) {
    if (idx < 0) return;
    std::lock_guard<std::mutex> lk(g_mu);
    if (idx < (long)g_recs.size()) g_recs[idx].skipped = true;
}

}  // namespace gnk

using namespace gnk;

extern "C" {

int gnk_profile_enable(int on) {
    std::lock_guard<std::mutex> lk(g_mu);
    for (Rec& r : g_recs) cudaEventSynchronize(r.b);
    recycle_all();
    g_on = on != 0;
    return GNK_OK;
}

int gnk_profile_mask(unsigned mask) {
    std::lock_guard<std::mutex> lk(g_mu);
    g_mask = mask;
    return GNK_OK;
}

int gnk_profile_query(int kind, long long* launches, double* total_ms, double* work) {
    return gnk_profile_query_ex(kind, launches, total_ms, work, nullptr);
}

int gnk_profile_query_ex(int kind, long long* launches, double* total_ms, double* work, double* instr) {
    return gnk_profile_query_bytes(kind, launches, total_ms, work, instr, nullptr);
}

int gnk_profile_query_bytes(int kind, long long* launches, double* total_ms, double* work, double* instr,
                            double* bytes) {
    std::lock_guard<std::mutex> lk(g_mu);
    long long n = 0;
    double ms = 0.0, wk = 0.0, ins = 0.0, by = 0.0;
    for (const Rec& r : g_recs) {
        if (r.kind != kind || r.skipped) continue;
        if (cudaEventSynchronize(r.b) != cudaSuccess) {
            set_error("event synchronisation failed");
            cudaGetLastError();
            return GNK_ECUDA;
        }
        float t = 0.f;
        if (cudaEventElapsedTime(&t, r.a, r.b) != cudaSuccess) {
            cudaGetLastError();
            continue;
        }
        ++n;
        ms += t;
        wk += r.work;
        ins += r.instr;
        by += r.bytes;
    }
    if (launches) *launches = n;
    if (total_ms) *total_ms = ms;
    if (work) *work = wk;
    if (instr) *instr = ins;
    if (bytes) *bytes = by;
    return GNK_OK;
}

}  // extern "C"
