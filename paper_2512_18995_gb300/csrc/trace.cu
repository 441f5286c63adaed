// Launch accounting and opt-in CUDA-event tracing of every library kernel.
#include <cstring>

#include "dq_plan.h"

namespace dq {

thread_local Tracer *g_tracer = nullptr;

cudaEvent_t Tracer::get_event() {
    if (!pool.empty()) {
        cudaEvent_t e = pool.back();
        pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

int Tracer::name_id(const char *n) {
    for (size_t i = 0; i < names.size(); ++i)
        if (names[i] == n) return (int)i;
    names.emplace_back(n);
    acc.emplace_back(0, 0.0);
    return (int)names.size() - 1;
}

void Tracer::release() {
    for (auto &r : recs) {
        cudaEventDestroy(r.a);
        cudaEventDestroy(r.b);
    }
    for (auto e : pool) cudaEventDestroy(e);
    recs.clear();
    pool.clear();
    names.clear();
    acc.clear();
}

// Inside a stream capture the event records become nodes of the graph
// (recorded at every replay); outside they are ordinary stream records.
static void record(cudaEvent_t e, cudaStream_t s) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cs) == cudaSuccess && cs == cudaStreamCaptureStatusActive)
        cudaEventRecordWithFlags(e, s, cudaEventRecordExternal);
    else
        cudaEventRecord(e, s);
}

LaunchScope::LaunchScope(cudaStream_t st, const char *name, int64_t *c) : s(st), counter(c) {
    Tracer *t = g_tracer;
    if (t && t->on) {
        Tracer::Rec r;
        r.name = t->name_id(name);
        r.a = t->get_event();
        r.b = t->get_event();
        record(r.a, s);
        t->recs.push_back(r);
        rec = (int)t->recs.size() - 1;
    }
}

LaunchScope::~LaunchScope() {
    if (counter) ++*counter;
    Tracer *t = g_tracer;
    if (rec >= 0 && t) record(t->recs[rec].b, s);
}

}  // namespace dq
