// Call tracing: while enabled, each traced C-ABI call records one CUDA event
// on its stream before it enqueues anything and one when it returns, so the
// device time of the work that call enqueued can be read back later.  Off by
// default; when off a traced call pays one relaxed atomic load.  Calls made
// on a stream that is being captured into a CUDA graph are not traced (an
// event recorded during capture has no time to read).
#include <atomic>
#include <deque>
#include <mutex>

#include "airga_internal.cuh"

namespace airga {
namespace {

struct TraceRec {
    const char *name;
    cudaStream_t stream;
    cudaEvent_t e0, e1;
};

std::mutex g_mu;
std::atomic<int> g_on{0};
std::deque<TraceRec> g_recs;     // finished calls, oldest first
size_t g_cap = 0;
int64_t g_dropped = 0;

void destroy(cudaEvent_t e) {
    if (e) cudaEventDestroy(e);
}

}  // namespace

TraceScope::TraceScope(const char *name, void *stream)
    : name_(name), stream_(stream), e0_(nullptr) {
    if (!g_on.load(std::memory_order_relaxed)) return;
    cudaStream_t s = (cudaStream_t)stream;
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cap) != cudaSuccess || cap != cudaStreamCaptureStatusNone) return;
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) return;
    if (cudaEventRecord(e, s) != cudaSuccess) {
        destroy(e);
        return;
    }
    e0_ = e;
}

TraceScope::~TraceScope() {
    if (!e0_) return;
    cudaStream_t s = (cudaStream_t)stream_;
    cudaEvent_t e1 = nullptr;
    if (cudaEventCreate(&e1) != cudaSuccess || cudaEventRecord(e1, s) != cudaSuccess) {
        destroy(e1);
        destroy((cudaEvent_t)e0_);
        return;
    }
    std::lock_guard<std::mutex> lock(g_mu);
    if (g_on.load() && g_recs.size() < g_cap) {
        g_recs.push_back(TraceRec{name_, s, (cudaEvent_t)e0_, e1});
    } else {
        ++g_dropped;
        destroy((cudaEvent_t)e0_);
        destroy(e1);
    }
}

}  // namespace airga

using namespace airga;

extern "C" int airga_trace_enable(int32_t capacity) {
    if (capacity < 0 || capacity > (1 << 24))
        return fail(AIRGA_E_INVALID_ARG, "capacity must be in [0, 2^24]");
    std::lock_guard<std::mutex> lock(g_mu);
    if (capacity == 0) {
        g_on.store(0);
        for (auto &r : g_recs) {
            destroy(r.e0);
            destroy(r.e1);
        }
        g_recs.clear();
        g_cap = 0;
        g_dropped = 0;
        return AIRGA_OK;
    }
    g_cap = (size_t)capacity;
    g_on.store(1);
    return AIRGA_OK;
}

extern "C" int airga_trace_read(airga_trace_record *out, int32_t max_records, int32_t *count,
                                int64_t *dropped) {
    if (!count || max_records < 0 || (max_records > 0 && !out))
        return fail(AIRGA_E_INVALID_ARG, "trace_read needs count and room for max_records records");
    std::lock_guard<std::mutex> lock(g_mu);
    int32_t k = 0;
    while (k < max_records && !g_recs.empty()) {
        TraceRec r = g_recs.front();
        cudaError_t e = cudaEventSynchronize(r.e1);
        float ms = 0.0f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, r.e0, r.e1);
        if (e != cudaSuccess) {
            *count = k;
            return cuda_fail(e, "trace event");
        }
        out[k].name = r.name;
        out[k].ms = (double)ms;
        out[k].stream = (void *)r.stream;
        destroy(r.e0);
        destroy(r.e1);
        g_recs.pop_front();
        ++k;
    }
    *count = k;
    if (dropped) {
        *dropped = g_dropped;
        g_dropped = 0;
    }
    return AIRGA_OK;
}
