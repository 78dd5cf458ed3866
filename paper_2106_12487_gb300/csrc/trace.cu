// Phase tracer of the band solver: CUDA-event pairs on the plan's stream
// around the solver's phases (PCG, residual applies, orthogonalisation,
// projections), summed after the solve's final synchronisation.
#include <cuda_runtime.h>

#include "internal.h"

namespace bloch {

int trace_begin(bloch_plan* pl, int phase) {
    Tracer& t = pl->trace;
    if (!t.on) return -1;
    cudaEvent_t ev[2];
    for (int i = 0; i < 2; ++i) {
        if (!t.pool.empty()) {
            ev[i] = t.pool.back();
            t.pool.pop_back();
        } else if (cudaEventCreate(&ev[i]) != cudaSuccess) {
            cudaGetLastError();
            if (i == 1) t.pool.push_back(ev[0]);
            return -1;
        }
    }
    if (cudaEventRecord(ev[0], pl->stream) != cudaSuccess) {
        cudaGetLastError();
        t.pool.push_back(ev[0]);
        t.pool.push_back(ev[1]);
        return -1;
    }
    t.open.push_back({phase, ev[0], ev[1], false});
    return (int)t.open.size() - 1;
}

void trace_end(bloch_plan* pl, int idx) {
    Tracer& t = pl->trace;
    if (idx < 0 || idx >= (int)t.open.size()) return;
    if (cudaEventRecord(t.open[idx].b, pl->stream) != cudaSuccess) cudaGetLastError();
    else t.open[idx].ended = true;
}

void trace_add(bloch_plan* pl, int phase, double ms) {
    Tracer& t = pl->trace;
    if (!t.on) return;
    t.ms[phase] += ms;
    t.count[phase] += 1;
}

void trace_collect(bloch_plan* pl) {
    Tracer& t = pl->trace;
    for (auto& p : t.open) {
        float ms = 0.f;
        if (p.ended && cudaEventElapsedTime(&ms, p.a, p.b) == cudaSuccess) {
            t.ms[p.phase] += ms;
            t.count[p.phase] += 1;
        } else {
            cudaGetLastError();
        }
        t.pool.push_back(p.a);
        t.pool.push_back(p.b);
    }
    t.open.clear();
}

void trace_release(bloch_plan* pl) {
    Tracer& t = pl->trace;
    for (auto& p : t.open) {
        cudaEventDestroy(p.a);
        cudaEventDestroy(p.b);
    }
    for (auto e : t.pool) cudaEventDestroy(e);
    t.open.clear();
    t.pool.clear();
}

}  // namespace bloch

using namespace bloch;

extern "C" bloch_status bloch_plan_trace(bloch_plan* pl, int32_t enable, bloch_trace* out) {
    if (!pl) return set_error(BLOCH_EINVAL, "plan is NULL");
    if (enable != 0 && enable != 1) return set_error(BLOCH_EINVAL, "enable must be 0 or 1");
    Tracer& t = pl->trace;
    if (cudaStreamSynchronize(pl->stream) != cudaSuccess) return set_cuda_error(cudaGetLastError(), "trace sync");
    trace_collect(pl);
    if (out) {
        for (int i = 0; i < TR_NPHASE; ++i) {
            out->ms[i] = t.ms[i];
            out->count[i] = t.count[i];
        }
    }
    for (int i = 0; i < TR_NPHASE; ++i) {
        t.ms[i] = 0.0;
        t.count[i] = 0;
    }
    t.on = enable != 0;
    return BLOCH_OK;
}
