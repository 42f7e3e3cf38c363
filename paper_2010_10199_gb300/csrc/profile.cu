// Per-stage CUDA-event timing of the kernels a plan launches (measurement
// support for the benchmark; no counterpart in the paper).
#include <vector>

#include "internal.cuh"

namespace agft {

static const char *kStageNames[N_STAGES] = {"trafo_pre", "gather", "spread", "reduce_partials",
                                            "adjoint_post", "empty_sum", "solver_vec"};

struct Profiler {
    bool on = false;
    std::vector<cudaEvent_t> pool;
    struct Pending {
        int stage;
        cudaEvent_t a, b;
    };
    std::vector<Pending> pending;
    cudaEvent_t open[N_STAGES] = {};
    double ms[N_STAGES] = {};
    long long count[N_STAGES] = {};

    cudaEvent_t get() {
        if (!pool.empty()) {
            cudaEvent_t e = pool.back();
            pool.pop_back();
            return e;
        }
        cudaEvent_t e = nullptr;
        cudaEventCreate(&e);
        return e;
    }
    void resolve() {
        for (auto &q : pending) {
            float t = 0.f;
            if (cudaEventElapsedTime(&t, q.a, q.b) == cudaSuccess) {
                ms[q.stage] += t;
                count[q.stage] += 1;
            }
            pool.push_back(q.a);
            pool.push_back(q.b);
        }
        pending.clear();
    }
    ~Profiler() {
        for (auto &q : pending) {
            cudaEventDestroy(q.a);
            cudaEventDestroy(q.b);
        }
        for (auto e : pool) cudaEventDestroy(e);
    }
};

static bool capturing(cudaStream_t s) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    cudaStreamIsCapturing(s, &cs);
    return cs != cudaStreamCaptureStatusNone;
}

void stage_begin(Plan &p, int stage) {
    if (!p.prof || !p.prof->on || capturing(p.stream)) return;
    cudaEvent_t e = p.prof->get();
    cudaEventRecord(e, p.stream);
    p.prof->open[stage] = e;
}

void stage_end(Plan &p, int stage) {
    if (!p.prof || !p.prof->on || !p.prof->open[stage]) return;
    cudaEvent_t e = p.prof->get();
    cudaEventRecord(e, p.stream);
    p.prof->pending.push_back({stage, p.prof->open[stage], e});
    p.prof->open[stage] = nullptr;
    if (p.prof->pending.size() > 4096) {
        cudaEventSynchronize(e);
        p.prof->resolve();
    }
}

void profiler_free(Plan &p) {
    delete p.prof;
    p.prof = nullptr;
}

}  // namespace agft

using namespace agft;

extern "C" {

int anova_profile_enable(anova_plan_t plan, int on) {
    if (!plan) return ANOVA_ERR_INVALID;
    Plan &p = plan->p;
    if (!p.prof) p.prof = new Profiler();
    p.prof->on = on != 0;
    return ANOVA_OK;
}

int anova_profile_read(anova_plan_t plan, double *ms, int64_t *launches, const char **names, int max_stages,
                       int *n_stages, int reset) {
    if (!plan) return ANOVA_ERR_INVALID;
    Plan &p = plan->p;
    if (n_stages) *n_stages = N_STAGES;
    cudaError_t e = cudaStreamSynchronize(p.stream);
    if (e != cudaSuccess) return cuda_status(e);
    if (p.prof) p.prof->resolve();
    for (int s = 0; s < N_STAGES && s < max_stages; ++s) {
        if (ms) ms[s] = p.prof ? p.prof->ms[s] : 0.0;
        if (launches) launches[s] = p.prof ? p.prof->count[s] : 0;
        if (names) names[s] = kStageNames[s];
    }
    if (reset && p.prof) {
        for (int s = 0; s < N_STAGES; ++s) {
            p.prof->ms[s] = 0;
            p.prof->count[s] = 0;
        }
    }
    return ANOVA_OK;
}

}  // extern "C"
