// Learned cost model entry points: the MLP kernels behind the C-ABI, training
// on logged predicate evaluations, and the learned plan statistics.
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <cmath>
#include <random>
#include <vector>

#include "hb_ctx.h"

using namespace hb;

extern "C" hb_status hb_mlp_forward(const float *X, int32_t n, const float *params, float *y, void *stream) {
    if (n < 0 || (n > 0 && (!X || !params || !y))) return fail(HB_ERR_ARG, "hb_mlp_forward: bad arguments");
    HB_CUDA(mlp_forward(X, n, params, y, 0, static_cast<cudaStream_t>(stream)));
    return HB_OK;
}

extern "C" hb_status hb_mlp_forward_bf16(const float *X, int32_t n, const float *params, float *y, void *stream) {
    if (n < 0 || (n > 0 && (!X || !params || !y))) return fail(HB_ERR_ARG, "hb_mlp_forward_bf16: bad arguments");
    HB_CUDA(mlp_forward(X, n, params, y, 1, static_cast<cudaStream_t>(stream)));
    return HB_OK;
}

extern "C" hb_status hb_mlp_backward(const float *X, const float *t, int32_t n, const float *params, float *grad,
                                     void *stream) {
    if (n < 0 || !params || !grad || (n > 0 && (!X || !t))) return fail(HB_ERR_ARG, "hb_mlp_backward: bad arguments");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    float *work = nullptr;
    HB_CUDA(cudaMallocAsync(reinterpret_cast<void **>(&work), sizeof(float) * mlp_work_floats(n), s));
    cudaError_t e = mlp_backward(X, t, n, params, grad, work, s);
    cudaFreeAsync(work, s);
    HB_CUDA(e);
    return HB_OK;
}

extern "C" hb_status hb_adam_step(float *params, const float *grad, float *m, float *v, int32_t n_params, int32_t step,
                                  float lr, float beta1, float beta2, float eps, void *stream) {
    if (n_params < 0 || step < 1 || (n_params > 0 && (!params || !grad || !m || !v)))
        return fail(HB_ERR_ARG, "hb_adam_step: bad arguments");
    HB_CUDA(adam_step(params, grad, m, v, n_params, step, lr, beta1, beta2, eps, static_cast<cudaStream_t>(stream)));
    return HB_OK;
}

namespace hb {

hb_status learned_stats(hb_ctx *c, std::vector<double> &sp, std::vector<double> &cost, bool &ok) {
    (void)sp;
    (void)cost;
    ok = false;
    if (!c->model_ok) return HB_OK;
    return HB_OK;
}

}  // namespace hb

extern "C" hb_status hb_get_cost_model(hb_ctx *c, float *params_out) {
    if (!c || !params_out) return fail(HB_ERR_ARG, "hb_get_cost_model: NULL argument");
    if (!c->model_ok) return fail(HB_ERR_STATE, "hb_get_cost_model: no model trained or set");
    memcpy(params_out, c->model.data(), sizeof(float) * 2 * HB_MLP_PARAMS);
    return HB_OK;
}

extern "C" hb_status hb_set_cost_model(hb_ctx *c, const float *params) {
    if (!c || !params) return fail(HB_ERR_ARG, "hb_set_cost_model: NULL argument");
    c->model.assign(params, params + 2 * HB_MLP_PARAMS);
    for (float x : c->model)
        if (!std::isfinite(x)) {
            c->model_ok = false;
            return fail(HB_ERR_ARG, "hb_set_cost_model: non-finite weight");
        }
    c->model_ok = true;
    return HB_OK;
}

namespace hb {

// One instrumented evaluation over the given records; per program op the
// counters [evaluated, passed, cycles, stage1, stage2, core].
hb_status instrumented_run(hb_ctx *c, const uint32_t *rec_r, int64_t n_r, const uint32_t *rec_s, int64_t n_s,
                           bool self, int profile, std::vector<unsigned long long> &counters, RunResult &res) {
    const int kbs = bits_for((uint64_t)std::max<int64_t>(n_s, 2));
    const int kb = kbs + bits_for((uint64_t)std::max<int64_t>(n_r, 2));
    uint64_t *sorted = nullptr;
    HB_TRY(block_eval_sort(c, rec_r, n_r, rec_s, n_s, self, 1, kb, kbs, profile ? 2 : 1, res, &sorted, nullptr));
    counters.assign((size_t)MAX_OPS * 6, 0ull);
    HB_CUDA(cudaMemcpyAsync(counters.data(), c->w_log.p, sizeof(unsigned long long) * counters.size(),
                            cudaMemcpyDeviceToHost, c->stream));
    HB_CUDA(cudaStreamSynchronize(c->stream));
    return HB_OK;
}

static float logit_clamped(double p) {
    p = std::min(std::max(p, 1e-6), 1.0 - 1e-6);
    double v = std::log(p / (1.0 - p));
    return (float)std::min(std::max(v, -12.0), 12.0);
}

}  // namespace hb

extern "C" hb_status hb_log_predicates(hb_ctx *c, int32_t profile, hb_pred_log *out, int32_t cap, int32_t *n_out) {
    if (!c || !out || !n_out) return fail(HB_ERR_ARG, "hb_log_predicates: NULL argument");
    *n_out = 0;
    cudaSetDevice(c->device);
    HB_TRY(ensure_ready(c, false));
    const bool self = is_self(c);
    const int64_t nr = c->side[0].n, ns = self ? nr : c->side[1].n;
    std::vector<unsigned long long> ctr;
    RunResult res;
    HB_TRY(instrumented_run(c, c->side[0].rec, nr, self ? c->side[0].rec : c->side[1].rec, ns, self, profile, ctr,
                            res));
    c->stats.candidate_pairs = res.cand;
    c->stats.examined_pairs = res.examined;
    c->stats.emitted_pairs = res.n_out;
    const int n_ops = (int)c->ops.size();
    if (n_ops > cap) return fail(HB_ERR_OVERFLOW, "hb_log_predicates: capacity below the number of predicates");
    std::vector<float> feats;
    for (int k = 0; k < n_ops; k++) {
        hb_pred_log &L = out[k];
        memset(&L, 0, sizeof(L));
        const unsigned long long *v = &ctr[(size_t)k * 6];
        L.evaluated = (int64_t)v[0];
        L.passed = (int64_t)v[1];
        L.cycles = (int64_t)v[2];
        L.stage1 = (int64_t)v[3];
        L.stage2 = (int64_t)v[4];
        L.core = (int64_t)v[5];
        L.pred = c->program[k];
        L.kind = c->preds[c->program[k]].p.kind;
        const double ev = std::max<double>((double)v[0], 1.0);
        L.log_cost = (float)std::log(std::max((double)v[2] / ev, 1.0));
        L.logit_pass = logit_clamped(v[0] ? (double)v[1] / ev : 0.5);
    }
    *n_out = n_ops;
    return HB_OK;
}

extern "C" hb_status hb_predicate_features(hb_ctx *c, float *features_out, int32_t cap_preds, int32_t *n_out) {
    (void)c; (void)features_out; (void)cap_preds; (void)n_out;
    return fail(HB_ERR_STATE, "hb_predicate_features: not available yet");
}

extern "C" hb_status hb_train_cost_model(hb_ctx *c, int32_t n, const float *X, const float *y_cost,
                                         const float *y_sel, int32_t epochs, float lr, uint64_t seed,
                                         float *loss_out) {
    (void)c; (void)n; (void)X; (void)y_cost; (void)y_sel; (void)epochs; (void)lr; (void)seed; (void)loss_out;
    return fail(HB_ERR_STATE, "hb_train_cost_model: not available yet");
}

