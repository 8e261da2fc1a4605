// Learned cost model entry points: the MLP kernels behind the C-ABI, training
// on logged predicate evaluations, and the learned plan statistics.
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
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

constexpr double FILTER_CYCLES = 16.0;   // cheap filter of one pair on shared-memory operands

static float logit_clamped(double p) {
    p = std::min(std::max(p, 1e-6), 1.0 - 1e-6);
    double v = std::log(p / (1.0 - p));
    return (float)std::min(std::max(v, -12.0), 12.0);
}

__global__ void k_gather_rows(const uint32_t *src, int W, int64_t stride, int64_t n_out, uint32_t *dst) {
    const int64_t total = n_out * W;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t row = i / W, w = i % W;
        dst[i] = src[(row * stride) * W + w];
    }
}

// Features of every distinct predicate (HB_FEATURES each): the predicate's
// kind and threshold, the sampled column statistics of the planner, and the
// pass rate / cost / filter rates measured by one instrumented evaluation of
// a row sample (every predicate evaluated on every candidate pair of the
// sample, no early exit).  Requires the current layout to be encoded.
hb_status predicate_features(hb_ctx *c, std::vector<float> &F) {
    const int P = (int)c->preds.size();
    F.assign((size_t)P * HB_FEATURES, 0.f);
    const bool self = is_self(c);
    const int64_t target = 200000;
    SideData &R = c->side[0];
    SideData &S = c->side[1];
    const int64_t sR = std::max<int64_t>(1, R.n / target), mR = R.n / sR;
    const int64_t nS = self ? 0 : S.n;
    const int64_t sS = std::max<int64_t>(1, nS / target), mS = self ? 0 : nS / sS;
    Buf rr, rh, sr, sh;
    auto gather = [&](const uint32_t *src, int W, int64_t stride, int64_t m, Buf &dst) -> hb_status {
        HB_TRY(grow(c, dst, sizeof(uint32_t) * (size_t)W * (size_t)std::max<int64_t>(m, 1) + 64));
        if (m > 0) {
            HB_LAUNCHED(1);
            k_gather_rows<<<(unsigned)(4 * c->n_sm), 256, 0, c->stream>>>(src, W, stride, m, as<uint32_t>(dst));
        }
        return HB_OK;
    };
    HB_TRY(gather(R.rec, c->W, sR, mR, rr));
    HB_TRY(gather(R.hot, c->HW, sR, mR, rh));
    if (!self) {
        HB_TRY(gather(S.rec, c->W, sS, mS, sr));
        HB_TRY(gather(S.hot, c->HW, sS, mS, sh));
    }
    uint32_t *save[4] = {R.rec, R.hot, S.rec, S.hot};
    R.rec = as<uint32_t>(rr);
    R.hot = as<uint32_t>(rh);
    if (!self) {
        S.rec = as<uint32_t>(sr);
        S.hot = as<uint32_t>(sh);
    }
    std::vector<unsigned long long> ctr;
    RunResult res;
    hb_status st = instrumented_run(c, R.rec, mR, self ? R.rec : S.rec, self ? mR : mS, self, 1, ctr, res);
    R.rec = save[0];
    R.hot = save[1];
    S.rec = save[2];
    S.hot = save[3];
    Buf *tmp[] = {&rr, &rh, &sr, &sh};
    for (Buf *b : tmp) free_buf(c, *b);
    HB_TRY(st);
    std::vector<int> op_of(P, -1);
    for (size_t k = 0; k < c->program.size(); k++) op_of[c->program[k]] = (int)k;
    ensure_pred_stats(c);
    for (int p = 0; p < P; p++) {
        float *f = &F[(size_t)p * HB_FEATURES];
        const hb_predicate &q = c->preds[p].p;
        // kind one-hot over the five basic kinds: a constant reads like an equality, containment and
        // word-token Jaccard like q-gram Jaccard
        const int kslot = q.kind == HB_P_CONST_EQ ? HB_P_EQ
                          : (q.kind == HB_P_CONTAIN_GE || q.kind == HB_P_TOKEN_JACCARD_GE) ? HB_P_JACCARD_GE : q.kind;
        f[kslot] = 1.f;
        if (q.kind == HB_P_ED_LE) f[5] = q.k / 8.f;
        if (q.kind == HB_P_EQ_PREFIX) f[5] = q.k / 8.f;
        if (q.kind == HB_P_JACCARD_GE || q.kind == HB_P_CONTAIN_GE || q.kind == HB_P_TOKEN_JACCARD_GE) {
            f[6] = (float)q.num / (float)q.den;
            f[7] = q.q / 4.f;
        }
        if (q.kind == HB_P_ABSDIFF_LE) f[8] = std::log1p(q.delta);
        const int k = op_of[p];
        double ev = 0;
        if (k >= 0) {
            const unsigned long long *v = &ctr[(size_t)k * 6];
            ev = (double)v[0];
            const double e1 = std::max(ev, 1.0);
            const double pr = ev > 0 ? v[1] / e1 : 0.5;
            f[9] = (float)pr;
            f[10] = logit_clamped(pr) / 12.f;
            f[11] = (float)(std::log(std::max(v[2] / e1, 1.0)) / 10.0);
            f[12] = (float)(v[3] / e1);
            f[13] = (float)(v[4] / e1);
            f[14] = (float)(std::log1p(v[5] / e1) / 5.0);
        }
        f[15] = p < (int)c->plain_sp.size() ? (float)c->plain_sp[p] : 0.f;
        f[16] = p < (int)c->plain_cost.size() ? (float)c->plain_cost[p] : 0.f;
        if (p < (int)c->pred_stats.size()) {
            const std::vector<float> &s = c->pred_stats[p];
            for (int i = 0; i < 6; i++) f[17 + i] = std::log1p(std::max(s[i], 0.f)) / 5.f;
            f[23] = std::log1p(std::max(s[6], 0.f)) / 5.f;
            f[24] = std::log1p(std::max(s[7], 0.f)) / 5.f;
            f[25] = s[8];
        }
        f[26] = (float)(std::log1p(ev) / 20.0);
        int nmd = 0;
        double msz = 0;
        for (auto &md : c->md_preds)
            if (std::find(md.begin(), md.end(), p) != md.end()) {
                nmd++;
                msz += md.size();
            }
        f[27] = nmd / 16.f;
        f[28] = nmd ? (float)(msz / nmd / 10.0) : 0.f;
        f[29] = (float)(std::log1p((double)res.cand) / 25.0);
        f[30] = (float)(ev / std::max<double>((double)res.cand, 1.0));
        f[31] = 1.f;
    }
    return HB_OK;
}

// Predicted (sp, cost) of every predicate from the two networks (bf16
// inference): the selectivity net gives the logit of the pass rate, the cost
// net the log of device cycles per evaluation.  Equality predicates are
// decided by blocking and keep the rule- and data-aware values.
hb_status learned_stats(hb_ctx *c, std::vector<double> &sp, std::vector<double> &cost, bool &ok) {
    ok = false;
    if (!c->model_ok || c->model.size() != 2 * (size_t)HB_MLP_PARAMS) return HB_OK;
    HB_TRY(ensure_ready(c, c->batch_layout));
    std::vector<float> F;
    HB_TRY(predicate_features(c, F));
    const int P = (int)c->preds.size();
    if (P == 0) return HB_OK;
    Buf x, prm, y;
    HB_TRY(grow(c, x, sizeof(float) * F.size()));
    HB_TRY(grow(c, prm, sizeof(float) * c->model.size()));
    HB_TRY(grow(c, y, sizeof(float) * 2 * P));
    HB_CUDA(cudaMemcpyAsync(x.p, F.data(), sizeof(float) * F.size(), cudaMemcpyHostToDevice, c->stream));
    HB_CUDA(cudaMemcpyAsync(prm.p, c->model.data(), sizeof(float) * c->model.size(), cudaMemcpyHostToDevice,
                            c->stream));
    HB_CUDA(mlp_forward(as<float>(x), P, as<float>(prm), as<float>(y), 1, c->stream));
    HB_CUDA(mlp_forward(as<float>(x), P, as<float>(prm) + HB_MLP_PARAMS, as<float>(y) + P, 1, c->stream));
    std::vector<float> out(2 * P);
    HB_CUDA(cudaMemcpyAsync(out.data(), y.p, sizeof(float) * out.size(), cudaMemcpyDeviceToHost, c->stream));
    HB_CUDA(cudaStreamSynchronize(c->stream));
    free_buf(c, x);
    free_buf(c, prm);
    free_buf(c, y);
    std::vector<double> lc(P, 0.0);
    double mx = 0;
    for (int p = 0; p < P; p++) {
        if (c->preds[p].eq_index >= 0) continue;
        const double lcost = out[p], lsel = out[P + p];
        if (!std::isfinite(lcost) || !std::isfinite(lsel) || std::fabs(lcost) > 60 || std::fabs(lsel) > 60)
            return HB_OK;   // unusable prediction: the rule- and data-aware plan stays
        lc[p] = std::exp(lcost);
        mx = std::max(mx, lc[p]);
        sp[p] = 1.0 / (1.0 + std::exp(-lsel));
    }
    for (int p = 0; p < P; p++) {
        if (c->preds[p].eq_index >= 0) cost[p] = 1e-3;
        else cost[p] = mx > 0 ? std::max(lc[p] / mx, 1e-6) : 1.0;
        sp[p] = std::min(std::max(sp[p], 1e-6), 1.0);
    }
    ok = true;
    return HB_OK;
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
    HB_TRY(predicate_features(c, feats));
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
        // time of the predicate when it is evaluated first: every candidate pair
        // pays its cheap filter on staged operands (a fixed FILTER_CYCLES), and
        // the pairs that pass the filter pay the measured full evaluation
        const double pass_filter = L.kind == HB_P_ABSDIFF_LE ? (double)v[1] / ev : (double)v[3] / ev;
        L.log_cost = (float)std::log(FILTER_CYCLES + pass_filter * std::max((double)v[2] / ev, 1.0));
        L.logit_pass = logit_clamped(v[0] ? (double)v[1] / ev : 0.5);
        memcpy(L.features, &feats[(size_t)c->program[k] * HB_FEATURES], sizeof(float) * HB_FEATURES);
    }
    *n_out = n_ops;
    return HB_OK;
}

extern "C" hb_status hb_predicate_features(hb_ctx *c, float *features_out, int32_t cap_preds, int32_t *n_out) {
    if (!c || !features_out || !n_out) return fail(HB_ERR_ARG, "hb_predicate_features: NULL argument");
    *n_out = 0;
    cudaSetDevice(c->device);
    HB_TRY(ensure_ready(c, false));
    std::vector<float> F;
    HB_TRY(predicate_features(c, F));
    const int P = (int)c->preds.size();
    if (P > cap_preds) return fail(HB_ERR_OVERFLOW, "hb_predicate_features: capacity below the predicate count");
    memcpy(features_out, F.data(), sizeof(float) * F.size());
    *n_out = P;
    return HB_OK;
}

namespace hb {

// One network trained with the library's kernels: full-batch forward /
// backward (MSE) and Adam, on standardized inputs and targets; the
// standardization is folded into the first and last layers afterwards so the
// stored network maps raw features to raw targets.
static hb_status train_one(hb_ctx *c, int n, const std::vector<float> &Xn, const std::vector<float> &t_raw, int epochs,
                           float lr, uint64_t seed, const std::vector<double> &mu, const std::vector<double> &sd,
                           float *params_out, float &loss) {
    const int NP = HB_MLP_PARAMS;
    double tm = 0, tv = 0;
    for (float v : t_raw) tm += v;
    tm /= n;
    for (float v : t_raw) tv += (v - tm) * (v - tm);
    const double ts = std::max(std::sqrt(tv / n), 1e-3);
    std::vector<float> tn(n);
    for (int i = 0; i < n; i++) tn[i] = (float)((t_raw[i] - tm) / ts);
    // He-uniform initial weights, zero biases
    std::vector<float> w(NP, 0.f);
    std::mt19937_64 rng(seed);
    auto fill = [&](int off, int fan_in, int count) {
        const double lim = std::sqrt(6.0 / fan_in);
        std::uniform_real_distribution<double> u(-lim, lim);
        for (int i = 0; i < count; i++) w[off + i] = (float)u(rng);
    };
    fill(0, 32, 32 * 64);
    fill(32 * 64 + 64, 64, 64 * 64);
    fill(32 * 64 + 64 + 64 * 64 + 64, 64, 64);
    Buf bx, bt, bp, bg, bm, bv, bw, by;
    HB_TRY(grow(c, bx, sizeof(float) * Xn.size()));
    HB_TRY(grow(c, bt, sizeof(float) * n));
    HB_TRY(grow(c, bp, sizeof(float) * NP));
    HB_TRY(grow(c, bg, sizeof(float) * NP));
    HB_TRY(grow(c, bm, sizeof(float) * NP));
    HB_TRY(grow(c, bv, sizeof(float) * NP));
    HB_TRY(grow(c, bw, sizeof(float) * mlp_work_floats(n)));
    HB_TRY(grow(c, by, sizeof(float) * n));
    HB_CUDA(cudaMemcpyAsync(bx.p, Xn.data(), sizeof(float) * Xn.size(), cudaMemcpyHostToDevice, c->stream));
    HB_CUDA(cudaMemcpyAsync(bt.p, tn.data(), sizeof(float) * n, cudaMemcpyHostToDevice, c->stream));
    HB_CUDA(cudaMemcpyAsync(bp.p, w.data(), sizeof(float) * NP, cudaMemcpyHostToDevice, c->stream));
    HB_CUDA(cudaMemsetAsync(bm.p, 0, sizeof(float) * NP, c->stream));
    HB_CUDA(cudaMemsetAsync(bv.p, 0, sizeof(float) * NP, c->stream));
    for (int e = 1; e <= epochs; e++) {
        HB_CUDA(mlp_backward(as<float>(bx), as<float>(bt), n, as<float>(bp), as<float>(bg), as<float>(bw), c->stream));
        HB_CUDA(adam_step(as<float>(bp), as<float>(bg), as<float>(bm), as<float>(bv), NP, e, lr, 0.9f, 0.999f, 1e-8f,
                          c->stream));
    }
    HB_CUDA(mlp_forward(as<float>(bx), n, as<float>(bp), as<float>(by), 0, c->stream));
    std::vector<float> y(n);
    HB_CUDA(cudaMemcpyAsync(y.data(), by.p, sizeof(float) * n, cudaMemcpyDeviceToHost, c->stream));
    HB_CUDA(cudaMemcpyAsync(w.data(), bp.p, sizeof(float) * NP, cudaMemcpyDeviceToHost, c->stream));
    HB_CUDA(cudaStreamSynchronize(c->stream));
    Buf *bufs[] = {&bx, &bt, &bp, &bg, &bm, &bv, &bw, &by};
    for (Buf *b : bufs) free_buf(c, *b);
    double l = 0;
    for (int i = 0; i < n; i++) l += (double)(y[i] - tn[i]) * (y[i] - tn[i]);
    loss = (float)(l / n);
    // fold x_n = (x - mu) / sd into layer 1 and y = y_n * ts + tm into layer 3
    float *W1 = w.data(), *b1 = W1 + 32 * 64, *W3 = w.data() + 32 * 64 + 64 + 64 * 64 + 64, *b3 = W3 + 64;
    for (int j = 0; j < 64; j++) {
        double shift = 0;
        for (int i = 0; i < 32; i++) {
            shift += mu[i] / sd[i] * W1[i * 64 + j];
            W1[i * 64 + j] = (float)(W1[i * 64 + j] / sd[i]);
        }
        b1[j] = (float)(b1[j] - shift);
    }
    for (int j = 0; j < 64; j++) W3[j] = (float)(W3[j] * ts);
    b3[0] = (float)(b3[0] * ts + tm);
    memcpy(params_out, w.data(), sizeof(float) * NP);
    return HB_OK;
}

}  // namespace hb

extern "C" hb_status hb_train_cost_model(hb_ctx *c, int32_t n, const float *X, const float *y_cost,
                                         const float *y_sel, int32_t epochs, float lr, uint64_t seed,
                                         float *loss_out) {
    if (!c || n < 2 || !X || !y_cost || !y_sel || epochs < 1 || !(lr > 0.f))
        return fail(HB_ERR_ARG, "hb_train_cost_model: needs >= 2 rows, epochs >= 1, lr > 0");
    for (size_t i = 0; i < (size_t)n * HB_FEATURES; i++)
        if (!std::isfinite(X[i])) return fail(HB_ERR_ARG, "hb_train_cost_model: non-finite feature");
    for (int i = 0; i < n; i++)
        if (!std::isfinite(y_cost[i]) || !std::isfinite(y_sel[i]))
            return fail(HB_ERR_ARG, "hb_train_cost_model: non-finite target");
    cudaSetDevice(c->device);
    std::vector<double> mu(HB_FEATURES, 0.0), sd(HB_FEATURES, 0.0);
    for (int i = 0; i < n; i++)
        for (int f = 0; f < HB_FEATURES; f++) mu[f] += X[(size_t)i * HB_FEATURES + f];
    for (int f = 0; f < HB_FEATURES; f++) mu[f] /= n;
    for (int i = 0; i < n; i++)
        for (int f = 0; f < HB_FEATURES; f++) {
            const double d = X[(size_t)i * HB_FEATURES + f] - mu[f];
            sd[f] += d * d;
        }
    for (int f = 0; f < HB_FEATURES; f++) {
        sd[f] = std::sqrt(sd[f] / n);
        if (sd[f] < 1e-6) sd[f] = 1.0;
    }
    std::vector<float> Xn((size_t)n * HB_FEATURES);
    for (int i = 0; i < n; i++)
        for (int f = 0; f < HB_FEATURES; f++)
            Xn[(size_t)i * HB_FEATURES + f] = (float)((X[(size_t)i * HB_FEATURES + f] - mu[f]) / sd[f]);
    std::vector<float> model(2 * (size_t)HB_MLP_PARAMS);
    float loss[2] = {0, 0};
    HB_TRY(train_one(c, n, Xn, std::vector<float>(y_cost, y_cost + n), epochs, lr, seed, mu, sd, model.data(),
                     loss[0]));
    HB_TRY(train_one(c, n, Xn, std::vector<float>(y_sel, y_sel + n), epochs, lr, seed + 1, mu, sd,
                     model.data() + HB_MLP_PARAMS, loss[1]));
    for (float v : model)
        if (!std::isfinite(v)) return fail(HB_ERR_INTERNAL, "hb_train_cost_model: training diverged");
    c->model = model;
    c->model_ok = true;
    if (loss_out) {
        loss_out[0] = loss[0];
        loss_out[1] = loss[1];
    }
    return HB_OK;
}


// ---------------------------------------------------------------------------
// The paper's per-pair cost model N: per-pair timing logs, kernels and trainer
// ---------------------------------------------------------------------------
extern "C" hb_status hb_time_pairs(hb_ctx *c, int32_t pred, int32_t n, const uint32_t *pi, const uint32_t *pj,
                                   uint32_t *cycles_out, uint8_t *verdict_out, float *features_out) {
    if (!c || n < 0 || (n > 0 && (!pi || !pj || !cycles_out || !verdict_out || !features_out)))
        return fail(HB_ERR_ARG, "hb_time_pairs: bad arguments");
    cudaSetDevice(c->device);
    HB_TRY(ensure_ready(c, false));
    int k = -1;
    for (size_t q = 0; q < c->program.size(); q++)
        if (c->program[q] == pred) k = (int)q;
    if (k < 0) return fail(HB_ERR_ARG, "hb_time_pairs: pred is not a non-equality predicate of the plan's program");
    const int kind = c->ops[k].kind;
    if (kind != OP_ED && kind != OP_JAC && kind != OP_ABS)
        return fail(HB_ERR_ARG, "hb_time_pairs: the per-pair model covers edit distance, Jaccard and |a-b|");
    const bool self = is_self(c);
    const int64_t nr = c->side[0].n, ns = self ? nr : c->side[1].n;
    for (int32_t t = 0; t < n; t++)
        if ((int64_t)pi[t] >= nr || (int64_t)pj[t] >= ns) return fail(HB_ERR_ARG, "hb_time_pairs: row out of range");
    if (n == 0) return HB_OK;
    Buf dev;
    const size_t n8 = (size_t)n;
    HB_TRY(grow(c, dev, n8 * (4 + 4 + 4 + 1 + 4 * HB_PAIR_FEATURES) + 256));
    uint32_t *di = as<uint32_t>(dev), *dj = di + n8, *dc = dj + n8;
    float *dX = reinterpret_cast<float *>(dc + n8);
    uint8_t *dv = reinterpret_cast<uint8_t *>(dX + n8 * HB_PAIR_FEATURES);
    HB_CUDA(cudaMemcpyAsync(di, pi, 4 * n8, cudaMemcpyHostToDevice, c->stream));
    HB_CUDA(cudaMemcpyAsync(dj, pj, 4 * n8, cudaMemcpyHostToDevice, c->stream));
    EvalParams P = make_params(c, c->side[0].rec, self ? c->side[0].rec : c->side[1].rec, 1, self,
                               as<unsigned long long>(c->w_counters), 32);
    HB_CUDA(launch_pair_times(P, k, di, dj, n, dc, dv, dX, c->stream));
    HB_CUDA(cudaMemcpyAsync(cycles_out, dc, 4 * n8, cudaMemcpyDeviceToHost, c->stream));
    HB_CUDA(cudaMemcpyAsync(verdict_out, dv, n8, cudaMemcpyDeviceToHost, c->stream));
    HB_CUDA(cudaMemcpyAsync(features_out, dX, 4 * n8 * HB_PAIR_FEATURES, cudaMemcpyDeviceToHost, c->stream));
    HB_CUDA(cudaStreamSynchronize(c->stream));
    free_buf(c, dev);
    return HB_OK;
}

extern "C" hb_status hb_pair_model_forward(const float *X, int32_t n, const float *params, float *y, void *stream) {
    if (n < 0 || (n > 0 && (!X || !params || !y))) return fail(HB_ERR_ARG, "hb_pair_model_forward: bad arguments");
    HB_CUDA(pair_model_forward(X, n, params, y, static_cast<cudaStream_t>(stream)));
    return HB_OK;
}

extern "C" hb_status hb_pair_model_backward(const float *X, const float *t, int32_t n, const float *params,
                                            float *grad, void *stream) {
    if (n < 0 || !params || !grad || (n > 0 && (!X || !t)))
        return fail(HB_ERR_ARG, "hb_pair_model_backward: bad arguments");
    HB_CUDA(pair_model_backward(X, t, n, params, grad, static_cast<cudaStream_t>(stream)));
    return HB_OK;
}

extern "C" hb_status hb_train_pair_model(int32_t n, const float *X, const float *y, int32_t epochs, float lr,
                                         uint64_t seed, float *params_out, float *loss_out) {
    if (n < 1 || !X || !y || !params_out || epochs < 0 || !(lr > 0.f))
        return fail(HB_ERR_ARG, "hb_train_pair_model: bad arguments");
    const int PN = HB_PAIR_MODEL_PARAMS;
    // He-uniform start: fan-in 8 for W1, 2 for W2, 6 for W3; zero biases
    std::vector<float> p0(PN, 0.f);
    std::mt19937_64 rng(seed);
    std::uniform_real_distribution<double> U(-1.0, 1.0);
    const int fan[3] = {8, 2, 6}, off[3] = {0, 8 * 2 + 2, 8 * 2 + 2 + 2 * 6 + 6}, cnt[3] = {16, 12, 6};
    for (int l = 0; l < 3; l++) {
        const double lim = std::sqrt(6.0 / fan[l]);
        for (int i = 0; i < cnt[l]; i++) p0[off[l] + i] = (float)(lim * U(rng));
    }
    cudaStream_t s = nullptr;
    float *d = nullptr;
    const size_t nf = (size_t)n * HB_PAIR_FEATURES;
    cudaError_t e = cudaMallocAsync(reinterpret_cast<void **>(&d), sizeof(float) * (nf + 2 * (size_t)n + 4 * PN + 64), s);
    if (e != cudaSuccess) return fail(HB_ERR_OOM, "hb_train_pair_model: device allocation failed");
    float *dX = d, *dy = dX + nf, *dp = dy + n, *dg = dp + PN, *dm = dg + PN, *dv = dm + PN, *dout = dv + PN;
    auto done = [&](hb_status st) {
        cudaFreeAsync(d, s);
        cudaStreamSynchronize(s);
        return st;
    };
    e = cudaMemcpyAsync(dX, X, sizeof(float) * nf, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(dy, y, sizeof(float) * n, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(dp, p0.data(), sizeof(float) * PN, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(dm, 0, sizeof(float) * 2 * PN, s);
    for (int ep = 0; ep < epochs && e == cudaSuccess; ep++) {
        e = pair_model_backward(dX, dy, n, dp, dg, s);
        if (e == cudaSuccess) e = adam_step(dp, dg, dm, dv, PN, ep + 1, lr, 0.9f, 0.999f, 1e-8f, s);
    }
    if (e == cudaSuccess) e = pair_model_forward(dX, n, dp, dout, s);
    std::vector<float> out(n);
    if (e == cudaSuccess) e = cudaMemcpyAsync(params_out, dp, sizeof(float) * PN, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(out.data(), dout, sizeof(float) * n, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return done(fail(HB_ERR_CUDA, std::string("hb_train_pair_model: ") + cudaGetErrorString(e)));
    double mse = 0;
    for (int r = 0; r < n; r++) mse += (double)(out[r] - y[r]) * (out[r] - y[r]);
    if (loss_out) *loss_out = (float)(mse / n);
    for (int i = 0; i < PN; i++)
        if (!std::isfinite(params_out[i])) return done(fail(HB_ERR_INTERNAL, "hb_train_pair_model: training diverged"));
    return done(HB_OK);
}

// The tile-shape model: the same network, trained on the batch autotuner's
// measurements (features of a job-size signature and a tile shape, log ms).
extern "C" hb_status hb_train_tile_model(hb_ctx *c, int32_t n, const float *X, const float *y, int32_t epochs,
                                         float lr, uint64_t seed, float *loss_out) {
    if (!c || n < 2 || !X || !y || epochs < 1 || !(lr > 0.f))
        return fail(HB_ERR_ARG, "hb_train_tile_model: needs >= 2 rows, epochs >= 1, lr > 0");
    for (size_t i = 0; i < (size_t)n * HB_FEATURES; i++)
        if (!std::isfinite(X[i])) return fail(HB_ERR_ARG, "hb_train_tile_model: non-finite feature");
    for (int i = 0; i < n; i++)
        if (!std::isfinite(y[i])) return fail(HB_ERR_ARG, "hb_train_tile_model: non-finite target");
    cudaSetDevice(c->device);
    std::vector<double> mu(HB_FEATURES, 0.0), sd(HB_FEATURES, 0.0);
    for (int i = 0; i < n; i++)
        for (int f = 0; f < HB_FEATURES; f++) mu[f] += X[(size_t)i * HB_FEATURES + f];
    for (int f = 0; f < HB_FEATURES; f++) mu[f] /= n;
    for (int i = 0; i < n; i++)
        for (int f = 0; f < HB_FEATURES; f++) {
            const double d = X[(size_t)i * HB_FEATURES + f] - mu[f];
            sd[f] += d * d;
        }
    for (int f = 0; f < HB_FEATURES; f++) {
        sd[f] = std::sqrt(sd[f] / n);
        if (sd[f] < 1e-6) sd[f] = 1.0;
    }
    std::vector<float> Xn((size_t)n * HB_FEATURES);
    for (int i = 0; i < n; i++)
        for (int f = 0; f < HB_FEATURES; f++)
            Xn[(size_t)i * HB_FEATURES + f] = (float)((X[(size_t)i * HB_FEATURES + f] - mu[f]) / sd[f]);
    std::vector<float> model(HB_MLP_PARAMS);
    float loss = 0;
    HB_TRY(train_one(c, n, Xn, std::vector<float>(y, y + n), epochs, lr, seed, mu, sd, model.data(), loss));
    for (float v : model)
        if (!std::isfinite(v)) return fail(HB_ERR_INTERNAL, "hb_train_tile_model: training diverged");
    c->tile_model = model;
    c->tile_model_ok = true;
    c->tune_cache.clear();
    if (loss_out) *loss_out = loss;
    return HB_OK;
}
