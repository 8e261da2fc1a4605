// Batched blocking of many independent jobs (hb_block_batch) and the tile
// autotuner.
//
// The jobs are stacked row-wise in relation R.  The job id becomes one more
// equality key held by every MD, so no block spans two jobs and the whole
// batch is one self-join: one block build, ONE persistent evaluation launch
// whose work queue holds the tiles of every block of every job (Section 3:
// the host schedules partitions onto the device without interrupting it;
// Section 5.2: idle thread blocks take the next unclaimed work), one sort and
// one pass that splits the sorted pairs into per-job ranges with job-local
// row ids.  The launch sequence has no host round trip, so after its first
// eager run it is captured into a CUDA graph and replayed while the shapes
// stay the same.
//
// HB_FLAG_PER_JOB_LAUNCHES runs the same work as one launch sequence per job
// (block build, evaluation, sort, copy for each job), the comparison point.
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <vector>

#include "hb_ctx.h"

namespace hb {
namespace {

__global__ void k_localize(const uint64_t *keys, const unsigned long long *n_dev, uint64_t n_max, int key_bits_s,
                           const int64_t *job_rows, int n_jobs, hb_pair *out, uint32_t *job_count) {
    const uint64_t n = min((uint64_t)*n_dev, n_max);
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t k = keys[i];
        const int64_t a = (int64_t)(k >> key_bits_s), b = (int64_t)(k & ((1ull << key_bits_s) - 1ull));
        int lo = 0, hi = n_jobs;   // job_rows[lo] <= a < job_rows[hi]
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (job_rows[mid] <= a) lo = mid;
            else hi = mid;
        }
        hb_pair p;
        p.tid1 = (uint32_t)(a - job_rows[lo]);
        p.tid2 = (uint32_t)(b - job_rows[lo]);
        out[i] = p;
        atomicAdd(&job_count[lo], 1u);
    }
}

}  // namespace

// The batch launch sequence: no host synchronisation inside (capturable).
static hb_status batch_sequence(hb_ctx *c, int n_jobs, int key_bits, int kbs, uint32_t &block_cap, int grid,
                                size_t smem, uint64_t **sorted) {
    unsigned long long *ctr = as<unsigned long long>(c->w_counters);
    const int64_t n = c->side[0].n;
    const uint32_t *rec = c->side[0].rec;
    HB_CUDA(cudaMemsetAsync(ctr, 0, 64 * sizeof(unsigned long long), c->stream));
    HB_TRY(build_blocks(c, rec, n, rec, n, true, ctr, block_cap));
    EvalParams P = make_params(c, rec, rec, 1, true, ctr, kbs);
    HB_CUDA(launch_eval(P, grid, smem, 0, c->stream));
    radix_sort_u64(as<uint64_t>(c->w_out), as<uint64_t>(c->w_alt), c->out_cap, ctr + 1, key_bits, c->w_sort.p,
                   c->w_sort.bytes, c->stream, sorted);
    HB_CUDA(cudaMemsetAsync(c->w_jobcount.p, 0, sizeof(uint32_t) * (n_jobs + 1), c->stream));
    HB_LAUNCHED(1);
    k_localize<<<(unsigned)(4 * c->n_sm), 256, 0, c->stream>>>(*sorted, ctr + 1, (uint64_t)c->out_cap, kbs,
                                                              as<int64_t>(c->w_jobrows), n_jobs,
                                                              as<hb_pair>(c->w_pairs), as<uint32_t>(c->w_jobcount));
    scan_exclusive_u32(as<uint32_t>(c->w_jobcount), as<uint32_t>(c->w_joboff), n_jobs, nullptr, c->w_scan.p,
                       c->w_scan.bytes, c->stream);
    HB_CUDA(cudaGetLastError());
    return HB_OK;
}

static void drop_graph(hb_ctx *c) {
    if (c->batch_exec) cudaGraphExecDestroy(c->batch_exec);
    if (c->batch_graph) cudaGraphDestroy(c->batch_graph);
    c->batch_exec = nullptr;
    c->batch_graph = nullptr;
    c->batch_graph_key.clear();
}

static std::vector<int64_t> graph_key(hb_ctx *c, int n_jobs) {
    std::vector<int64_t> k = {c->side[0].n, n_jobs, c->out_cap, c->tile, c->claim, c->W, c->HW,
                              (int64_t)c->ops.size(), (int64_t)(uintptr_t)c->side[0].rec,
                              (int64_t)(uintptr_t)c->side[0].hot};
    const Buf *bufs[] = {&c->w_members_r,
                         &c->w_blocks, &c->w_tiles, &c->w_prefix, &c->w_scan, &c->w_out, &c->w_alt, &c->w_sort,
                         &c->w_pairs, &c->w_counters, &c->w_lut, &c->w_jobrows, &c->w_jobcount, &c->w_joboff};
    for (const Buf *b : bufs) k.push_back((int64_t)(uintptr_t)b->p);
    k.push_back((int64_t)(uintptr_t)c->w_small.p);
    for (const hb_ctx::MdLane &L : c->md_lanes) {
        const Buf *lb[] = {&L.table, &L.slot_r, &L.count_r, &L.start_r, &L.cursor, &L.scan, &L.meta};
        for (const Buf *b : lb) k.push_back((int64_t)(uintptr_t)b->p);
    }
    for (const Op &op : c->ops) k.push_back((int64_t)op.need ^ ((int64_t)op.cp << 1) ^ op.kind);
    return k;
}

// one measured run of the batch sequence with the given tile shape (ms)
static hb_status time_batch(hb_ctx *c, int n_jobs, int key_bits, int kbs, int tile, int claim, float &ms) {
    c->tile = tile;
    c->claim = claim;
    const size_t smem = eval_smem_bytes(c->HW, c->n_eq_total, c->lut.empty() ? 0 : 1, tile);
    const int bps = eval_blocks_per_sm(tile, 0, smem);
    if (bps < 1) {
        ms = 1e30f;
        return HB_OK;
    }
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    uint32_t cap = 0;
    uint64_t *sorted = nullptr;
    cudaEventRecord(a, c->stream);
    hb_status st = batch_sequence(c, n_jobs, key_bits, kbs, cap, bps * c->n_sm, smem, &sorted);
    cudaEventRecord(b, c->stream);
    cudaEventSynchronize(b);
    cudaEventElapsedTime(&ms, a, b);
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    return st;
}

// Features of a batch and a tile shape for the tile-shape model (HB_FEATURES
// floats): the fraction of rows in jobs of 2^(5+b) .. 2^(6+b) rows for
// b = 0..15 (smaller jobs in b = 0, larger in b = 15), log2 of the rows and of
// the jobs, the tile side (1 for 64), log2 of the tiles per claim / 3, the
// program's ops, MDs and equality keys, and log10 of the sum of squared job
// sizes / 14 (the pair volume).
static void tile_features(const hb_ctx *c, int n_jobs, int tile, int claim, float *f) {
    for (int i = 0; i < HB_FEATURES; i++) f[i] = 0.f;
    const double total = (double)std::max<int64_t>(c->job_rows[n_jobs], 1);
    double sq = 0;
    for (int j = 0; j < n_jobs; j++) {
        const int64_t s = c->job_rows[j + 1] - c->job_rows[j];
        int b = 0;
        while (b < 40 && (1ll << (b + 1)) <= s) b++;
        f[std::min(std::max(b - 5, 0), 15)] += (float)((double)s / total);
        sq += (double)s * (double)s;
    }
    f[16] = (float)(std::log2(total + 1.0) / 24.0);
    f[17] = (float)(std::log2((double)n_jobs + 1.0) / 16.0);
    f[18] = tile == 64 ? 1.f : 0.f;
    f[19] = (float)(std::log2((double)claim) / 3.0);
    f[20] = (float)c->ops.size() / 16.f;
    f[21] = (float)c->md_preds.size() / 16.f;
    f[22] = (float)c->n_eq_total / 8.f;
    f[23] = (float)(std::log10(sq + 1.0) / 14.0);
}

// Autotuner: the first time a job-size signature is seen, every candidate tile
// shape (tile side x tiles per claim) is timed on the real batch and the
// fastest is cached for the signature (log2 histogram of job sizes, job count
// and the program); each measurement is logged for the tile-shape model.
// With a tile-shape model set, the shape of smallest predicted time is taken
// instead of timing all of them.
static hb_status autotune_batch(hb_ctx *c, int n_jobs, int key_bits, int kbs) {
    if (c->opt.tile != 0) {
        c->tile = c->opt.tile;
        return HB_OK;
    }
    std::vector<int64_t> sig(33, 0);
    for (int j = 0; j < n_jobs; j++) {
        int64_t s = c->job_rows[j + 1] - c->job_rows[j];
        int b = 0;
        while (b < 31 && (1ll << (b + 1)) <= s) b++;
        sig[b]++;
    }
    sig[32] = n_jobs;
    for (const Op &op : c->ops) sig.push_back((int64_t)op.need ^ ((int64_t)op.kind << 60));
    for (auto &e : c->tune_cache)
        if (e.first == sig) {
            c->tile = e.second.first;
            c->claim = e.second.second;
            return HB_OK;
        }
    const int tiles[] = {32, 64};
    const int claims[] = {1, 2, 4, 8};
    float best = 1e30f;
    int bt = 32, bc = 2;
    if (c->tile_model_ok) {
        // the tile-shape model's argmin over the same candidates (bf16 inference, no trial runs)
        float F[8 * HB_FEATURES], y[8];
        int k = 0;
        for (int t : tiles)
            for (int cl : claims) tile_features(c, n_jobs, t, cl, F + (size_t)HB_FEATURES * k++);
        Buf d;
        HB_TRY(grow(c, d, sizeof(float) * (8 * HB_FEATURES + 8 + HB_MLP_PARAMS)));
        float *dX = as<float>(d), *dy = dX + 8 * HB_FEATURES, *dp = dy + 8;
        HB_CUDA(cudaMemcpyAsync(dX, F, sizeof(F), cudaMemcpyHostToDevice, c->stream));
        HB_CUDA(cudaMemcpyAsync(dp, c->tile_model.data(), sizeof(float) * HB_MLP_PARAMS, cudaMemcpyHostToDevice,
                                c->stream));
        HB_CUDA(mlp_forward(dX, 8, dp, dy, 1, c->stream));
        HB_CUDA(cudaMemcpyAsync(y, dy, sizeof(y), cudaMemcpyDeviceToHost, c->stream));
        HB_CUDA(cudaStreamSynchronize(c->stream));
        free_buf(c, d);
        k = 0;
        bool ok = true;
        for (int t : tiles)
            for (int cl : claims) {
                ok = ok && std::isfinite(y[k]);
                const size_t smem = eval_smem_bytes(c->HW, c->n_eq_total, c->lut.empty() ? 0 : 1, t);
                if (eval_blocks_per_sm(t, 0, smem) >= 1 && y[k] < best) {
                    best = y[k];
                    bt = t;
                    bc = cl;
                }
                k++;
            }
        if (ok && best < 1e30f) {
            c->tile = bt;
            c->claim = bc;
            c->tune_learned = 1;
            c->tune_cache.push_back({sig, {bt, bc}});
            return HB_OK;
        }
        best = 1e30f;   // unusable predictions: measure
    }
    c->tune_learned = 0;
    for (int t : tiles)
        for (int cl : claims) {
            float ms = 0;
            HB_TRY(time_batch(c, n_jobs, key_bits, kbs, t, cl, ms));
            if (ms < 1e29f) {
                float F[HB_FEATURES];
                tile_features(c, n_jobs, t, cl, F);
                c->tune_log.insert(c->tune_log.end(), F, F + HB_FEATURES);
                c->tune_log.push_back((float)std::log(std::max(ms, 1e-3f)));
            }
            if (ms < best) {
                best = ms;
                bt = t;
                bc = cl;
            }
        }
    c->tile = bt;
    c->claim = bc;
    c->tune_cache.push_back({sig, {bt, bc}});
    return HB_OK;
}

static hb_status per_job(hb_ctx *c, int n_jobs, const int64_t *job_rows, hb_pair **pairs_out, int64_t *job_pairs_out) {
    if (!c->planned || c->batch_layout) HB_TRY(do_plan(c, HB_PLAN_RULE_DATA, false));
    HB_TRY(ensure_ready(c, false));
    if (c->opt.tile) c->tile = c->opt.tile;
    std::vector<hb_pair> all;
    job_pairs_out[0] = 0;
    int64_t cand = 0, tiles = 0;
    const uint32_t *rec = c->side[0].rec;
    const uint32_t *hot = c->side[0].hot;
    for (int j = 0; j < n_jobs; j++) {
        const int64_t a = job_rows[j], nj = job_rows[j + 1] - job_rows[j];
        const int kbs = bits_for((uint64_t)std::max<int64_t>(nj, 2));
        const int kb = 2 * kbs;
        // evaluate the job's rows as a table of its own: shift the record bases
        uint32_t *save_rec = c->side[0].rec, *save_hot = c->side[0].hot;
        c->side[0].rec = const_cast<uint32_t *>(rec) + (size_t)a * c->W;
        c->side[0].hot = const_cast<uint32_t *>(hot) + (size_t)a * c->HW;
        RunResult res;
        uint64_t *sorted = nullptr;
        hb_status st = block_eval_sort(c, c->side[0].rec, nj, c->side[0].rec, nj, true, 1, kb, kbs, 0, res, &sorted,
                                       nullptr);
        hb_pair *h = nullptr;
        if (st == HB_OK) st = check_bounds(c, "hb_block_batch");
        if (st == HB_OK) st = deliver(c, sorted, res.n_out, kbs, true, &h);
        c->side[0].rec = save_rec;
        c->side[0].hot = save_hot;
        if (st != HB_OK) return st;
        all.insert(all.end(), h, h + res.n_out);
        free(h);
        job_pairs_out[j + 1] = job_pairs_out[j] + res.n_out;
        cand += res.cand;
        tiles += res.tiles;
    }
    hb_pair *out = static_cast<hb_pair *>(malloc(sizeof(hb_pair) * std::max<size_t>(all.size(), 1)));
    if (!out) return fail(HB_ERR_OOM, "host allocation of the result failed");
    if (!all.empty()) memcpy(out, all.data(), sizeof(hb_pair) * all.size());
    *pairs_out = out;
    c->stats.candidate_pairs = cand;
    c->stats.emitted_pairs = (int64_t)all.size();
    c->stats.tiles = tiles;
    return HB_OK;
}

}  // namespace hb

using namespace hb;

extern "C" hb_status hb_block_batch(hb_ctx *c, int32_t n_jobs, const int64_t *job_rows, hb_pair **pairs_out,
                                    int64_t *job_pairs_out) {
    if (!c || !job_rows || !pairs_out || !job_pairs_out) return fail(HB_ERR_ARG, "hb_block_batch: NULL argument");
    *pairs_out = nullptr;
    if (n_jobs < 1) return fail(HB_ERR_ARG, "hb_block_batch: n_jobs must be >= 1");
    if (!is_self(c)) return fail(HB_ERR_STATE, "hb_block_batch: jobs are stacked in R only (do not load S)");
    if (c->shard_world > 1) return fail(HB_ERR_STATE, "hb_block_batch: sharded evaluation runs on hb_block only");
    const int64_t n = c->side[0].n;
    if (job_rows[0] != 0 || job_rows[n_jobs] != n)
        return fail(HB_ERR_ARG, "hb_block_batch: job_rows must start at 0 and end at the row count of R");
    for (int j = 0; j < n_jobs; j++)
        if (job_rows[j + 1] < job_rows[j]) return fail(HB_ERR_ARG, "hb_block_batch: job_rows must not decrease");
    cudaSetDevice(c->device);
    auto w0 = std::chrono::steady_clock::now();
    if (c->opt.flags & HB_FLAG_PER_JOB_LAUNCHES) {
        HB_TRY(per_job(c, n_jobs, job_rows, pairs_out, job_pairs_out));
        c->stats.ms_total = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - w0).count();
        return HB_OK;
    }
    std::vector<int64_t> jr(job_rows, job_rows + n_jobs + 1);
    if (jr != c->job_rows) {
        c->job_rows = jr;
        c->planned = false;   // the job key changes the layout and the encoding
        drop_graph(c);
    }
    if (!c->planned || !c->batch_layout) {
        c->planned = false;
        HB_TRY(do_plan(c, HB_PLAN_RULE_DATA, true));
    }
    HB_TRY(ensure_ready(c, true));
    HB_TRY(grow(c, c->w_jobrows, sizeof(int64_t) * (n_jobs + 1)));
    HB_CUDA(cudaMemcpyAsync(c->w_jobrows.p, jr.data(), sizeof(int64_t) * (n_jobs + 1), cudaMemcpyHostToDevice,
                            c->stream));
    HB_TRY(grow(c, c->w_jobcount, sizeof(uint32_t) * (n_jobs + 2)));
    HB_TRY(grow(c, c->w_joboff, sizeof(uint32_t) * (n_jobs + 2)));
    const int kbs = bits_for((uint64_t)std::max<int64_t>(n, 2));
    const int kb = 2 * kbs;
    if (c->out_cap == 0) c->out_cap = c->opt.out_capacity > 0 ? c->opt.out_capacity : std::max<int64_t>(1 << 20, n);
    for (int attempt = 0; attempt < 3; attempt++) {
        HB_TRY(grow(c, c->w_out, sizeof(uint64_t) * (size_t)c->out_cap));
        HB_TRY(grow(c, c->w_alt, sizeof(uint64_t) * (size_t)c->out_cap));
        HB_TRY(grow(c, c->w_sort, radix_tmp_bytes(c->out_cap)));
        HB_TRY(grow(c, c->w_pairs, sizeof(hb_pair) * (size_t)c->out_cap));
        HB_TRY(grow(c, c->w_scan, scan_tmp_bytes(n_jobs + 1)));
        HB_TRY(autotune_batch(c, n_jobs, kb, kbs));
        const size_t smem = eval_smem_bytes(c->HW, c->n_eq_total, c->lut.empty() ? 0 : 1, c->tile);
        const int bps = eval_blocks_per_sm(c->tile, 0, smem);
        if (bps < 1) return fail(HB_ERR_ARG, "record too wide for the evaluation kernel's shared memory");
        const int grid = bps * c->n_sm;
        uint32_t cap = 0;
        uint64_t *sorted = nullptr;
        const bool use_graph = !(c->opt.flags & HB_FLAG_NO_GRAPH);
        std::vector<int64_t> key = graph_key(c, n_jobs);
        if (use_graph && c->batch_exec && key == c->batch_graph_key) {
            HB_CUDA(cudaGraphLaunch(c->batch_exec, c->stream));
            HB_LAUNCHED(c->graph_kernels);
        } else {
            drop_graph(c);
            HB_TRY(batch_sequence(c, n_jobs, kb, kbs, cap, grid, smem, &sorted));
            HB_CUDA(cudaStreamSynchronize(c->stream));
            if (use_graph) {
                // record the same sequence for replays (buffers are already large enough)
                const long long before = g_kernel_launches.load();
                HB_CUDA(cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal));
                hb_status st = batch_sequence(c, n_jobs, kb, kbs, cap, grid, smem, &sorted);
                cudaGraph_t g = nullptr;
                cudaError_t e = cudaStreamEndCapture(c->stream, &g);
                if (st != HB_OK) {
                    if (g) cudaGraphDestroy(g);
                    return st;
                }
                HB_CUDA(e);
                c->batch_graph = g;
                HB_CUDA(cudaGraphInstantiate(&c->batch_exec, g, 0));
                c->batch_graph_key = key;
                c->graph_kernels = g_kernel_launches.load() - before;
                g_kernel_launches.fetch_sub(c->graph_kernels);
            }
        }
        unsigned long long h[8];
        HB_CUDA(cudaMemcpyAsync(h, c->w_counters.p, sizeof(h), cudaMemcpyDeviceToHost, c->stream));
        HB_CUDA(cudaStreamSynchronize(c->stream));
        if (h[4]) return fail(HB_ERR_INTERNAL, "block list overflow");
        const int64_t n_out = (int64_t)h[1];
        // job offsets are 32-bit on the device
        if (n_out >= (int64_t)(1ll << 32)) return fail(HB_ERR_OVERFLOW, "hb_block_batch: 2^32 or more result pairs");
        if (n_out > c->out_cap) {
            c->out_cap = n_out + n_out / 8 + 1024;
            drop_graph(c);
            continue;
        }
        HB_TRY(check_bounds(c, "hb_block_batch"));
        std::vector<uint32_t> off(n_jobs + 1);
        HB_CUDA(cudaMemcpyAsync(off.data(), c->w_joboff.p, sizeof(uint32_t) * (n_jobs + 1), cudaMemcpyDeviceToHost,
                                c->stream));
        hb_pair *out = static_cast<hb_pair *>(malloc(sizeof(hb_pair) * (size_t)std::max<int64_t>(n_out, 1)));
        if (!out) return fail(HB_ERR_OOM, "host allocation of the result failed");
        if (n_out > 0) {
            cudaError_t e = cudaMemcpyAsync(out, c->w_pairs.p, sizeof(hb_pair) * (size_t)n_out, cudaMemcpyDeviceToHost,
                                            c->stream);
            if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
            if (e != cudaSuccess) {
                free(out);
                return fail(HB_ERR_CUDA, std::string("result copy: ") + cudaGetErrorString(e));
            }
        } else {
            HB_CUDA(cudaStreamSynchronize(c->stream));
        }
        for (int j = 0; j <= n_jobs; j++) job_pairs_out[j] = off[j];
        *pairs_out = out;
        c->stats.candidate_pairs = (int64_t)h[2];
        c->stats.examined_pairs = (int64_t)h[5];
        c->stats.emitted_pairs = n_out;
        c->stats.blocks = (int64_t)(uint32_t)h[3] - (int64_t)(uint32_t)h[6] + (int64_t)(uint32_t)h[7];
        c->stats.tile = c->tile;
        c->stats.ms_total = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - w0).count();
        return HB_OK;
    }
    return fail(HB_ERR_OVERFLOW, "hb_block_batch: result capacity could not be settled");
}

extern "C" hb_status hb_tile_log(hb_ctx *c, int32_t cap, float *X_out, float *y_out, int32_t *n_out) {
    if (!c || !n_out || (cap > 0 && (!X_out || !y_out))) return fail(HB_ERR_ARG, "hb_tile_log: bad arguments");
    const int rows = (int)(c->tune_log.size() / (HB_FEATURES + 1));
    *n_out = rows;
    for (int r = 0; r < rows && r < cap; r++) {
        memcpy(X_out + (size_t)r * HB_FEATURES, &c->tune_log[(size_t)r * (HB_FEATURES + 1)], sizeof(float) * HB_FEATURES);
        y_out[r] = c->tune_log[(size_t)r * (HB_FEATURES + 1) + HB_FEATURES];
    }
    return HB_OK;
}

extern "C" hb_status hb_set_tile_model(hb_ctx *c, const float *params) {
    if (!c) return fail(HB_ERR_ARG, "hb_set_tile_model: ctx is NULL");
    c->tune_cache.clear();
    if (!params) {
        c->tile_model.clear();
        c->tile_model_ok = false;
        return HB_OK;
    }
    for (int i = 0; i < HB_MLP_PARAMS; i++)
        if (!std::isfinite(params[i])) return fail(HB_ERR_ARG, "hb_set_tile_model: non-finite parameter");
    c->tile_model.assign(params, params + HB_MLP_PARAMS);
    c->tile_model_ok = true;
    return HB_OK;
}

extern "C" hb_status hb_get_tile_model(hb_ctx *c, float *params_out) {
    if (!c || !params_out) return fail(HB_ERR_ARG, "hb_get_tile_model: NULL argument");
    if (!c->tile_model_ok) return fail(HB_ERR_STATE, "hb_get_tile_model: no tile model trained or set");
    memcpy(params_out, c->tile_model.data(), sizeof(float) * HB_MLP_PARAMS);
    return HB_OK;
}

extern "C" hb_status hb_batch_tile(const hb_ctx *c, int32_t *tile, int32_t *claim, int32_t *learned) {
    if (!c || !tile || !claim || !learned) return fail(HB_ERR_ARG, "hb_batch_tile: NULL argument");
    *tile = c->tile;
    *claim = c->claim;
    *learned = c->tune_learned;
    return HB_OK;
}
