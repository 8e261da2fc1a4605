// Context of the libhb C-ABI (shared by the host-side translation units).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <deque>
#include <vector>

#include "hb_internal.h"

namespace hb {

hb_status fail(hb_status st, const std::string &msg);

#define HB_CUDA(call)                                                                              \
    do {                                                                                           \
        cudaError_t e__ = (call);                                                                  \
        if (e__ != cudaSuccess)                                                                    \
            return ::hb::fail(e__ == cudaErrorMemoryAllocation ? HB_ERR_OOM : HB_ERR_CUDA,         \
                              std::string(#call) + ": " + cudaGetErrorString(e__));                \
    } while (0)

#define HB_TRY(expr)                  \
    do {                              \
        hb_status s__ = (expr);       \
        if (s__ != HB_OK) return s__; \
    } while (0)

static inline uint64_t pow2_at_least(uint64_t x) {
    uint64_t p = 1;
    while (p < x) p <<= 1;
    return p;
}
static inline int bits_for(uint64_t n) {   // bits to hold values 0..n-1 (at least 1)
    int b = 1;
    while (b < 63 && (1ull << b) < n) b++;
    return b;
}

struct EqKey {
    int col_t, col_s, prefix;   // prefix < 0: whole value
};
struct FeatGroup {
    int kind;   // OP_ED, OP_JAC, OP_ABS, OP_EQX, OP_CONST, OP_CONT (uses the OP_JAC groups)
    int col_t, col_s, q;
    int word;
    int tokens = 0;   // OP_JAC: 1 = word-token codes instead of q-grams
    int pred = -1;    // OP_CONST: the predicate whose constant the flag word tests
};
struct PredInfo {
    hb_predicate p;
    int eq_index = -1;   // equality key (EQ / EQ_PREFIX)
    int group = -1;      // feature group (others)
};

// device buffer that grows on demand (stream-ordered allocator)
struct Buf {
    void *p = nullptr;
    size_t bytes = 0;
};

struct SideData {
    int64_t n = 0;
    std::vector<DevCol> cols;
    std::vector<void *> allocs;
    // encoded state
    uint32_t *rec = nullptr;
    uint32_t *hot = nullptr;   // per tuple: equality codes + one filter word per feature group (+ bin counts)
    std::vector<int32_t> hot_map;   // layout the hot records were packed with
    std::vector<uint32_t *> grams;   // per feature group (JAC only)
    std::vector<uint64_t> gram_len;  // entries of grams[g]
    bool encoded = false;
};

}  // namespace hb

using hb::Buf;
using hb::DevCol;
using hb::EqKey;
using hb::FeatGroup;
using hb::Op;
using hb::PredInfo;
using hb::SideData;

struct hb_ctx {
    int device = 0;
    int n_sm = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    hb_options opt{};
    SideData side[2];
    // rules
    std::vector<std::vector<hb_predicate>> md_raw;
    std::deque<std::string> consts;   // constants of CONST_EQ predicates (md_raw points here)
    int n_user_mds = 0;               // MDs added; md_preds also holds transposed copies (self-join)
    // Section 5.3 data partitioning (hb_set_partitions): m partitions per
    // root-edge hash function, 0 = exact equality groups; when partitioned,
    // one grouping MD per root branch follows the rules' MDs in eqset
    int64_t fail_alloc_after = -1;   // HB_FAIL_ALLOC_AFTER fault injection (-1: off)
    uint32_t part_m = 0;
    // sharded evaluation (hb_set_shard): this process evaluates the blocks owned by rank
    uint32_t shard_rank = 0, shard_world = 1;
    uint32_t layout_part_m = 0;       // part_m the layout was built for
    uint64_t group_mds = 0;           // bits of the grouping MDs
    std::vector<int> branch_key;      // per branch: equality key index (-1: one partition of all tuples)
    std::vector<int> branch_pred;     // per branch: its root predicate (-1: none)
    // plan
    bool planned = false;
    bool batch_layout = false;   // extra job key
    std::vector<PredInfo> preds;
    std::vector<std::vector<int>> md_preds;
    std::vector<EqKey> eqkeys;
    std::vector<FeatGroup> groups;
    int W = 4;
    int HW = 4;
    std::vector<int32_t> hot_map;   // hot word -> record word (-1: zero)
    int n_eq_total = 0;            // eqkeys + job key
    std::vector<uint16_t> eqset;
    std::vector<int> active;       // MDs whose blocks can own pairs
    std::vector<int> program;      // predicate ids
    std::vector<Op> ops;
    uint64_t eqonly = 0;
    std::vector<uint64_t> lut;
    hb_plan_info info{};
    int tile = 32;
    // R-side dictionaries (kept for probing S)
    std::vector<uint64_t *> dict;
    std::vector<uint64_t> dict_cap;
    // word-token dictionaries of R's token groups (kept to probe S's tokens)
    struct TokDict {
        uint64_t *table = nullptr;
        uint64_t cap = 0;
        uint32_t *start = nullptr, *len = nullptr;
        const uint8_t *bytes = nullptr;
    };
    std::vector<TokDict> tok;
    // work buffers
    Buf w_slot_r, w_slot_s, w_count_s, w_start_s, w_cursor, w_members_r,
        w_members_s, w_blocks, w_tiles, w_prefix, w_scan, w_out, w_alt, w_sort, w_pairs, w_counters, w_lut, w_log,
        w_jac;
    int64_t out_cap = 0;
    // stats
    hb_stats stats{};
    // learned model: [cost net | selectivity net]
    std::vector<float> model;
    bool model_ok = false;
    // tile-shape model (same 32-64-64-1 network): predicts the log of a batch launch
    // sequence's milliseconds for a job-size signature and a tile shape
    std::vector<float> tile_model;
    bool tile_model_ok = false;
    std::vector<float> tune_log;      // autotuner measurements: HB_FEATURES features + log(ms) per shape
    int tune_learned = 0;             // 1 when the last batch's shape came from the tile model
    // pinned staging
    void *pin[2] = {nullptr, nullptr};
    cudaEvent_t pin_ev[2] = {nullptr, nullptr};
    bool direct_pending = false;   // a DMA from the caller's page-locked memory is in flight
    // streamed S chunks (hb_block_stream): device chunk buffers, copy stream, events
    Buf w_chunk[2];
    cudaStream_t copy_stream = nullptr;
    cudaEvent_t chunk_copied[2] = {nullptr, nullptr}, chunk_consumed[2] = {nullptr, nullptr};
    size_t pin_bytes = 0;
    // batched jobs: row offsets of the stacked jobs (hb_block_batch)
    std::vector<int64_t> job_rows;
    // captured batch pipeline and the shapes it was captured for
    cudaGraph_t batch_graph = nullptr;
    cudaGraphExec_t batch_exec = nullptr;
    std::vector<int64_t> batch_graph_key;
    Buf w_jobrows, w_jobcount, w_joboff;
    Buf w_small;   // member starts of packed small blocks
    Buf w_check;   // per column: first row whose string offsets decrease (hb_load_table)
    // block building of several MDs at once: per-lane scratch, side streams, events
    struct MdLane {
        Buf table, slot_r, count_r, start_r, cursor, slot_s, count_s, start_s, scan, meta;
        Buf jac;   // q-gram encoder scratch when the lane encodes a Jaccard column
        Buf minrow;   // sharded evaluation: each group's smallest row
        cudaStream_t stream = nullptr;
        cudaEvent_t done = nullptr;
    };
    std::vector<MdLane> md_lanes;
    cudaEvent_t md_fork = nullptr;
    // autotuner cache: job-size signature -> (tile, claim)
    std::vector<std::pair<std::vector<int64_t>, std::pair<int, int>>> tune_cache;
    int claim = 16;
    // planner statistics kept for the learned model: per predicate [len mean, len std, p10, p50, p90, max,
    // gram mean, gram std, null fraction, LSH bucket stddev], summarised on demand (ensure_pred_stats)
    // from the sampled lengths / gram counts ([predicate][stat_keep]) and bucket deviations
    std::vector<std::vector<float>> pred_stats;
    std::vector<uint32_t> stat_lens, stat_grams;
    std::vector<double> stat_sd;
    int stat_keep = 0;
    std::vector<double> plain_sp, plain_cost;
    long long graph_kernels = 0;   // kernels in the captured batch graph
    // results
    hb_pair *dev_result = nullptr;
    size_t dev_result_bytes = 0;
};


namespace hb {

struct RunResult {
    int64_t n_out = 0;
    int64_t cand = 0;
    int64_t tiles = 0;
    int64_t blocks = 0;     // block descriptors (a packed one holds several small blocks)
    int64_t examined = 0;
    int64_t real_blocks = 0;   // blocks, small ones counted one by one
};

struct Timer {
    cudaEvent_t e[8];
    int n = 0;
    cudaStream_t s;
    explicit Timer(cudaStream_t st) : s(st) {
        for (auto &x : e) cudaEventCreate(&x);
    }
    ~Timer() {
        for (auto &x : e) cudaEventDestroy(x);
    }
    void mark() {
        if (n < 8) cudaEventRecord(e[n++], s);
    }
    float ms(int a, int b) {
        float v = 0;
        if (a < n && b < n) cudaEventElapsedTime(&v, e[a], e[b]);
        return v;
    }
};

hb_status grow(hb_ctx *c, Buf &b, size_t bytes);
void free_buf(hb_ctx *c, Buf &b);
hb_status dmalloc(hb_ctx *c, void **p, size_t bytes);
hb_status upload(hb_ctx *c, void *dst, const void *src, size_t bytes);
// two pinned staging buffers of at least `bytes` each (c->pin)
hb_status ensure_pinned(hb_ctx *c, size_t bytes);
// true when p is page-locked host memory (cudaMallocHost / cudaHostRegister)
bool page_locked(const void *p);
// wait for the DMAs upload() issued from page-locked caller memory
hb_status sync_direct(hb_ctx *c);
hb_status do_plan(hb_ctx *c, int mode, bool job_key);
// summarise the sampled predicate statistics for the learned cost model's features
void ensure_pred_stats(hb_ctx *c);
hb_status encode_side(hb_ctx *c, int side);
hb_status ensure_ready(hb_ctx *c, bool job_key);
bool is_self(hb_ctx *c);
hb_status block_eval_sort(hb_ctx *c, const uint32_t *rec_r, int64_t n_r, const uint32_t *rec_s, int64_t n_s,
                          bool self, int side_s, int key_bits, int key_bits_s, int logging, RunResult &res,
                          uint64_t **sorted, Timer *tm);
hb_status deliver(hb_ctx *c, const uint64_t *keys, int64_t n, int key_bits_s, bool to_host, hb_pair **out);
hb_status learned_stats(hb_ctx *c, std::vector<double> &sp, std::vector<double> &cost, bool &ok);
// counters (u64 words): 0 tile claims, 1 output count, 2 candidates, 3 block count (u32), 4 block overflow,
// 5 examined pairs
hb_status build_blocks(hb_ctx *c, const uint32_t *rec_r, int64_t n_r, const uint32_t *rec_s, int64_t n_s, bool self,
                       unsigned long long *ctr, uint32_t &block_cap);
EvalParams make_params(hb_ctx *c, const uint32_t *rec_r, const uint32_t *rec_s, int side_s, bool self,
                       unsigned long long *ctr, int key_bits_s);

template <typename T>
static inline T *as(Buf &b) {
    return static_cast<T *>(b.p);
}

}  // namespace hb
