/*
 * libhb — rule-based blocking for entity resolution on one GB300 GPU.
 *
 * The library computes, for a set Delta of matching dependencies (MDs), the
 * candidate pairs Ca of Section 2 ("Blocking"): a tuple pair is a candidate
 * iff some MD phi = X -> t.eid = s.eid in Delta is a witness at it, i.e. the
 * pair satisfies every predicate of the precondition X ("Semantics").
 *
 *   self-join : Ca = { (i, j) : 0 <= i < j < n,  some phi satisfied by (t_i, t_j) }
 *   R x S     : Ca = { (i, j) : i in R, j in S,  some phi satisfied by (r_i, s_j) }
 *
 * Predicates (Section 2, "Predicates": t.A = c, t.A = s.B and t.A ~ s.B with
 * a symmetric or asymmetric similarity measure and a threshold):
 *   HB_P_EQ          t.A = s.B          strings by bytes, int32 by value; A and B may be
 *                                       two columns of one relation in a self-join
 *   HB_P_EQ_PREFIX   first k bytes equal (strings; a shorter string is its own prefix)
 *   HB_P_ED_LE       Levenshtein distance over bytes <= k          (edit distance, Example 2)
 *   HB_P_JACCARD_GE  q-gram set Jaccard >= num/den, compared as    (Jaccard measure, Example 2)
 *                    |A n B| * den >= num * |A u B| (q = 1..4, contiguous q-byte
 *                    substrings, no padding; a string shorter than q has no grams)
 *   HB_P_ABSDIFF_LE  fabsf(a - b) <= delta in binary32 (fp32 columns)
 *   HB_P_CONST_EQ    t.A = c or s.A = c (string or int32 column; the constant is copied)
 *   HB_P_CONTAIN_GE  |G(t.A) n G(s.B)| * den >= num * |G(side's value)|, q-grams as for
 *                    Jaccard: how much of one side's gram set the other contains (asymmetric)
 *   HB_P_TOKEN_JACCARD_GE  Jaccard of the sets of word tokens (maximal runs of bytes other
 *                    than the space 0x20) >= num/den, compared in integers as above
 * A missing operand (valid[i] == 0) makes every predicate false (Example 3:
 * (t2, t3) is not a witness because t2.price is missing).
 *
 * A self-join emits each unordered pair once as (i, j) with i < j: the pair is
 * in the result when some MD is a witness at (t_i, t_j) or at (t_j, t_i).
 * With symmetric predicates only the two valuations agree (Section 5.1, last
 * paragraph of "Reusing computation"); an MD with a constant, a containment or
 * two different columns is evaluated at both.  The result is exact: no
 * sampling, no approximation.
 *
 * Errors: every call returns an hb_status; nothing throws across this
 * boundary.  On a non-OK status hb_last_error() describes it.  Calls on one
 * context must not run concurrently.  Inputs are copied: the caller may free
 * its buffers as soon as a call returns.
 */
#ifndef HB_H
#define HB_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#if defined(__GNUC__)
#define HB_API __attribute__((visibility("default")))
#else
#define HB_API
#endif

typedef struct hb_ctx hb_ctx;

typedef enum {
    HB_OK = 0,
    HB_ERR_ARG = -1,            /* invalid argument (message names it) */
    HB_ERR_OOM = -2,            /* host or device allocation failed */
    HB_ERR_CUDA = -3,           /* a CUDA call failed (message has the CUDA error) */
    HB_ERR_STATE = -4,          /* call out of order (e.g. hb_block before hb_load_table) */
    HB_ERR_OVERFLOW = -5,       /* a fixed-capacity output could not hold the result */
    HB_ERR_DEVICE_TIMEOUT = -6, /* a bounded device-side wait gave up */
    HB_ERR_INTERNAL = -7,
    HB_ERR_BOUNDS = -8          /* checked build (libhb_checked.so) only: an index left its buffer (message names the site) */
} hb_status;

typedef enum { HB_COL_STRING = 0, HB_COL_INT32 = 1, HB_COL_FP32 = 2 } hb_coltype;

/* One column of a relation (Section 2, "Relations": schema R = (eid, A1..An)). */
typedef struct {
    int32_t type;             /* hb_coltype */
    int32_t reserved;         /* 0 */
    const void *data;         /* STRING: bytes; INT32: int32_t[n]; FP32: float[n] */
    const uint32_t *offsets;  /* STRING: n+1 nondecreasing byte offsets, offsets[0] = 0; else NULL */
    const uint8_t *valid;     /* n bytes, nonzero = present; NULL = every row present */
    uint64_t data_bytes;      /* STRING: offsets[n]; ignored otherwise */
} hb_column;

typedef enum {
    HB_P_EQ = 0,
    HB_P_EQ_PREFIX = 1,
    HB_P_ED_LE = 2,
    HB_P_JACCARD_GE = 3,
    HB_P_ABSDIFF_LE = 4,
    HB_P_CONST_EQ = 5,          /* t.A = c (side 0) or s.A = c (side 1) */
    HB_P_CONTAIN_GE = 6,        /* q-gram containment, asymmetric */
    HB_P_TOKEN_JACCARD_GE = 7   /* Jaccard of word-token sets */
} hb_pkind;

/* One predicate of an MD precondition (Section 2, "Predicates"). */
typedef struct {
    int32_t kind;             /* hb_pkind */
    int32_t col_t;            /* column of the left tuple (relation R) */
    int32_t col_s;            /* column of the right tuple (S; = col_t for a self-join) */
    int32_t k;                /* ED_LE: max distance, 0..31 (larger: HB_ERR_ARG);
                                 EQ_PREFIX: prefix length (>= 1) */
    int32_t q;                /* JACCARD_GE: gram length, 1..4; a compared string may hold at most
                                 8192 grams (a longer one makes hb_plan / hb_block return HB_ERR_ARG) */
    uint32_t num, den;        /* JACCARD_GE, CONTAIN_GE, TOKEN_JACCARD_GE: threshold num/den,
                                 0 <= num <= den, den >= 1 */
    float delta;              /* ABSDIFF_LE: threshold (>= 0) */
    int32_t side;             /* CONST_EQ: 0 = the pair's first tuple (t.A = c, column col_t),
                                 1 = its second (s.A = c, column col_s);
                                 CONTAIN_GE: whose gram set divides, 0 = t's (col_t), 1 = s's (col_s) */
    uint32_t value_len;       /* CONST_EQ: bytes of value (string column) or 4 (int32 column) */
    const void *value;        /* CONST_EQ: the constant (host memory, copied by hb_add_md) */
} hb_predicate;

typedef struct { uint32_t tid1, tid2; } hb_pair;

/* hb_options.flags */
#define HB_FLAG_PER_JOB_LAUNCHES 1   /* hb_block_batch: one launch sequence per job (comparison baseline) */
#define HB_FLAG_NO_GRAPH 2           /* hb_block_batch: never capture or replay a CUDA graph */

typedef struct {
    int32_t device;           /* CUDA device ordinal */
    int32_t tile;             /* tuples per tile side: 0 = autotuned, else 32 or 64 */
    uint64_t chunk_bytes;     /* pinned staging chunk for host uploads; 0 = 256 MiB */
    uint64_t seed;            /* seed of the planner's samples */
    void *stream;             /* cudaStream_t to run on; NULL = a stream owned by the context */
    int64_t out_capacity;     /* initial capacity (pairs) of the result slab; 0 = automatic */
    int32_t flags;            /* reserved, 0 */
    int32_t reserved;
} hb_options;

/* Planner modes.  Every mode yields the same pair set; they differ in speed. */
typedef enum {
    HB_PLAN_RULE_DATA = 0,    /* Section 4.2: order by (1 - sp) / cost, tree, wp, edge scores, DFS */
    HB_PLAN_LEARNED = 1,      /* same, with sp and cost predicted by the trained cost model;
                                 falls back to HB_PLAN_RULE_DATA when no usable model is loaded */
    HB_PLAN_GIVEN_ORDER = 2,  /* MDs and predicates exactly as added */
    HB_PLAN_RANDOM = 3,       /* a seeded random order */
    HB_PLAN_COST_FIRST = 4,   /* cheapest predicate first (cost only) */
    HB_PLAN_SEL_FIRST = 5     /* most selective predicate first (sp only) */
} hb_plan_mode;

#define HB_MAX_MDS 64
#define HB_MAX_PREDS 128

typedef struct {
    int32_t mode;                     /* the mode that was applied */
    int32_t n_preds;                  /* distinct predicates over all MDs */
    int32_t n_ops;                    /* non-equality predicates in the evaluation program */
    int32_t n_eq;                     /* distinct equality keys (blocking keys) */
    int32_t op_pred[HB_MAX_PREDS];    /* program order: distinct predicate ids */
    int32_t md_order[HB_MAX_MDS];     /* DFS order of the MDs */
    double sp[HB_MAX_PREDS];          /* sp(p, D) used for ordering */
    double cost[HB_MAX_PREDS];        /* cost(p, D) used for ordering */
    int32_t pred_md[HB_MAX_PREDS];    /* first MD that holds each distinct predicate */
    int32_t tile;                     /* tile side chosen for evaluation */
    int32_t n_mds;
    int32_t record_words;             /* 32-bit words of a tuple's packed record (codes and features) */
    int32_t hot_words;                /* 32-bit words of a tuple's hot record (what every pair's first test reads) */
    int32_t n_branches;               /* partitioned blocking (hb_set_partitions): root branches, else 0 */
    int32_t branch_pred[HB_MAX_MDS];  /* per branch: its root-edge predicate id (-1: one partition of all tuples) */
} hb_plan_info;

typedef struct {
    int64_t n_rows_r, n_rows_s;
    int64_t candidate_pairs;   /* pairs that agree on every equality predicate of some MD, each once */
    int64_t emitted_pairs;     /* |Ca| of the last call */
    int64_t tiles;             /* evaluation work items of the last call */
    int64_t blocks;            /* non-trivial blocks over all MDs */
    double ms_h2d, ms_encode, ms_plan, ms_block_build, ms_eval, ms_sort, ms_d2h, ms_total;
    int64_t device_bytes;      /* device memory held by the context */
    int32_t tile;              /* tile side used */
    int32_t n_mds;
    int64_t kernel_launches;   /* CUDA kernels launched by the library so far (process-wide) */
    int64_t examined_pairs;    /* pairs inside blocks looked at by the evaluation kernel (last call) */
} hb_stats;

/* ---- context ---- */
/*
 * opt may be NULL (defaults).  Fault injection for tests of the error paths:
 * when the environment holds HB_FAIL_ALLOC_AFTER=N (a decimal N >= 0) at
 * hb_create, the context's (N+1)-th device or page-locked allocation fails
 * once with HB_ERR_OOM; the call that met it returns HB_ERR_OOM and leaves the
 * context usable (a repeated call allocates again).
 */
HB_API hb_status hb_create(hb_ctx **out, const hb_options *opt);
HB_API void hb_destroy(hb_ctx *ctx);
HB_API const char *hb_last_error(void);                            /* thread-local; "" when none */
HB_API const char *hb_version(void);

/*
 * Load relation `side` (0 = R, 1 = S; a self-join loads only R) of n_rows rows
 * and n_cols columns.  on_device = 0: pointers are host memory; a page-locked
 * array (cudaMallocHost / cudaHostRegister) is copied by one DMA, a pageable
 * one through pinned staging chunks of chunk_bytes; on_device = 1: pointers
 * are device memory of this context's device, copied device to device.  The
 * call returns once every host array has been read.  Replaces any previous
 * table of that side.  HB_ERR_ARG when string offsets do not start at 0, end
 * at data_bytes or never decrease (host arrays; the last is checked on the
 * device after the copy, and the side is then left empty).
 */
HB_API hb_status hb_load_table(hb_ctx *ctx, int32_t side, int64_t n_rows, int32_t n_cols, const hb_column *cols,
                        int32_t on_device);

/*
 * Add one MD (Section 2, "Rules": phi = X -> t.eid = s.eid, X a conjunction
 * of predicates; the default parameters of Section 6 cap an MD at ten) with
 * 1..10 predicates; *md_id_out (optional) receives its id (0, 1, ...).
 * Checks each predicate's parameters (HB_ERR_ARG: unknown kind, negative
 * column, ED threshold outside 0..31, Jaccard q outside 1..4 or num > den,
 * prefix length < 1, delta < 0 or NaN); columns are checked against the
 * tables by hb_plan.
 */
HB_API hb_status hb_add_md(hb_ctx *ctx, int32_t n_pred, const hb_predicate *preds, int32_t *md_id_out);
HB_API hb_status hb_clear_mds(hb_ctx *ctx);

/*
 * Build the execution plan (Section 4.2) for the loaded tables and MDs:
 * samples the data on the GPU for sp and cost, orders predicates, builds the
 * execution tree and flattens it into the sequential program of Section 5.1.
 * Must follow the last hb_add_md / hb_load_table.  info_out is optional.
 */
HB_API hb_status hb_plan(hb_ctx *ctx, int32_t mode, hb_plan_info *info_out);

/*
 * Section 5.3 "Data partitioning": block by root-edge hash partitions instead
 * of exact equality groups.  Each child of the execution tree's root gives one
 * hash function, built from the predicate on that edge; here an MD's root edge
 * is its first equality predicate in written order (equality predicates are
 * the block keys and head every path), and MDs without one share a branch
 * whose single partition holds all tuples (the section's remark: a partition
 * may pull all others).  A tuple's partition under a function is the 32-bit
 * FNV-1a hash (offset basis 2166136261, prime 16777619) of the value's bytes
 * (a string or its prefix, an int32's four little-endian bytes) modulo m; a
 * missing value is in no partition.  A pair is a candidate when some branch
 * puts both tuples in one partition; it is evaluated once, in the first such
 * branch, against every MD, so the result equals the unpartitioned one while
 * the candidate count (hb_get_stats) grows as m shrinks.
 *
 * m = 0 restores exact equality groups (the default); m >= 1 applies from the
 * next hb_plan (a later hb_block plans again if needed).  Partitioned blocking
 * runs on hb_block and hb_block_device with at most 8 distinct equality keys;
 * hb_block_stream and hb_block_batch then return HB_ERR_STATE.  m > 2^31 is
 * HB_ERR_ARG.
 */
HB_API hb_status hb_set_partitions(hb_ctx *ctx, uint32_t m);

/*
 * Sharded evaluation over `world` processes, each with a GPU of its own (a
 * build addition: the paper spreads partitions over GPUs, Section 5.3
 * "Multi-GPU scheduling"; here the unit of work is a block).  Every process
 * loads the same tables and rules and encodes and groups them alike; a block
 * (one MD's group of tuples that agree on its equality keys, with all the
 * pairs the owner rule gives that MD) is evaluated by rank
 *     (fmix32(r ^ (md * 0x9E3779B9)) mod world),
 * r = the smallest row id of the group (of R in R x S) and fmix32 the 32-bit
 * finaliser of MurmurHash3 (h ^= h >> 16; h *= 0x85EBCA6B; h ^= h >> 13;
 * h *= 0xC2B2AE35; h ^= h >> 16), a function of the data alone.  hb_block and
 * hb_block_device then return this rank's pairs, sorted; the ranks' outputs are
 * disjoint and their union is the unsharded result (merge them with
 * hb_merge_pairs).  Candidate counts in hb_get_stats are this rank's.
 * 0 <= rank < world, else HB_ERR_ARG; world = 1 (the default) evaluates every
 * block.  hb_block_stream and hb_block_batch return HB_ERR_STATE while
 * world > 1.  Applies from the next hb_block.
 */
HB_API hb_status hb_set_shard(hb_ctx *ctx, int32_t rank, int32_t world);

/*
 * Host-side k-way merge (a build addition: the final gather step of a sharded
 * evaluation): lists[l] holds counts[l] pairs sorted ascending by (tid1, tid2);
 * out (caller-allocated, sum of counts entries) receives all of them sorted
 * the same way (pairs equal across lists are all kept, list order among
 * them).  Reads and writes host memory only; no GPU is needed.  HB_ERR_ARG on
 * k < 0, a negative count, or a NULL array where a count is positive.
 */
HB_API hb_status hb_merge_pairs(const hb_pair *const *lists, const int64_t *counts, int32_t k, hb_pair *out);

/*
 * Compute Ca for the loaded tables (self-join when only R is loaded).
 * *pairs_out receives a library-allocated host array of *n_out pairs sorted
 * ascending by (tid1, tid2), unique; free it with hb_free_pairs.  Plans with
 * HB_PLAN_RULE_DATA first if hb_plan was not called.
 */
HB_API hb_status hb_block(hb_ctx *ctx, hb_pair **pairs_out, int64_t *n_out);

/*
 * As hb_block, but the sorted pairs stay in device memory owned by the
 * context (valid until the next call on it); *dev_pairs_out is a device pointer.
 */
HB_API hb_status hb_block_device(hb_ctx *ctx, hb_pair **dev_pairs_out, int64_t *n_out);

/*
 * Section 5.3 ("Data transfer between host and devices"): partitions are read
 * into device memory while in-device ones are evaluated (CUDA streams overlap
 * transfer and compute).  This call is that pipeline for R x S, with S
 * streamed from host memory: R must be loaded (side 0); S's
 * columns (host pointers, same column order as used by the MDs' col_s) are
 * copied in chunks of at most chunk_bytes (straight from the caller's arrays
 * when all of them are page-locked, else through two pinned staging buffers),
 * and every chunk is encoded, blocked and evaluated while the next one is in
 * flight.  The call returns after the last chunk.  Output as hb_block (tid2
 * indexes S as given).
 */
HB_API hb_status hb_block_stream(hb_ctx *ctx, int64_t n_rows_s, int32_t n_cols, const hb_column *cols_s,
                          hb_pair **pairs_out, int64_t *n_out);

/*
 * Build addition: the paper blocks the partitions P1..Pm of its problem
 * statement (Section 2) one after another; this blocks many independent
 * relations in one launch sequence.  The loaded R holds n_jobs independent
 * relations stacked by rows; job j is rows [job_rows[j], job_rows[j+1]).  Every job is blocked
 * with the context's MDs in one persistent work-queue launch sequence (replayed
 * from a CUDA graph when the shapes repeat).  Pairs use job-local row ids;
 * job j's pairs are (*pairs_out)[job_pairs_out[j] .. job_pairs_out[j+1]),
 * each range sorted.  job_pairs_out has n_jobs + 1 entries (caller-owned).
 */
HB_API hb_status hb_block_batch(hb_ctx *ctx, int32_t n_jobs, const int64_t *job_rows, hb_pair **pairs_out,
                         int64_t *job_pairs_out);

HB_API void hb_free_pairs(hb_pair *pairs);
HB_API hb_status hb_get_stats(const hb_ctx *ctx, hb_stats *out);

/*
 * Order predicates and MDs from given sp / cost values only (no data, no GPU):
 * the pure host part of hb_plan.  mds are given as predicate ids:
 * md_pred[md_start[m] .. md_start[m+1]).  Writes the flattened program
 * (program_out, n_prog_out, skipping ids with skip[p] != 0), the per-MD
 * checkpoint index (cp_out[m], -1 when none) and the DFS MD order.
 */
HB_API hb_status hb_plan_order(int32_t n_preds, const double *sp, const double *cost, int32_t n_mds,
                        const int32_t *md_start, const int32_t *md_pred, const uint8_t *skip,
                        int32_t *program_out, int32_t *n_prog_out, int32_t *cp_out, int32_t *md_order_out);

/* ---------------- learned cost model (small MLP, 32 -> 64 -> 64 -> 1, ReLU) ----------------
 * Section 4.2 ("Shallow NNs", "Estimated cost") estimates predicate cost with
 * a shallow network trained on historical logs.  Here two such networks
 * predict, per predicate, its log cost per evaluated pair and the logit of its
 * pass rate from HB_FEATURES features of sampled column statistics.
 */
#define HB_FEATURES 32
#define HB_MLP_PARAMS (32 * 64 + 64 + 64 * 64 + 64 + 64 + 1)   /* W1 b1 W2 b2 W3 b3, row-major */

/* One logged predicate evaluation record of the blocker. */
typedef struct {
    float features[HB_FEATURES];
    float log_cost;          /* log of the device cycles per pair when the predicate is evaluated first:
                                16 for its cheap filter (length / size / |a-b| test on staged operands)
                                plus, times the filter pass rate, the measured cycles of a full evaluation */
    float logit_pass;        /* logit(pass rate), clamped to [-12, 12] */
    int64_t evaluated;       /* evaluations counted */
    int64_t passed;
    int64_t cycles;          /* clock64 cycles spent in the evaluations */
    int64_t stage1;          /* evaluations past the length / size filter (ED, Jaccard) */
    int64_t stage2;          /* evaluations past the character-bin / gram-bin filter (ED, Jaccard) */
    int64_t core;            /* ED: band cells computed; Jaccard: merge steps */
    int32_t pred;            /* distinct predicate id in the context */
    int32_t kind;            /* hb_pkind */
} hb_pred_log;

/*
 * Run the current plan once with per-predicate instrumentation (evaluations,
 * passes, filter passes, core work and clock cycles per predicate) and write
 * one record per non-equality predicate, in program order, to out (capacity
 * cap).  profile = 0: the plan as it runs (early exit at the first witness
 * or when every MD has failed); profile = 1: every predicate of every MD
 * whose equality keys match is evaluated (no early exit), which measures each
 * predicate's own pass rate and cost.  *n_out receives the record count.
 */
HB_API hb_status hb_log_predicates(hb_ctx *ctx, int32_t profile, hb_pred_log *out, int32_t cap, int32_t *n_out);

/* Features the cost model sees for each distinct predicate of the current plan. */
HB_API hb_status hb_predicate_features(hb_ctx *ctx, float *features_out, int32_t cap_preds, int32_t *n_out);

/*
 * Train the two networks on the GPU with the library's own forward, backward
 * and Adam kernels (FP32, mean squared error): rows are n records of
 * HB_FEATURES floats (host), targets y_cost[n], y_sel[n] (host).  The trained
 * weights become the context's model (used by HB_PLAN_LEARNED).  Returns the
 * final training losses in loss_out[2] (optional).
 */
HB_API hb_status hb_train_cost_model(hb_ctx *ctx, int32_t n, const float *X, const float *y_cost, const float *y_sel,
                              int32_t epochs, float lr, uint64_t seed, float *loss_out);

/* Copy the model weights out (2 x HB_MLP_PARAMS floats) or in. */
HB_API hb_status hb_get_cost_model(hb_ctx *ctx, float *params_out);
HB_API hb_status hb_set_cost_model(hb_ctx *ctx, const float *params);

/*
 * MLP kernels on device buffers (all pointers device memory, row-major):
 * X [n, 32] fp32, params [HB_MLP_PARAMS] fp32, y [n] fp32.
 * hb_mlp_forward_bf16 rounds X, weights and hidden activations to bfloat16
 * and accumulates in fp32.  hb_mlp_backward computes the gradient of
 * mean((y - t)^2) into grad [HB_MLP_PARAMS] (overwritten).  hb_adam_step
 * applies Adam (Kingma & Ba) step number `step` (1-based) in place.
 * `stream` is a cudaStream_t (NULL = default stream).
 */
HB_API hb_status hb_mlp_forward(const float *X, int32_t n, const float *params, float *y, void *stream);
HB_API hb_status hb_mlp_forward_bf16(const float *X, int32_t n, const float *params, float *y, void *stream);
HB_API hb_status hb_mlp_backward(const float *X, const float *t, int32_t n, const float *params, float *grad,
                          void *stream);
/*
 * hb_mlp_backward without any device allocation (the paper has no
 * counterpart; this serves callers that cannot allocate device memory when
 * they need a gradient, e.g. a process whose device memory is pre-partitioned
 * by its own pool or a loop that must not call cudaMalloc / cudaFree).  Same
 * arguments and result as hb_mlp_backward, for n <= 4096 rows (larger n:
 * HB_ERR_ARG).  Its work buffers live in one fixed device array of the library
 * (about 4.2 MB, held on every GPU that loads the library until exit).  The
 * first call on a device looks up that array's address (call it once before
 * any stream capture); every call shares the array, so calls that overlap on
 * the GPU race.  No state carries over between calls.  The array's address
 * is kept per device with the CUDA context it was found in; do not call this
 * across a device reset (cudaDeviceReset) whose new context could reuse the
 * old handle.
 */
HB_API hb_status hb_mlp_backward_noalloc(const float *X, const float *t, int32_t n, const float *params,
                                         float *grad, void *stream);
HB_API hb_status hb_adam_step(float *params, const float *grad, float *m, float *v, int32_t n_params, int32_t step,
                       float lr, float beta1, float beta2, float eps, void *stream);

/*
 * Tile shape chosen by a learned model (batched form).  hb_block_batch's
 * autotuner times every candidate shape (tuples per tile side 32 or 64 x 1, 2,
 * 4 or 8 tiles per claim) the first time it meets a job-size signature and
 * logs each measurement (HB_FEATURES features of the signature and the shape,
 * log of the milliseconds).  hb_tile_log copies the logged rows out (up to cap;
 * *n_out receives the total); hb_train_tile_model trains a 32-64-64-1 network
 * on such rows (as hb_train_cost_model) and makes it the context's tile model;
 * hb_set_tile_model installs one (NULL removes it), hb_get_tile_model copies it
 * out (HB_MLP_PARAMS floats).  With a tile model, a new signature takes the
 * shape of smallest predicted time without trial runs; without one, or when a
 * prediction is not finite, the autotuner measures.  hb_batch_tile reports the
 * shape of the last batch and whether the model chose it (learned = 1).
 */
HB_API hb_status hb_tile_log(hb_ctx *ctx, int32_t cap, float *X_out, float *y_out, int32_t *n_out);
HB_API hb_status hb_train_tile_model(hb_ctx *ctx, int32_t n, const float *X, const float *y, int32_t epochs, float lr,
                                     uint64_t seed, float *loss_out);
HB_API hb_status hb_set_tile_model(hb_ctx *ctx, const float *params);
HB_API hb_status hb_get_tile_model(hb_ctx *ctx, float *params_out);
HB_API hb_status hb_batch_tile(const hb_ctx *ctx, int32_t *tile, int32_t *claim, int32_t *learned);

/* ---------------- the paper's per-pair cost model N ----------------
 * Section 4.2 ("Shallow NNs") trains a small network N(p, t1, t2) on logged
 * times of checking p on tuple pairs; cost(p, D) is then estimated as
 * norm(sum of N over sampled pairs).  Section 6's defaults give hidden layers
 * of 2, 6 and 1 neurons; here N maps HB_PAIR_FEATURES features to one output
 * through layers of 2 and 6 ReLU units (the last neuron is the output).
 * Features of (p, t1, t2): kind one-hot (edit distance, Jaccard, |a-b|),
 * threshold (k/8, num/den or log1p(delta)), s(o1), s(o2), s(|o1 - o2|) and
 * min/max of |o1|, |o2|, where o is the tuple's operand (string length,
 * distinct q-gram count, or value), s(v) = v/64 for lengths and counts and
 * log1p(|v|)/8 for values; a missing operand sets the last four to -1.
 */
#define HB_PAIR_FEATURES 8
#define HB_PAIR_MODEL_PARAMS (8 * 2 + 2 + 2 * 6 + 6 + 6 + 1)   /* W1 b1 W2 b2 W3 b3, row-major */

/*
 * Check distinct predicate `pred` (an edit-distance, Jaccard or |a-b|
 * predicate of the current plan's program) on n given pairs (host arrays i[],
 * j[]: rows of R and of S, or of R twice in a self-join), one thread per pair,
 * and write per pair the clock64 cycles of the check (cycles_out), its
 * verdict (verdict_out, 0/1) and N's features (features_out, n x
 * HB_PAIR_FEATURES floats).  All outputs are host arrays.  HB_ERR_ARG for an
 * unknown or unsupported predicate or a row out of range.
 */
HB_API hb_status hb_time_pairs(hb_ctx *ctx, int32_t pred, int32_t n, const uint32_t *i, const uint32_t *j,
                               uint32_t *cycles_out, uint8_t *verdict_out, float *features_out);
/* N's forward pass and the gradient of mean((y - t)^2) (device pointers; grad overwritten). */
HB_API hb_status hb_pair_model_forward(const float *X, int32_t n, const float *params, float *y, void *stream);
HB_API hb_status hb_pair_model_backward(const float *X, const float *t, int32_t n, const float *params, float *grad,
                                        void *stream);
/*
 * Train N on the GPU (full-batch Adam, lr, `epochs` steps, He-uniform start
 * from `seed`) on n rows (host arrays X [n x HB_PAIR_FEATURES], y [n]); writes
 * the trained parameters (params_out, HB_PAIR_MODEL_PARAMS floats, host) and
 * the final mean squared error (loss_out, optional).
 */
HB_API hb_status hb_train_pair_model(int32_t n, const float *X, const float *y, int32_t epochs, float lr,
                                     uint64_t seed, float *params_out, float *loss_out);

/*
 * Measurement aid (no counterpart in the paper): the integer issue rate of the
 * current device.  Launches 8 resident 256-thread blocks per SM whose threads
 * run 8 independent chains of three integer instructions (three-input add,
 * shift, three-input logic) for `iters` steps, timed with CUDA events on
 * `stream` (NULL = default stream) after one short warm-up launch.  Writes
 * integer operations per second to *ops_per_s and the timed launch's
 * milliseconds to *ms_out (optional).  Allocates and frees a small result
 * array on `stream`.  HB_ERR_ARG when iters < 1 or ops_per_s is NULL.
 */
HB_API hb_status hb_probe_int_issue(int32_t iters, double *ops_per_s, double *ms_out, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* HB_H */
