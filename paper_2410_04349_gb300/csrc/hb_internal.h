// Internal declarations shared by the libhb translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <string>
#include <vector>

#include "hb.h"

namespace hb {

// kernel launches made by the library (all contexts, cumulative)
extern std::atomic<long long> g_kernel_launches;
#define HB_LAUNCHED(n) (::hb::g_kernel_launches.fetch_add((n), std::memory_order_relaxed))

// ---- checked builds (HB_CHECKED: libhb_checked.so) ----
// The evaluation kernel's block, member, tuple, survivor, ring, string and
// gram-list indices and the encoder's and block builder's output positions
// are checked against their buffers.  A failing check records its site number
// in the translation unit's error word and the access goes to element 0 (or an
// empty range) instead, so nothing outside a buffer is touched; the host turns
// a recorded site into HB_ERR_BOUNDS.  Ordinary builds compile the checks away.
#if defined(HB_CHECKED) && defined(__CUDACC__)
static __device__ unsigned int hb_dev_err;
__device__ __forceinline__ uint64_t hb_checked_index(uint64_t i, uint64_t n, unsigned site) {
    if (i < n) return i;
    atomicCAS(&hb_dev_err, 0u, site);
    return 0;
}
__device__ __forceinline__ bool hb_checked_range(uint64_t lo, uint64_t len, uint64_t n, unsigned site) {
    if (lo <= n && len <= n - lo) return true;
    atomicCAS(&hb_dev_err, 0u, site);
    return false;
}
#define HB_IDX(i, n, site) ::hb::hb_checked_index((uint64_t)(i), (uint64_t)(n), (site))
#define HB_RANGE_OK(lo, len, n, site) ::hb::hb_checked_range((uint64_t)(lo), (uint64_t)(len), (uint64_t)(n), (site))
// reads and clears the unit's error word (the caller has synchronised the device)
#define HB_ERROR_READER(name)                                              \
    unsigned int name() {                                                  \
        unsigned int v = 0, z = 0;                                         \
        cudaMemcpyFromSymbol(&v, hb_dev_err, sizeof(v));                   \
        if (v) cudaMemcpyToSymbol(hb_dev_err, &z, sizeof(z));              \
        return v;                                                          \
    }
#else
#define HB_IDX(i, n, site) (i)
#define HB_RANGE_OK(lo, len, n, site) true
#define HB_ERROR_READER(name) \
    unsigned int name() { return 0; }
#endif
unsigned int checked_error_eval();     // k_eval.cu
unsigned int checked_error_encode();   // k_encode.cu
unsigned int checked_error_block();    // k_block.cu
hb_status check_bounds(hb_ctx *c, const char *what);   // hb_api.cu: HB_ERR_BOUNDS if a check failed

constexpr uint32_t NULL_CODE = 0xFFFFFFFFu;     // missing value: equal to nothing
constexpr uint32_t NOMATCH_CODE = 0xFFFFFFFEu;  // S value that no R tuple holds
constexpr uint32_t NULL_LEN = 0xFFFFFFFFu;      // missing string
constexpr uint64_t EMPTY_SLOT = 0xFFFFFFFFFFFFFFFFull;
constexpr int MAX_EQ = 16;     // distinct equality keys per context
constexpr int MAX_OPS = 48;    // non-equality predicates in one program
constexpr int MAX_MD = 64;
constexpr int LUT_MAX_EQ = 10; // equality-match -> MD-mask lookup table up to 2^10 entries
constexpr int SMALL_MAX = 16;  // self-join blocks of 2..SMALL_MAX tuples are packed several to a tile
constexpr int SMALL_META_WORDS = 160;
constexpr int MD_LANES = 4;    // MDs whose blocks are built at once (side streams)
// hot-record words beyond which only the mandatory words (keys, first-predicate
// filter operands) are staged: 16 keeps four 256-thread evaluation CTAs of
// 32-tuple tiles resident per SM
constexpr int HOT_BUDGET = 16;

// The member lists of all active MDs lie side by side and are addressed with
// 32 bits: the block build needs (active MDs) x (rows) < 2^32.
inline bool member_addressing_fits(int64_t n_active, int64_t rows) {
    const uint64_t a = (uint64_t)(n_active > 1 ? n_active : 1), r = (uint64_t)(rows > 1 ? rows : 1);
    return a * r < (1ull << 32);
}

// ---- device-side column of one relation ----
struct DevCol {
    int32_t type = 0;
    int64_t n = 0;
    uint8_t *bytes = nullptr;   // STRING
    uint64_t nbytes = 0;
    uint32_t *off = nullptr;    // STRING: n+1
    void *vals = nullptr;       // INT32 / FP32
    uint8_t *valid = nullptr;   // NULL = all present
};

// ---- evaluation program (Section 5.1: sequential execution path) ----
enum OpKind : uint8_t {
    OP_ED = 0,     // edit distance <= k
    OP_JAC = 1,    // Jaccard of q-gram or word-token code sets >= num/den
    OP_ABS = 2,    // |a - b| <= delta
    OP_EQX = 3,    // equality of two columns' codes (one dictionary): a[feat] == b[k]
    OP_CONST = 4,  // t.A = c (num 0: a[feat]) or s.A = c (num 1: b[feat]): the tuple's flag word
    OP_CONT = 5    // containment: |A n B| * den >= num * |side k's set| over a q-gram group
};

struct Op {
    uint8_t kind;
    uint8_t feat;       // first record word of this predicate's feature group
    uint8_t k;          // ED threshold
    uint8_t hot;        // hot-record word holding this predicate's filter operand (255: not staged)
    uint32_t num, den;  // Jaccard threshold
    float delta;        // |a-b| threshold
    uint8_t hot2;       // first hot-record word of its character / gram bins (255: not staged)
    uint8_t pad2[3];
    uint64_t need;      // MDs whose precondition holds this predicate
    uint64_t cp;        // MDs whose last remaining predicate is this one
};

// feature group sizes (record words)
constexpr int FEAT_ED_WORDS = 7;   // len, byte offset, 16 x 8-bit character-bin counts (byte & 15),
                                   // signature: 8 x 4-bit character-bin counts (byte & 7, saturating at 15)
constexpr int FEAT_JAC_WORDS = 12; // unique gram count, gram offset, 32 x 8-bit gram-bin counts,
                                   // 64-bit presence mask of the grams' 6-bit hash bins (low word first)
constexpr int FEAT_ED_SIG = 6;     // word of the ED signature in its group
constexpr int FEAT_JAC_MASK = 10;  // first word of the Jaccard presence mask in its group
constexpr int FEAT_ABS_WORDS = 1;  // fp32 value bits (NaN when missing)

struct BlockDesc {
    uint32_t md;
    uint32_t n_r;       // members on the row side (packed: blocks x size)
    uint32_t start_r;   // into members_r (packed: into the small-block start list)
    uint32_t n_s;       // members on the column side (self-join: = n_r)
    uint32_t start_s;   // into members_s (self-join: = start_r)
    uint32_t packed;    // 0: one block; n: a packed tile of self-join blocks of n tuples each
};

struct EvalParams {
    int32_t n_ops;
    int32_t n_eq;
    int32_t W;              // record words (multiple of 4)
    int32_t self_join;
    int32_t n_md;
    int32_t use_lut;
    int32_t tile;           // 32 or 64
    int32_t key_bits_s;     // packed output key = tid1 << key_bits_s | tid2
    uint64_t eqonly;        // MDs without any non-equality predicate
    // Section 5.3 partitions: MDs that only group pairs (one per root-edge hash
    // function, no predicates: never a witness), the MDs that may own a pair
    // (all by default; the grouping MDs when partitioned) and the equality
    // words phase 1 compares (all by default)
    uint64_t group_mds;
    uint64_t owner_mds;
    uint32_t keymask;
    // buffer extents for the checks of checked builds: rows of each side,
    // member-list and packed-start entries, per op the string bytes (edit
    // distance) or gram codes (Jaccard) of each side
    uint64_t n_r, n_s, members_r_len, members_s_len, small_len;
    uint64_t len_r[MAX_OPS], len_s[MAX_OPS];
    uint16_t eqset[MAX_MD]; // equality keys of each MD (bit e = key e)
    int8_t first_op[MAX_MD];// first program op of each MD (-1: none)
    // per MD m: the MDs alive for every pair of m's blocks (equality keys a
    // subset of m's) and the distinct first ops of those MDs; base_nops 255 =
    // no phase-1 filter (an MD without non-equality predicates, or > 4 ops)
    uint64_t base_alive[MAX_MD];
    uint8_t base_nops[MAX_MD];
    uint8_t base_op[MAX_MD][4];
    // per MD: the (at most two) first program ops whose filter operand is in the
    // hot record (255: none); refine = phase 1b screens the survivors with them
    // (when some screen holds more than phase 1's filter) and batches phase 2
    uint8_t screen_op[MAX_MD][2];
    int32_t refine;
    int32_t multi;          // general phase 1 (2..4 distinct base filters or 4 varying keys in some block)
    int32_t HW;             // hot-record words (multiple of 4): keys, filter operands, bins
    const uint32_t *hot_r;
    const uint32_t *hot_s;
    Op ops[MAX_OPS];
    const void *ptr_r[MAX_OPS];   // ED: string bytes of R; JAC: gram array of R
    const void *ptr_s[MAX_OPS];
    const uint32_t *rec_r;
    const uint32_t *rec_s;
    const uint64_t *lut;          // 2^n_eq MD masks (use_lut)
    const uint32_t *members_r;
    const uint32_t *members_s;
    const uint32_t *small;        // member starts of packed small blocks
    const BlockDesc *blocks;
    const uint32_t *n_blocks;     // device count
    const uint64_t *tile_prefix;  // n_blocks + 1 entries
    unsigned long long *tile_counter;
    uint64_t *out;
    unsigned long long *out_count;
    uint64_t out_cap;
    unsigned long long *cand_count;
    unsigned long long *exam_count;
    uint32_t row_base, col_base;  // added to member ids when packing (chunked S)
    int32_t claim;                // tiles per atomic claim
    int32_t profile;              // logging variant: evaluate every needed predicate, no early exit
    // instrumentation (logging variant only)
    unsigned long long *log;      // per op: [evaluated, passed, cycles] (3 * MAX_OPS)
};

// ---- kernels / launchers (defined in the .cu files) ----
// k_sort.cu
size_t scan_tmp_bytes(int64_t n);
void scan_exclusive_u32(const uint32_t *in, uint32_t *out, int64_t n, const uint32_t *n_dev, void *tmp,
                        size_t tmp_bytes, cudaStream_t s);
void scan_exclusive_u64(const uint64_t *in, uint64_t *out, int64_t n, const uint32_t *n_dev, void *tmp,
                        size_t tmp_bytes, cudaStream_t s);
size_t radix_tmp_bytes(int64_t n);
// sorts keys[0..n) on bits [0, bits); n is read from n_dev when given (bounded by n_max)
void radix_sort_u64(uint64_t *keys, uint64_t *alt, int64_t n_max, const unsigned long long *n_dev, int bits,
                    void *tmp, size_t tmp_bytes, cudaStream_t s, uint64_t **result);

// k_encode.cu
// exact codes (the slot of an equal value) written to codes[i * stride]
void dict_build(const DevCol &c, int prefix, uint64_t *table, uint64_t cap, uint32_t *codes, int64_t stride,
                cudaStream_t s);
void dict_probe(const DevCol &probe, int prefix, const DevCol &owner, int owner_prefix, const uint64_t *table,
                uint64_t cap, uint32_t *codes, int64_t stride, cudaStream_t s);
void part_feature(const DevCol &c, int prefix, uint32_t m, uint32_t *rec, int W, int word, cudaStream_t s);
// hot[i][h] = rec[i][map[h]] (0 where map[h] < 0); HW <= 64
void hot_pack(const uint32_t *rec, int W, int64_t n, uint32_t *hot, int HW, const int32_t *map, cudaStream_t s);
void ed_features(const DevCol &c, uint32_t *rec, int W, int feat, cudaStream_t s);
void abs_feature(const DevCol &c, uint32_t *rec, int W, int feat, cudaStream_t s);
// one word per row: 1 when the row's value equals the constant (device bytes; int32 little-endian)
void const_feature(const DevCol &c, const uint8_t *cval_dev, uint32_t clen, uint32_t *rec, int W, int feat,
                   cudaStream_t s);
// word tokens (maximal runs of bytes other than 0x20): toff[n+1] exclusive starts; returns the total
size_t tok_scratch_bytes(int64_t n);
int64_t tok_count(const DevCol &c, uint32_t *toff, void *scratch, size_t scratch_bytes, cudaStream_t s);
void tok_fill(const DevCol &c, const uint32_t *toff, uint32_t *tstart, uint32_t *tlen, cudaStream_t s);
void tok_insert(const uint8_t *bytes, const uint32_t *tstart, const uint32_t *tlen, int64_t T, uint64_t *table,
                uint64_t cap, uint32_t *codes, cudaStream_t s);
void tok_probe(const uint8_t *bytes, const uint32_t *tstart, const uint32_t *tlen, int64_t T, const uint8_t *obytes,
               const uint32_t *ostart, const uint32_t *olen, const uint64_t *table, uint64_t cap, uint32_t *codes,
               cudaStream_t s);
// per string: local codes for tokens absent from the owner, sort, unique, Jaccard feature words
void tok_lists(const DevCol &c, const uint32_t *toff, const uint32_t *tstart, const uint32_t *tlen, uint32_t *codes,
               uint32_t *rec, int W, int feat, unsigned int *too_long, cudaStream_t s);
size_t jac_scratch_bytes(int64_t n);
// grams: capacity >= the column's byte count; too_long: device flag set for strings of > 8192 grams
void jac_features_impl(const DevCol &c, int q, uint32_t *rec, int W, int feat, uint32_t *grams, void *scratch,
                       unsigned int *too_long, int n_sm, cudaStream_t s);

// k_block.cu
void group_build(const uint32_t *rec, int W, int64_t n, const int32_t *eq_words, int n_keys, uint64_t *table,
                 uint64_t cap, uint32_t *slot, cudaStream_t s);
void group_probe(const uint32_t *rec_probe, int64_t n, const uint32_t *rec_owner, int W, const int32_t *eq_words,
                 int n_keys, const uint64_t *table, uint64_t cap, uint32_t *slot, cudaStream_t s);
void count_slots(const uint32_t *slot, int64_t n, uint32_t *count, cudaStream_t s);
void scatter_slots(const uint32_t *slot, int64_t n, const uint32_t *start, uint32_t *cursor, uint32_t *members,
                   cudaStream_t s);
// sharded evaluation: the counts of groups (slots) owned by another rank are set
// to 0, so their blocks are not emitted; minrow: cap words of scratch
void shard_filter(const uint32_t *slot_r, int64_t n_r, uint32_t *count_r, uint32_t *count_s, uint32_t *minrow,
                  uint64_t cap, uint32_t md, uint32_t rank, uint32_t world, cudaStream_t s);
void emit_blocks(const uint32_t *count_r, const uint32_t *start_r, const uint32_t *count_s, const uint32_t *start_s,
                 uint64_t cap, uint32_t md, int self_join, uint32_t member_base_r, uint32_t member_base_s, int tile,
                 BlockDesc *blocks, uint64_t *tiles, uint32_t *n_blocks, uint32_t block_cap, unsigned int *overflow,
                 cudaStream_t s);
// self-join: blocks of more than SMALL_MAX tuples as emit_blocks; smaller ones
// packed into tiles (start list `small`, metadata `small_meta`)
void emit_blocks_packed(const uint32_t *count_r, const uint32_t *start_r, uint64_t cap, uint32_t md,
                        uint32_t member_base_r, int tile, BlockDesc *blocks, uint64_t *tiles, uint32_t *n_blocks,
                        uint32_t *n_packed, uint32_t block_cap, unsigned int *overflow, uint32_t *small_meta,
                        uint32_t *small, uint32_t small_cap, uint32_t *small_total, int n_sm, cudaStream_t s);
void clamp_blocks(uint32_t *n_blocks, uint32_t block_cap, cudaStream_t s);

// k_eval.cu
size_t eval_smem_bytes(int W, int n_eq, int use_lut, int tile);
int eval_blocks_per_sm(int tile, int logging, size_t smem);
// the paper's per-pair model N, 8 -> 2 -> 6 -> 1 (k_mlp.cu)
cudaError_t pair_model_forward(const float *X, int n, const float *params, float *y, cudaStream_t s);
cudaError_t pair_model_backward(const float *X, const float *t, int n, const float *params, float *grad,
                                cudaStream_t s);
// per-pair cycles, verdict and the paper's per-pair model features of program op k (k_eval.cu)
cudaError_t launch_pair_times(const EvalParams &p, int k, const uint32_t *pi, const uint32_t *pj, int n,
                              uint32_t *cycles, uint8_t *verdict, float *X, cudaStream_t s);
cudaError_t launch_eval(const EvalParams &p, int grid, size_t smem, int logging, cudaStream_t s);
void pack_pairs(const uint64_t *keys, int64_t n, int key_bits_s, hb_pair *out, cudaStream_t s);

// k_stats.cu
struct SampleSpec {
    int32_t kind;
    int32_t type;
    const uint8_t *bytes;
    const uint32_t *off;
    const void *vals;
    const uint8_t *valid;
    int32_t prefix;
    int32_t q;
    float delta;
    int32_t pad;
};
void lsh_hist(const SampleSpec *specs_dev, int n_preds, int64_t n_rows, int n_samples, int k_buckets,
              uint32_t *hist, uint32_t *lens, uint32_t *grams, int n_keep, cudaStream_t s);

// planner.cpp
struct PlanResult {
    std::vector<int> pred_order;
    std::vector<int> md_order;
    std::vector<int> program;
    std::vector<int> cp;
    std::vector<double> wp;
};
PlanResult make_plan(int n_preds, const double *sp, const double *cost, const std::vector<std::vector<int>> &mds,
                     const std::vector<uint8_t> &skip);

// k_mlp.cu
cudaError_t mlp_forward(const float *X, int n, const float *params, float *y, int bf16, cudaStream_t s);
cudaError_t mlp_backward(const float *X, const float *t, int n, const float *params, float *grad, float *work,
                         cudaStream_t s);
size_t mlp_work_floats(int n);
cudaError_t adam_step(float *params, const float *grad, float *m, float *v, int n, int step, float lr, float b1,
                      float b2, float eps, cudaStream_t s);

}  // namespace hb
