// R x S blocking with S streamed from host memory (hb_block_stream).
//
// Section 3 pipelines host-to-device transfer with device work so that the
// transfer of one part overlaps the processing of another.  Here R is
// resident and grouped once per MD; S arrives in chunks of at most
// chunk_bytes, copied on a copy stream into one of two device buffers (straight
// from page-locked caller memory, or packed into one of two pinned buffers
// first) while the previous chunk is encoded (dictionary codes
// looked up in R's dictionaries, string features), grouped against R's groups
// and evaluated on the compute stream.  Pairs of all chunks accumulate in one
// slab and are sorted once at the end.
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <thread>
#include <vector>

#include "hb_ctx.h"

namespace hb {
namespace {

__global__ void k_rebase(uint32_t *off, int64_t n1, uint32_t base) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n1) off[i] -= base;
}

struct ChunkCol {
    size_t bytes_off = 0, off_off = 0, vals_off = 0, valid_off = 0;   // byte offsets in the chunk buffer
    size_t bytes_len = 0, off_len = 0, vals_len = 0, valid_len = 0;
};

inline size_t a16(size_t x) { return (x + 255) & ~size_t(255); }

// layout of rows [r0, r1) of the needed columns in one contiguous buffer
size_t chunk_layout(const hb_column *cols, const std::vector<int> &need, int64_t r0, int64_t r1,
                    std::vector<ChunkCol> &cc) {
    size_t pos = 0;
    cc.assign(need.size(), ChunkCol());
    for (size_t i = 0; i < need.size(); i++) {
        const hb_column &c = cols[need[i]];
        ChunkCol &k = cc[i];
        const int64_t n = r1 - r0;
        if (c.type == HB_COL_STRING) {
            k.bytes_off = pos;
            k.bytes_len = (size_t)(c.offsets[r1] - c.offsets[r0]);
            pos = a16(pos + k.bytes_len + 16);
            k.off_off = pos;
            k.off_len = sizeof(uint32_t) * (size_t)(n + 1);
            pos = a16(pos + k.off_len);
        } else {
            k.vals_off = pos;
            k.vals_len = 4 * (size_t)n;
            pos = a16(pos + k.vals_len);
        }
        if (c.valid) {
            k.valid_off = pos;
            k.valid_len = (size_t)n;
            pos = a16(pos + k.valid_len);
        }
    }
    return pos;
}

void pack_chunk(const hb_column *cols, const std::vector<int> &need, int64_t r0, int64_t r1,
                const std::vector<ChunkCol> &cc, uint8_t *dst) {
    for (size_t i = 0; i < need.size(); i++) {
        const hb_column &c = cols[need[i]];
        const ChunkCol &k = cc[i];
        if (c.type == HB_COL_STRING) {
            memcpy(dst + k.bytes_off, static_cast<const uint8_t *>(c.data) + c.offsets[r0], k.bytes_len);
            memcpy(dst + k.off_off, c.offsets + r0, k.off_len);   // rebased on the device
        } else {
            memcpy(dst + k.vals_off, static_cast<const uint8_t *>(c.data) + 4 * (size_t)r0, k.vals_len);
        }
        if (c.valid) memcpy(dst + k.valid_off, c.valid + r0, k.valid_len);
    }
}

// the same chunk copied from page-locked caller memory, one DMA per array
cudaError_t copy_chunk_direct(const hb_column *cols, const std::vector<int> &need, int64_t r0, int64_t r1,
                              const std::vector<ChunkCol> &cc, uint8_t *dst, cudaStream_t s) {
    (void)r1;
    for (size_t i = 0; i < need.size(); i++) {
        const hb_column &c = cols[need[i]];
        const ChunkCol &k = cc[i];
        cudaError_t e = cudaSuccess;
        if (c.type == HB_COL_STRING) {
            if (k.bytes_len)
                e = cudaMemcpyAsync(dst + k.bytes_off, static_cast<const uint8_t *>(c.data) + c.offsets[r0],
                                    k.bytes_len, cudaMemcpyHostToDevice, s);
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(dst + k.off_off, c.offsets + r0, k.off_len, cudaMemcpyHostToDevice, s);
        } else {
            e = cudaMemcpyAsync(dst + k.vals_off, static_cast<const uint8_t *>(c.data) + 4 * (size_t)r0, k.vals_len,
                                cudaMemcpyHostToDevice, s);
        }
        if (e == cudaSuccess && c.valid)
            e = cudaMemcpyAsync(dst + k.valid_off, c.valid + r0, k.valid_len, cudaMemcpyHostToDevice, s);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace

// encoding of one S chunk, asynchronous (the Jaccard length flag is checked later)
static hb_status encode_chunk(hb_ctx *c, SideData &S, unsigned int *too_long, Buf &grams_buf,
                              std::vector<size_t> &gram_off) {
    const int64_t n = S.n;
    const int W = c->W;
    HB_CUDA(cudaMemsetAsync(S.rec, 0, sizeof(uint32_t) * (size_t)W * (size_t)std::max<int64_t>(n, 1), c->stream));
    for (size_t e = 0; e < c->eqkeys.size(); e++) {
        const EqKey &k = c->eqkeys[e];
        dict_probe(S.cols[k.col_s], k.prefix, c->side[0].cols[k.col_t], k.prefix, c->dict[e], c->dict_cap[e],
                   S.rec + e, W, c->stream);
    }
    S.grams.assign(c->groups.size(), nullptr);
    S.gram_len.assign(c->groups.size(), 0);
    for (size_t g = 0; g < c->groups.size(); g++) {
        const FeatGroup &G = c->groups[g];
        const DevCol &col = S.cols[G.col_s];
        if (G.kind == OP_ED) {
            ed_features(col, S.rec, W, G.word, c->stream);
        } else if (G.kind == OP_ABS) {
            abs_feature(col, S.rec, W, G.word, c->stream);
        } else {
            S.grams[g] = as<uint32_t>(grams_buf) + gram_off[g];
            S.gram_len[g] = (g + 1 < gram_off.size() ? gram_off[g + 1] : grams_buf.bytes / 4) - gram_off[g];
            jac_features_impl(col, G.q, S.rec, W, G.word, S.grams[g], c->w_jac.p, too_long, c->n_sm, c->stream);
        }
    }
    hot_pack(S.rec, W, n, S.hot, c->HW, c->hot_map.data(), c->stream);
    HB_CUDA(cudaGetLastError());
    return HB_OK;
}

}  // namespace hb

using namespace hb;

extern "C" hb_status hb_block_stream(hb_ctx *c, int64_t n_rows_s, int32_t n_cols, const hb_column *cols_s,
                                     hb_pair **pairs_out, int64_t *n_out) {
    if (!c || !pairs_out || !n_out || (n_cols > 0 && !cols_s)) return fail(HB_ERR_ARG, "hb_block_stream: NULL argument");
    *pairs_out = nullptr;
    *n_out = 0;
    if (c->side[0].cols.empty() && c->side[0].n == 0) return fail(HB_ERR_STATE, "hb_block_stream: R not loaded");
    if (c->part_m) return fail(HB_ERR_STATE, "hb_block_stream: partitioned blocking runs on hb_block only");
    if (c->shard_world > 1) return fail(HB_ERR_STATE, "hb_block_stream: sharded evaluation runs on hb_block only");
    if (n_rows_s < 0 || n_rows_s >= (1ll << 30)) return fail(HB_ERR_ARG, "hb_block_stream: n_rows_s out of range");
    for (int k = 0; k < n_cols; k++) {
        const hb_column &col = cols_s[k];
        if (col.type < 0 || col.type > 2) return fail(HB_ERR_ARG, "hb_block_stream: unknown column type");
        if (col.type == HB_COL_STRING) {
            if (!col.offsets || col.offsets[0] != 0) return fail(HB_ERR_ARG, "hb_block_stream: bad string offsets");
            uint32_t dec = 0;   // branch-free (vectorises)
            for (int64_t i = 0; i < n_rows_s; i++) dec |= col.offsets[i + 1] < col.offsets[i] ? 1u : 0u;
            if (dec) return fail(HB_ERR_ARG, "hb_block_stream: offsets decrease");
        }
    }
    cudaSetDevice(c->device);
    auto w0 = std::chrono::steady_clock::now();
    // S is described (types) but not resident: the plan validates col_s against it
    bool retype = c->side[1].cols.size() != (size_t)n_cols;
    for (int k = 0; k < n_cols && !retype; k++) retype = c->side[1].cols[k].type != cols_s[k].type;
    if (retype || !c->side[1].allocs.empty()) {
        for (void *p : c->side[1].allocs) cudaFreeAsync(p, c->stream);
        c->side[1].allocs.clear();
        c->side[1].cols.assign(n_cols, DevCol());
        for (int k = 0; k < n_cols; k++) c->side[1].cols[k].type = cols_s[k].type;
        c->planned = false;
    }
    c->side[1].n = 0;
    if (!c->planned || c->batch_layout) HB_TRY(do_plan(c, HB_PLAN_RULE_DATA, false));
    for (const FeatGroup &G : c->groups)
        if (G.kind == OP_CONST || G.tokens)
            return fail(HB_ERR_ARG, "hb_block_stream: constants and word-token Jaccard are not supported when S is "
                                    "streamed (load S with hb_load_table and call hb_block)");
    HB_TRY(encode_side(c, 0));
    HB_TRY(grow(c, c->w_counters, 64 * sizeof(unsigned long long)));
    if (!c->lut.empty()) {
        HB_TRY(grow(c, c->w_lut, sizeof(uint64_t) * c->lut.size()));
        HB_CUDA(cudaMemcpyAsync(c->w_lut.p, c->lut.data(), sizeof(uint64_t) * c->lut.size(), cudaMemcpyHostToDevice,
                                c->stream));
    }
    if (!c->tile) c->tile = 32;

    // needed S columns and chunk boundaries
    std::vector<int> need;
    for (auto &G : c->groups) need.push_back(G.col_s);
    for (auto &k : c->eqkeys) need.push_back(k.col_s);
    std::sort(need.begin(), need.end());
    need.erase(std::unique(need.begin(), need.end()), need.end());
    const size_t chunk_bytes = c->opt.chunk_bytes ? c->opt.chunk_bytes : (256ull << 20);
    // bytes of rows [0, i) in a chunk: string bytes (from the offsets) plus a
    // fixed part per row; a chunk is the longest run of rows within the budget
    size_t fixed_row = 0;
    for (int k : need) fixed_row += 4 + (cols_s[k].valid ? 1 : 0);   // offset or value, validity byte
    auto cum = [&](int64_t i) {
        size_t b = (size_t)i * fixed_row;
        for (int k : need)
            if (cols_s[k].type == HB_COL_STRING) b += cols_s[k].offsets[i];
        return b;
    };
    std::vector<int64_t> bounds = {0};
    {
        const size_t budget = chunk_bytes > 8192 ? chunk_bytes - 256 * (need.size() * 3 + 4) : chunk_bytes / 2;
        int64_t b0 = 0;
        while (b0 < n_rows_s) {
            const size_t base = cum(b0);
            int64_t lo = b0 + 1, hi = n_rows_s;   // the chunk end: largest e in [lo, hi] within the budget
            if (cum(lo) - base <= budget) {
                while (lo < hi) {
                    const int64_t mid = lo + (hi - lo + 1) / 2;
                    if (cum(mid) - base <= budget) lo = mid;
                    else hi = mid - 1;
                }
            }
            bounds.push_back(lo);
            b0 = lo;
        }
    }
    const int K = (int)bounds.size() - 1;
    int64_t max_rows = 1;
    size_t max_buf = 256, max_str = 16;
    std::vector<std::vector<ChunkCol>> layouts(K);
    std::vector<size_t> sizes(K);
    for (int k = 0; k < K; k++) {
        sizes[k] = chunk_layout(cols_s, need, bounds[k], bounds[k + 1], layouts[k]);
        max_buf = std::max(max_buf, sizes[k]);
        max_rows = std::max<int64_t>(max_rows, bounds[k + 1] - bounds[k]);
        for (auto &cc : layouts[k]) max_str = std::max(max_str, cc.bytes_len);
    }
    if (max_buf > chunk_bytes && K > 0 && max_rows > 1)
        return fail(HB_ERR_ARG, "hb_block_stream: a chunk exceeds chunk_bytes");
    // R's member lists and a chunk's are addressed with 32 bits per active MD
    if (!member_addressing_fits((int64_t)c->active.size(), std::max<int64_t>(c->side[0].n, max_rows)))
        return fail(HB_ERR_ARG, "hb_block_stream: rows x active MDs exceed the 32-bit member addressing");

    // staging: two device chunk buffers and a copy stream kept by the context;
    // page-locked S arrays are copied straight from the caller's memory, any
    // other S goes through two pinned buffers (c->pin)
    bool direct = true;
    for (int k : need) {
        const hb_column &col = cols_s[k];
        if (n_rows_s > 0 && col.data && !page_locked(col.data)) direct = false;
        if (col.type == HB_COL_STRING && !page_locked(col.offsets)) direct = false;
        if (col.valid && !page_locked(col.valid)) direct = false;
    }
    if (!direct) HB_TRY(ensure_pinned(c, max_buf));
    for (int b = 0; b < 2; b++) {
        HB_TRY(grow(c, c->w_chunk[b], max_buf));
        if (!c->chunk_copied[b]) HB_CUDA(cudaEventCreateWithFlags(&c->chunk_copied[b], cudaEventDisableTiming));
        if (!c->chunk_consumed[b]) HB_CUDA(cudaEventCreateWithFlags(&c->chunk_consumed[b], cudaEventDisableTiming));
        HB_CUDA(cudaEventRecord(c->chunk_consumed[b], c->stream));
    }
    if (!c->copy_stream) HB_CUDA(cudaStreamCreateWithFlags(&c->copy_stream, cudaStreamNonBlocking));
    void *dbuf[2] = {c->w_chunk[0].p, c->w_chunk[1].p};
    cudaStream_t cs = c->copy_stream;
    cudaEvent_t *copied = c->chunk_copied, *consumed = c->chunk_consumed;
    auto cleanup = [&]() {
        cudaStreamSynchronize(c->stream);
        cudaStreamSynchronize(cs);
        c->side[1].rec = nullptr;
        c->side[1].hot = nullptr;
        c->side[1].grams.clear();
        c->side[1].n = 0;
        for (auto &col : c->side[1].cols) {
            int t = col.type;
            col = DevCol();
            col.type = t;
        }
    };
#define HB_SCUDA(call)                                                                     \
    do {                                                                                   \
        cudaError_t e__ = (call);                                                          \
        if (e__ != cudaSuccess) {                                                          \
            cleanup();                                                                     \
            return fail(HB_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e__)); \
        }                                                                                  \
    } while (0)
#define HB_STRY(expr)           \
    do {                        \
        hb_status s__ = (expr); \
        if (s__ != HB_OK) {     \
            cleanup();          \
            return s__;         \
        }                       \
    } while (0)

    // R side: groups of every active MD, kept for all chunks
    const int64_t n_r = c->side[0].n;
    const int W = c->W;
    const int na = (int)c->active.size();
    const uint64_t H = pow2_at_least(std::max<uint64_t>(2 * (uint64_t)std::max<int64_t>(n_r, 1), 1024));
    Buf tables, cnt_r, start_r, chunk_rec, chunk_hot, chunk_grams, flag;
    HB_STRY(grow(c, tables, sizeof(uint64_t) * H * std::max(na, 1)));
    HB_STRY(grow(c, cnt_r, sizeof(uint32_t) * (H + 1) * std::max(na, 1)));
    HB_STRY(grow(c, start_r, sizeof(uint32_t) * (H + 1) * std::max(na, 1)));
    HB_STRY(grow(c, c->w_slot_r, sizeof(uint32_t) * (size_t)(n_r + 1)));
    HB_STRY(grow(c, c->w_cursor, sizeof(uint32_t) * (H + 1)));
    HB_STRY(grow(c, c->w_members_r, sizeof(uint32_t) * (size_t)std::max<int64_t>(n_r, 1) * std::max(na, 1)));
    HB_STRY(grow(c, c->w_scan, scan_tmp_bytes((int64_t)H + 1)));
    std::vector<std::vector<int32_t>> words(na);
    for (int a = 0; a < na; a++) {
        const int m = c->active[a];
        for (int e = 0; e < c->n_eq_total; e++)
            if (c->eqset[m] & (1u << e)) words[a].push_back(e);
        uint64_t *tab = as<uint64_t>(tables) + H * a;
        uint32_t *cr = as<uint32_t>(cnt_r) + (H + 1) * a, *sr = as<uint32_t>(start_r) + (H + 1) * a;
        group_build(c->side[0].rec, W, n_r, words[a].data(), (int)words[a].size(), tab, H, as<uint32_t>(c->w_slot_r),
                    c->stream);
        HB_SCUDA(cudaMemsetAsync(cr, 0, sizeof(uint32_t) * (H + 1), c->stream));
        count_slots(as<uint32_t>(c->w_slot_r), n_r, cr, c->stream);
        scan_exclusive_u32(cr, sr, (int64_t)H, nullptr, c->w_scan.p, c->w_scan.bytes, c->stream);
        HB_SCUDA(cudaMemsetAsync(c->w_cursor.p, 0, sizeof(uint32_t) * (H + 1), c->stream));
        scatter_slots(as<uint32_t>(c->w_slot_r), n_r, sr, as<uint32_t>(c->w_cursor),
                      as<uint32_t>(c->w_members_r) + (size_t)a * (size_t)std::max<int64_t>(n_r, 1), c->stream);
    }
    // per-chunk buffers (sized for the largest chunk)
    const uint64_t per_md = (uint64_t)std::min<int64_t>(n_r, max_rows) + 1;
    const uint32_t block_cap = (uint32_t)std::min<uint64_t>(per_md * std::max(na, 1), 0xFFFFFFF0ull);
    HB_STRY(grow(c, chunk_rec, sizeof(uint32_t) * (size_t)W * (size_t)max_rows + 64));
    HB_STRY(grow(c, chunk_hot, sizeof(uint32_t) * (size_t)c->HW * (size_t)max_rows + 64));
    std::vector<size_t> gram_off(c->groups.size(), 0);
    size_t gram_words = 16;
    for (size_t g = 0; g < c->groups.size(); g++) {
        gram_off[g] = gram_words;
        if (c->groups[g].kind == OP_JAC) gram_words += max_str + 16;
    }
    HB_STRY(grow(c, chunk_grams, sizeof(uint32_t) * gram_words));
    HB_STRY(grow(c, flag, 16));
    HB_STRY(grow(c, c->w_jac, jac_scratch_bytes(max_rows)));
    HB_STRY(grow(c, c->w_slot_s, sizeof(uint32_t) * (size_t)(max_rows + 1)));
    HB_STRY(grow(c, c->w_count_s, sizeof(uint32_t) * (H + 1)));
    HB_STRY(grow(c, c->w_start_s, sizeof(uint32_t) * (H + 1)));
    HB_STRY(grow(c, c->w_members_s, sizeof(uint32_t) * (size_t)max_rows * std::max(na, 1)));
    HB_STRY(grow(c, c->w_blocks, sizeof(BlockDesc) * (size_t)block_cap));
    HB_STRY(grow(c, c->w_tiles, sizeof(uint64_t) * ((size_t)block_cap + 1)));
    HB_STRY(grow(c, c->w_prefix, sizeof(uint64_t) * ((size_t)block_cap + 1)));
    HB_STRY(grow(c, c->w_scan, std::max(scan_tmp_bytes((int64_t)H + 1), scan_tmp_bytes((int64_t)block_cap + 1))));
    HB_STRY(grow(c, c->w_log, sizeof(unsigned long long) * MAX_OPS * 8));
    if (c->out_cap == 0) c->out_cap = c->opt.out_capacity > 0 ? c->opt.out_capacity : std::max<int64_t>(1 << 20, n_r);
    HB_STRY(grow(c, c->w_out, sizeof(uint64_t) * (size_t)c->out_cap));
    unsigned long long *ctr = as<unsigned long long>(c->w_counters);
    HB_SCUDA(cudaMemsetAsync(ctr, 0, 64 * sizeof(unsigned long long), c->stream));
    HB_SCUDA(cudaMemsetAsync(flag.p, 0, 16, c->stream));
    const int kbs = bits_for((uint64_t)std::max<int64_t>(n_rows_s, 2));
    const int kb = kbs + bits_for((uint64_t)std::max<int64_t>(n_r, 2));
    const size_t smem = eval_smem_bytes(c->HW, c->n_eq_total, c->lut.empty() ? 0 : 1, c->tile);
    const int bps = eval_blocks_per_sm(c->tile, 0, smem);
    if (bps < 1) {
        cleanup();
        return fail(HB_ERR_ARG, "record too wide for the evaluation kernel's shared memory");
    }
    const int grid = bps * c->n_sm;
    HB_SCUDA(cudaStreamSynchronize(c->stream));

    double ms_copy_wait = 0;
    int64_t cand = 0, exam = 0, tiles = 0, blocks = 0;
    unsigned long long out_before = 0;
    // chunk 0 in flight
    auto issue_copy = [&](int k) -> cudaError_t {
        const int b = k & 1;
        cudaError_t e;
        if (direct) {
            // the copy stream waits for the device buffer's previous chunk
            e = cudaStreamWaitEvent(cs, consumed[b], 0);
            if (e != cudaSuccess) return e;
            e = copy_chunk_direct(cols_s, need, bounds[k], bounds[k + 1], layouts[k],
                                  static_cast<uint8_t *>(dbuf[b]), cs);
        } else {
            // the pinned buffer and the device buffer of chunk k-2 are both free
            e = cudaEventSynchronize(consumed[b]);
            if (e != cudaSuccess) return e;
            uint8_t *pin = static_cast<uint8_t *>(c->pin[b]);
            pack_chunk(cols_s, need, bounds[k], bounds[k + 1], layouts[k], pin);
            e = cudaMemcpyAsync(dbuf[b], pin, sizes[k], cudaMemcpyHostToDevice, cs);
        }
        if (e != cudaSuccess) return e;
        return cudaEventRecord(copied[b], cs);
    };
    if (K > 0) HB_SCUDA(issue_copy(0));
    for (int k = 0; k < K; k++) {
        const int b = k & 1;
        const int64_t r0 = bounds[k], nk = bounds[k + 1] - bounds[k];
        HB_SCUDA(cudaStreamWaitEvent(c->stream, copied[b], 0));
        // chunk columns on the device
        SideData &S = c->side[1];
        S.n = nk;
        uint8_t *base = static_cast<uint8_t *>(dbuf[b]);
        for (size_t i = 0; i < need.size(); i++) {
            const hb_column &hc = cols_s[need[i]];
            const ChunkCol &cc = layouts[k][i];
            DevCol &d = S.cols[need[i]];
            d.type = hc.type;
            d.n = nk;
            if (hc.type == HB_COL_STRING) {
                d.bytes = base + cc.bytes_off;
                d.nbytes = cc.bytes_len;
                d.off = reinterpret_cast<uint32_t *>(base + cc.off_off);
                HB_LAUNCHED(1);
                k_rebase<<<(unsigned)((nk + 1 + 255) / 256), 256, 0, c->stream>>>(d.off, nk + 1, hc.offsets[r0]);
            } else {
                d.vals = base + cc.vals_off;
            }
            d.valid = hc.valid ? base + cc.valid_off : nullptr;
        }
        S.rec = as<uint32_t>(chunk_rec);
        S.hot = as<uint32_t>(chunk_hot);
        HB_STRY(encode_chunk(c, S, as<unsigned int>(flag), chunk_grams, gram_off));
        // groups of the chunk against R's groups, blocks, tiles
        HB_SCUDA(cudaMemsetAsync(ctr, 0, sizeof(unsigned long long), c->stream));          // tile claims
        HB_SCUDA(cudaMemsetAsync(ctr + 3, 0, 2 * sizeof(unsigned long long), c->stream));  // blocks, overflow
        for (int a = 0; a < na; a++) {
            const int m = c->active[a];
            uint64_t *tab = as<uint64_t>(tables) + H * a;
            uint32_t *cr = as<uint32_t>(cnt_r) + (H + 1) * a, *sr = as<uint32_t>(start_r) + (H + 1) * a;
            group_probe(S.rec, nk, c->side[0].rec, W, words[a].data(), (int)words[a].size(), tab, H,
                        as<uint32_t>(c->w_slot_s), c->stream);
            HB_SCUDA(cudaMemsetAsync(c->w_count_s.p, 0, sizeof(uint32_t) * (H + 1), c->stream));
            count_slots(as<uint32_t>(c->w_slot_s), nk, as<uint32_t>(c->w_count_s), c->stream);
            scan_exclusive_u32(as<uint32_t>(c->w_count_s), as<uint32_t>(c->w_start_s), (int64_t)H, nullptr,
                               c->w_scan.p, c->w_scan.bytes, c->stream);
            HB_SCUDA(cudaMemsetAsync(c->w_cursor.p, 0, sizeof(uint32_t) * (H + 1), c->stream));
            scatter_slots(as<uint32_t>(c->w_slot_s), nk, as<uint32_t>(c->w_start_s), as<uint32_t>(c->w_cursor),
                          as<uint32_t>(c->w_members_s) + (size_t)a * (size_t)max_rows, c->stream);
            emit_blocks(cr, sr, as<uint32_t>(c->w_count_s), as<uint32_t>(c->w_start_s), H, (uint32_t)m, 0,
                        (uint32_t)((size_t)a * (size_t)std::max<int64_t>(n_r, 1)), (uint32_t)((size_t)a * max_rows),
                        c->tile, as<BlockDesc>(c->w_blocks), as<uint64_t>(c->w_tiles),
                        reinterpret_cast<uint32_t *>(ctr + 3), block_cap, reinterpret_cast<unsigned int *>(ctr + 4),
                        c->stream);
        }
        clamp_blocks(reinterpret_cast<uint32_t *>(ctr + 3), block_cap, c->stream);
        scan_exclusive_u64(as<uint64_t>(c->w_tiles), as<uint64_t>(c->w_prefix), (int64_t)block_cap,
                           reinterpret_cast<const uint32_t *>(ctr + 3), c->w_scan.p, c->w_scan.bytes, c->stream);
        // the next chunk's copy (into the other buffer) overlaps this chunk's evaluation
        if (k + 1 < K) HB_SCUDA(issue_copy(k + 1));
        for (int attempt = 0; attempt < 2; attempt++) {
            EvalParams P = make_params(c, c->side[0].rec, S.rec, 1, false, ctr, kbs);
            P.col_base = (uint32_t)r0;
            HB_SCUDA(launch_eval(P, grid, smem, 0, c->stream));
            unsigned long long h[6];
            HB_SCUDA(cudaMemcpyAsync(h, ctr, sizeof(h), cudaMemcpyDeviceToHost, c->stream));
            auto t0 = std::chrono::steady_clock::now();
            HB_SCUDA(cudaStreamSynchronize(c->stream));
            ms_copy_wait += std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
            if (h[4]) {
                cleanup();
                return fail(HB_ERR_INTERNAL, "block list overflow");
            }
            if (h[1] <= (unsigned long long)c->out_cap) {
                cand += (int64_t)h[2];
                exam += (int64_t)h[5];
                blocks += (int64_t)(uint32_t)h[3];
                uint64_t t = 0;
                HB_SCUDA(cudaMemcpy(&t, as<uint64_t>(c->w_prefix) + (uint32_t)h[3], sizeof(uint64_t),
                                    cudaMemcpyDeviceToHost));
                tiles += (int64_t)t;
                HB_SCUDA(cudaMemsetAsync(ctr + 2, 0, sizeof(unsigned long long), c->stream));
                HB_SCUDA(cudaMemsetAsync(ctr + 5, 0, sizeof(unsigned long long), c->stream));
                out_before = h[1];
                break;
            }
            // grow the slab, keeping the pairs of earlier chunks, and evaluate this chunk again
            const int64_t need_cap = (int64_t)h[1] + (int64_t)h[1] / 8 + 1024;
            Buf bigger;
            HB_STRY(grow(c, bigger, sizeof(uint64_t) * (size_t)need_cap));
            HB_SCUDA(cudaMemcpyAsync(bigger.p, c->w_out.p, sizeof(uint64_t) * out_before, cudaMemcpyDeviceToDevice,
                                     c->stream));
            free_buf(c, c->w_out);
            c->w_out = bigger;
            c->out_cap = need_cap;
            HB_SCUDA(cudaMemcpyAsync(ctr + 1, &out_before, sizeof(unsigned long long), cudaMemcpyHostToDevice,
                                     c->stream));
            HB_SCUDA(cudaMemsetAsync(ctr, 0, sizeof(unsigned long long), c->stream));
            HB_SCUDA(cudaMemsetAsync(ctr + 2, 0, sizeof(unsigned long long), c->stream));
            HB_SCUDA(cudaMemsetAsync(ctr + 5, 0, sizeof(unsigned long long), c->stream));
        }
        // the evaluation reads string bytes of the chunk: its buffer is free only now
        HB_SCUDA(cudaEventRecord(consumed[b], c->stream));
    }
    unsigned int too_long = 0;
    HB_SCUDA(cudaMemcpy(&too_long, flag.p, sizeof(unsigned int), cudaMemcpyDeviceToHost));
    if (too_long) {
        cleanup();
        return fail(HB_ERR_ARG, "a string compared by q-gram Jaccard has more than 8192 grams");
    }
    const int64_t n_pairs = (int64_t)out_before;
    HB_STRY(grow(c, c->w_alt, sizeof(uint64_t) * (size_t)std::max<int64_t>(n_pairs, 1)));
    HB_STRY(grow(c, c->w_sort, radix_tmp_bytes(std::max<int64_t>(n_pairs, 1))));
    uint64_t *sorted = nullptr;
    radix_sort_u64(as<uint64_t>(c->w_out), as<uint64_t>(c->w_alt), n_pairs, nullptr, kb, c->w_sort.p,
                   c->w_sort.bytes, c->stream, &sorted);
    hb_pair *out = nullptr;
    HB_STRY(check_bounds(c, "hb_block_stream"));
    HB_STRY(deliver(c, sorted, n_pairs, kbs, true, &out));
    cleanup();
    Buf *tmp[] = {&tables, &cnt_r, &start_r, &chunk_rec, &chunk_hot, &chunk_grams, &flag};
    for (Buf *t : tmp) free_buf(c, *t);
    *pairs_out = out;
    *n_out = n_pairs;
    c->stats.candidate_pairs = cand;
    c->stats.examined_pairs = exam;
    c->stats.emitted_pairs = n_pairs;
    c->stats.tiles = tiles;
    c->stats.blocks = blocks;
    c->stats.n_rows_s = n_rows_s;
    c->stats.ms_total = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - w0).count();
    c->stats.ms_h2d = ms_copy_wait;
    return HB_OK;
#undef HB_SCUDA
#undef HB_STRY
}
