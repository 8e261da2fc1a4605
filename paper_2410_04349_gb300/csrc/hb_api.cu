// libhb C-ABI: context, table loading, rules, planning and the blocking
// pipelines (self-join, R x S, streamed R x S, batched jobs).
//
// Pipeline of one blocking call (Section 3 overview, GB300 form):
//   encode    : exact dictionary codes of the equality keys, per-string
//               features for edit distance / q-gram Jaccard, packed records;
//   plan      : Section 4.2 ordering + execution tree -> sequential program;
//   blocks    : per MD, tuples grouped by all of its equality keys;
//   evaluate  : tiles of every block's pair space, persistent work queue;
//   output    : radix sort of the packed pairs, copy to the caller.
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <array>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <numeric>
#include <random>
#include <string>
#include <thread>
#include <vector>

#include "hb_ctx.h"

namespace hb {

std::atomic<long long> g_kernel_launches{0};

static thread_local std::string g_err;

hb_status fail(hb_status st, const std::string &msg) {
    g_err = msg;
    return st;
}

}  // namespace hb

using namespace hb;

namespace hb {

// Host-side fault injection: HB_FAIL_ALLOC_AFTER=N in the environment at
// hb_create makes the (N+1)-th device or page-locked allocation of the context
// fail once with HB_ERR_OOM, as a real shortage would.
static bool injected_failure(hb_ctx *c) {
    if (c->fail_alloc_after < 0) return false;
    if (c->fail_alloc_after == 0) {
        c->fail_alloc_after = -1;
        return true;
    }
    c->fail_alloc_after--;
    return false;
}

hb_status grow(hb_ctx *c, Buf &b, size_t bytes) {
    if (bytes == 0) bytes = 16;
    if (b.bytes >= bytes) return HB_OK;
    if (b.p) {
        cudaFreeAsync(b.p, c->stream);
        c->batch_graph_key.clear();   // a captured batch sequence may hold the old buffer
    }
    b.p = nullptr;
    b.bytes = 0;
    size_t want = bytes + bytes / 8;
    if (injected_failure(c)) return fail(HB_ERR_OOM, "device allocation of " + std::to_string(want) + " bytes failed (injected)");
    cudaError_t e = cudaMallocAsync(&b.p, want, c->stream);
    if (e != cudaSuccess) {
        cudaGetLastError();
        b.p = nullptr;
        return fail(HB_ERR_OOM, "device allocation of " + std::to_string(want) + " bytes failed");
    }
    b.bytes = want;
    return HB_OK;
}


void free_buf(hb_ctx *c, Buf &b) {
    if (b.p) cudaFreeAsync(b.p, c->stream);
    b.p = nullptr;
    b.bytes = 0;
}

static void free_side_encoding(hb_ctx *c, SideData &s) {
    if (s.rec) cudaFreeAsync(s.rec, c->stream);
    s.rec = nullptr;
    if (s.hot) cudaFreeAsync(s.hot, c->stream);
    s.hot = nullptr;
    for (auto g : s.grams)
        if (g) cudaFreeAsync(g, c->stream);
    s.grams.clear();
    s.gram_len.clear();
    s.encoded = false;
}

static void free_side(hb_ctx *c, SideData &s) {
    free_side_encoding(c, s);
    for (void *p : s.allocs) cudaFreeAsync(p, c->stream);
    s.allocs.clear();
    s.cols.clear();
    s.n = 0;
}

static void free_dicts(hb_ctx *c) {
    for (auto d : c->dict)
        if (d) cudaFreeAsync(d, c->stream);
    c->dict.clear();
    c->dict_cap.clear();
    for (auto &t : c->tok) {
        if (t.table) cudaFreeAsync(t.table, c->stream);
        if (t.start) cudaFreeAsync(t.start, c->stream);
        if (t.len) cudaFreeAsync(t.len, c->stream);
    }
    c->tok.clear();
}

static void invalidate_encoding(hb_ctx *c) {
    c->batch_graph_key.clear();
    free_side_encoding(c, c->side[0]);
    free_side_encoding(c, c->side[1]);
    free_dicts(c);
}

// checked builds: a site recorded by a device-side check fails the call
// (ordinary builds record nothing and return at once)
hb_status check_bounds(hb_ctx *c, const char *what) {
#ifdef HB_CHECKED
    HB_CUDA(cudaStreamSynchronize(c->stream));
    const unsigned int e = checked_error_eval(), n = checked_error_encode(), b = checked_error_block();
    const unsigned int site = e ? e : n ? n : b;
    if (site)
        return fail(HB_ERR_BOUNDS, std::string(what) + ": an index left its buffer at checked site " +
                                       std::to_string(site));
#else
    (void)c;
    (void)what;
#endif
    return HB_OK;
}

hb_status dmalloc(hb_ctx *c, void **p, size_t bytes) {
    if (bytes == 0) bytes = 16;
    if (injected_failure(c)) {
        *p = nullptr;
        return fail(HB_ERR_OOM, "device allocation of " + std::to_string(bytes) + " bytes failed (injected)");
    }
    cudaError_t e = cudaMallocAsync(p, bytes, c->stream);
    if (e != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        return fail(HB_ERR_OOM, "device allocation of " + std::to_string(bytes) + " bytes failed");
    }
    return HB_OK;
}

bool page_locked(const void *p) {
    cudaPointerAttributes at{};
    if (cudaPointerGetAttributes(&at, p) == cudaSuccess && at.type == cudaMemoryTypeHost) return true;
    cudaGetLastError();
    return false;
}

hb_status ensure_pinned(hb_ctx *c, size_t want) {
    if (c->pin_bytes >= want) return HB_OK;
    for (int b = 0; b < 2; b++) {
        if (c->pin[b]) {
            cudaEventSynchronize(c->pin_ev[b]);
            cudaFreeHost(c->pin[b]);
        }
        c->pin[b] = nullptr;
    }
    c->pin_bytes = 0;
    for (int b = 0; b < 2; b++) {
        if (injected_failure(c)) return fail(HB_ERR_OOM, "page-locked allocation failed (injected)");
        HB_CUDA(cudaMallocHost(&c->pin[b], want));
        if (!c->pin_ev[b]) HB_CUDA(cudaEventCreateWithFlags(&c->pin_ev[b], cudaEventDisableTiming));
    }
    c->pin_bytes = want;
    return HB_OK;
}

// host -> device.  A page-locked source (cudaMallocHost / cudaHostRegister)
// is copied by one DMA; the caller waits for it (sync_direct) before its
// buffer may change.  Pageable memory goes through the two pinned chunks: the
// copy of chunk i into pinned memory overlaps the DMA of chunk i-1.
hb_status upload(hb_ctx *c, void *dst, const void *src, size_t bytes) {
    if (bytes == 0) return HB_OK;
    if (page_locked(src)) {
        HB_CUDA(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, c->stream));
        c->direct_pending = true;
        return HB_OK;
    }
    HB_TRY(ensure_pinned(c, c->opt.chunk_bytes ? c->opt.chunk_bytes : (256ull << 20)));
    size_t off = 0;
    int i = 0;
    while (off < bytes) {
        const int b = i & 1;
        const size_t len = std::min(c->pin_bytes, bytes - off);
        HB_CUDA(cudaEventSynchronize(c->pin_ev[b]));
        memcpy(c->pin[b], static_cast<const char *>(src) + off, len);
        HB_CUDA(cudaMemcpyAsync(static_cast<char *>(dst) + off, c->pin[b], len, cudaMemcpyHostToDevice, c->stream));
        HB_CUDA(cudaEventRecord(c->pin_ev[b], c->stream));
        off += len;
        i++;
    }
    return HB_OK;
}

hb_status sync_direct(hb_ctx *c) {
    if (!c->direct_pending) return HB_OK;
    c->direct_pending = false;
    HB_CUDA(cudaStreamSynchronize(c->stream));
    return HB_OK;
}

// offsets of a string column must not decrease: bad[0] = the first row i with
// off[i + 1] < off[i] (0xFFFFFFFF when none)
__global__ void k_check_offsets(const uint32_t *off, int64_t n, unsigned int *bad) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        if (off[i + 1] < off[i]) atomicMin(bad, (unsigned int)i);
}

static hb_status copy_in(hb_ctx *c, void *dst, const void *src, size_t bytes, bool on_device) {
    if (bytes == 0) return HB_OK;
    if (on_device) {
        HB_CUDA(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToDevice, c->stream));
        return HB_OK;
    }
    return upload(c, dst, src, bytes);
}

}  // namespace hb

// ===================================================================== context
extern "C" const char *hb_last_error(void) { return g_err.c_str(); }
#ifdef HB_CHECKED
extern "C" const char *hb_version(void) { return "libhb 0.1 (sm_103a, checked)"; }
#else
extern "C" const char *hb_version(void) { return "libhb 0.1 (sm_103a)"; }
#endif

extern "C" hb_status hb_create(hb_ctx **out, const hb_options *opt) {
    if (!out) return fail(HB_ERR_ARG, "hb_create: out is NULL");
    *out = nullptr;
    hb_ctx *c = new (std::nothrow) hb_ctx();
    if (!c) return fail(HB_ERR_OOM, "hb_create: host allocation failed");
    if (opt) c->opt = *opt;
    if (c->opt.tile != 0 && c->opt.tile != 32 && c->opt.tile != 64) {
        delete c;
        return fail(HB_ERR_ARG, "hb_create: tile must be 0, 32 or 64");
    }
    c->device = c->opt.device;
    if (const char *inj = getenv("HB_FAIL_ALLOC_AFTER")) {
        char *end = nullptr;
        const long long v = strtoll(inj, &end, 10);
        if (end != inj && *end == 0 && v >= 0) c->fail_alloc_after = v;
    }
    cudaError_t e = cudaSetDevice(c->device);
    if (e != cudaSuccess) {
        delete c;
        return fail(HB_ERR_CUDA, std::string("hb_create: cudaSetDevice: ") + cudaGetErrorString(e));
    }
    cudaDeviceGetAttribute(&c->n_sm, cudaDevAttrMultiProcessorCount, c->device);
    if (c->opt.stream) {
        c->stream = static_cast<cudaStream_t>(c->opt.stream);
    } else {
        e = cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) {
            delete c;
            return fail(HB_ERR_CUDA, std::string("hb_create: stream: ") + cudaGetErrorString(e));
        }
        c->own_stream = true;
    }
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, c->device) == cudaSuccess) {
        uint64_t thr = UINT64_MAX;
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
    }
    c->stats.tile = 32;
    *out = c;
    return HB_OK;
}

extern "C" void hb_destroy(hb_ctx *c) {
    if (!c) return;
    cudaSetDevice(c->device);
    cudaStreamSynchronize(c->stream);
    free_side(c, c->side[0]);
    free_side(c, c->side[1]);
    free_dicts(c);
    Buf *bufs[] = {&c->w_slot_r, &c->w_slot_s, &c->w_count_s,
                   &c->w_start_s, &c->w_cursor, &c->w_members_r, &c->w_members_s, &c->w_blocks, &c->w_tiles,
                   &c->w_prefix, &c->w_scan, &c->w_out, &c->w_alt, &c->w_sort, &c->w_pairs, &c->w_counters,
                   &c->w_lut, &c->w_log, &c->w_jac, &c->w_jobrows, &c->w_jobcount, &c->w_joboff,
                   &c->w_small, &c->w_check};
    for (Buf *b : bufs) free_buf(c, *b);
    for (int b = 0; b < 2; b++) {
        free_buf(c, c->w_chunk[b]);
        if (c->chunk_copied[b]) cudaEventDestroy(c->chunk_copied[b]);
        if (c->chunk_consumed[b]) cudaEventDestroy(c->chunk_consumed[b]);
    }
    if (c->copy_stream) {
        cudaStreamSynchronize(c->copy_stream);
        cudaStreamDestroy(c->copy_stream);
    }
    for (hb_ctx::MdLane &L : c->md_lanes) {
        if (L.stream) cudaStreamSynchronize(L.stream);
        Buf *lb[] = {&L.table, &L.slot_r, &L.count_r, &L.start_r, &L.cursor, &L.slot_s, &L.count_s, &L.start_s,
                     &L.scan, &L.meta, &L.jac, &L.minrow};
        for (Buf *b : lb) free_buf(c, *b);
        if (L.done) cudaEventDestroy(L.done);
        if (L.stream) cudaStreamDestroy(L.stream);
    }
    if (c->md_fork) cudaEventDestroy(c->md_fork);
    if (c->batch_exec) cudaGraphExecDestroy(c->batch_exec);
    if (c->batch_graph) cudaGraphDestroy(c->batch_graph);
    cudaStreamSynchronize(c->stream);
    for (int b = 0; b < 2; b++) {
        if (c->pin[b]) cudaFreeHost(c->pin[b]);
        if (c->pin_ev[b]) cudaEventDestroy(c->pin_ev[b]);
    }
    if (c->own_stream) cudaStreamDestroy(c->stream);
    delete c;
}

// ===================================================================== tables
extern "C" hb_status hb_load_table(hb_ctx *c, int32_t side, int64_t n_rows, int32_t n_cols, const hb_column *cols,
                                   int32_t on_device) {
    if (!c) return fail(HB_ERR_ARG, "hb_load_table: ctx is NULL");
    if (side != 0 && side != 1) return fail(HB_ERR_ARG, "hb_load_table: side must be 0 (R) or 1 (S)");
    if (n_rows < 0 || n_rows >= (1ll << 30)) return fail(HB_ERR_ARG, "hb_load_table: n_rows must be in [0, 2^30)");
    if (n_cols < 0 || n_cols > 1024 || (n_cols > 0 && !cols)) return fail(HB_ERR_ARG, "hb_load_table: bad columns");
    cudaSetDevice(c->device);
    for (int k = 0; k < n_cols; k++) {
        const hb_column &col = cols[k];
        if (col.type < 0 || col.type > 2) return fail(HB_ERR_ARG, "hb_load_table: column " + std::to_string(k) + " has an unknown type");
        if (n_rows > 0 && !col.data && !(col.type == HB_COL_STRING && col.data_bytes == 0))
            return fail(HB_ERR_ARG, "hb_load_table: column " + std::to_string(k) + " has no data");
        if (col.type == HB_COL_STRING) {
            if (!col.offsets) return fail(HB_ERR_ARG, "hb_load_table: string column " + std::to_string(k) + " has no offsets");
            if (!on_device) {
                // the ends here; that the offsets never decrease is checked on the
                // device once they are there (k_check_offsets)
                if (col.offsets[0] != 0) return fail(HB_ERR_ARG, "hb_load_table: offsets[0] must be 0");
                if ((uint64_t)col.offsets[n_rows] != col.data_bytes)
                    return fail(HB_ERR_ARG, "hb_load_table: data_bytes != offsets[n] in column " + std::to_string(k));
            }
        }
    }
    SideData &S = c->side[side];
    free_side(c, S);
    invalidate_encoding(c);
    c->planned = false;
    S.n = n_rows;
    S.cols.resize(n_cols);
    const bool check = !on_device && n_cols > 0 && n_rows > 0;
    if (check) {
        HB_TRY(grow(c, c->w_check, sizeof(unsigned int) * (size_t)n_cols));
        HB_CUDA(cudaMemsetAsync(c->w_check.p, 0xFF, sizeof(unsigned int) * (size_t)n_cols, c->stream));
    }
    for (int k = 0; k < n_cols; k++) {
        const hb_column &col = cols[k];
        DevCol &d = S.cols[k];
        d.type = col.type;
        d.n = n_rows;
        void *p = nullptr;
        if (col.type == HB_COL_STRING) {
            d.nbytes = col.data_bytes;
            HB_TRY(dmalloc(c, &p, col.data_bytes + 16));
            S.allocs.push_back(p);
            d.bytes = static_cast<uint8_t *>(p);
            HB_TRY(copy_in(c, d.bytes, col.data, col.data_bytes, on_device));
            HB_TRY(dmalloc(c, &p, sizeof(uint32_t) * (n_rows + 1)));
            S.allocs.push_back(p);
            d.off = static_cast<uint32_t *>(p);
            HB_TRY(copy_in(c, d.off, col.offsets, sizeof(uint32_t) * (n_rows + 1), on_device));
            if (check) {
                HB_LAUNCHED(1);
                k_check_offsets<<<(unsigned)std::min<int64_t>((n_rows + 255) / 256, 4 * c->n_sm), 256, 0, c->stream>>>(
                    d.off, n_rows, as<unsigned int>(c->w_check) + k);
            }
        } else {
            HB_TRY(dmalloc(c, &p, 4 * (size_t)n_rows + 16));
            S.allocs.push_back(p);
            d.vals = p;
            HB_TRY(copy_in(c, d.vals, col.data, 4 * (size_t)n_rows, on_device));
        }
        if (col.valid) {
            HB_TRY(dmalloc(c, &p, (size_t)n_rows + 16));
            S.allocs.push_back(p);
            d.valid = static_cast<uint8_t *>(p);
            HB_TRY(copy_in(c, d.valid, col.valid, (size_t)n_rows, on_device));
        }
    }
    if (check) {
        std::vector<unsigned int> bad(n_cols);
        HB_CUDA(cudaMemcpyAsync(bad.data(), c->w_check.p, sizeof(unsigned int) * (size_t)n_cols, cudaMemcpyDeviceToHost,
                                c->stream));
        HB_CUDA(cudaStreamSynchronize(c->stream));
        c->direct_pending = false;
        for (int k = 0; k < n_cols; k++)
            if (bad[k] != 0xFFFFFFFFu) {
                free_side(c, S);
                S.n = 0;
                return fail(HB_ERR_ARG, "hb_load_table: offsets of column " + std::to_string(k) + " decrease at row " +
                                            std::to_string(bad[k]));
            }
    }
    HB_TRY(sync_direct(c));
    if (side == 0) c->stats.n_rows_r = n_rows;
    else c->stats.n_rows_s = n_rows;
    return HB_OK;
}

// ===================================================================== rules
static bool same_pred(const hb_predicate &a, const hb_predicate &b) {
    if (!(a.kind == b.kind && a.col_t == b.col_t && a.col_s == b.col_s && a.k == b.k && a.q == b.q &&
          a.num == b.num && a.den == b.den && a.delta == b.delta && a.side == b.side))
        return false;
    if (a.kind != HB_P_CONST_EQ) return true;
    return a.value_len == b.value_len && memcmp(a.value, b.value, a.value_len) == 0;
}

static hb_predicate normalize(hb_predicate p) {
    hb_predicate r{};
    r.kind = p.kind;
    r.col_t = p.col_t;
    r.col_s = p.col_s;
    switch (p.kind) {
    case HB_P_EQ_PREFIX: r.k = p.k; break;
    case HB_P_ED_LE: r.k = p.k; break;
    case HB_P_JACCARD_GE: {
        r.q = p.q;
        uint32_t g = std::gcd(p.num, p.den);
        if (g == 0) g = 1;
        r.num = p.num / g;
        r.den = p.den / g;
        break;
    }
    case HB_P_ABSDIFF_LE: r.delta = p.delta; break;
    case HB_P_CONTAIN_GE:
    case HB_P_TOKEN_JACCARD_GE: {
        r.q = p.kind == HB_P_CONTAIN_GE ? p.q : 0;
        r.side = p.kind == HB_P_CONTAIN_GE ? p.side : 0;
        uint32_t g = std::gcd(p.num, p.den);
        if (g == 0) g = 1;
        r.num = p.num / g;
        r.den = p.den / g;
        break;
    }
    case HB_P_CONST_EQ:
        r.side = p.side;
        r.value = p.value;
        r.value_len = p.value_len;
        if (p.side == 0) r.col_s = p.col_t;   // the constant's column, on the side it names
        else r.col_t = p.col_s;
        break;
    default: break;
    }
    return r;
}

extern "C" hb_status hb_add_md(hb_ctx *c, int32_t n_pred, const hb_predicate *preds, int32_t *md_id_out) {
    if (!c) return fail(HB_ERR_ARG, "hb_add_md: ctx is NULL");
    if (n_pred < 1 || n_pred > 10 || !preds) return fail(HB_ERR_ARG, "hb_add_md: an MD holds 1..10 predicates");
    if ((int)c->md_raw.size() >= HB_MAX_MDS) return fail(HB_ERR_ARG, "hb_add_md: at most 64 MDs");
    std::vector<hb_predicate> v;
    for (int i = 0; i < n_pred; i++) {
        const hb_predicate &p = preds[i];
        if (p.kind < 0 || p.kind > 7) return fail(HB_ERR_ARG, "hb_add_md: unknown predicate kind");
        if (p.col_t < 0 || p.col_s < 0) return fail(HB_ERR_ARG, "hb_add_md: negative column index");
        if (p.kind == HB_P_EQ_PREFIX && p.k < 1) return fail(HB_ERR_ARG, "hb_add_md: prefix length must be >= 1");
        if (p.kind == HB_P_ED_LE && (p.k < 0 || p.k > 31))
            return fail(HB_ERR_ARG, "hb_add_md: edit-distance threshold must be in [0, 31]");
        if (p.kind == HB_P_JACCARD_GE && (p.q < 1 || p.q > 4 || p.den < 1 || p.num > p.den))
            return fail(HB_ERR_ARG, "hb_add_md: Jaccard needs q in 1..4 and 0 <= num <= den, den >= 1");
        if (p.kind == HB_P_ABSDIFF_LE && !(p.delta >= 0.f))
            return fail(HB_ERR_ARG, "hb_add_md: |a-b| threshold must be >= 0");
        if (p.kind == HB_P_CONTAIN_GE && (p.q < 1 || p.q > 4 || p.den < 1 || p.num > p.den || p.side < 0 || p.side > 1))
            return fail(HB_ERR_ARG, "hb_add_md: containment needs q in 1..4, 0 <= num <= den, den >= 1, side 0 or 1");
        if (p.kind == HB_P_TOKEN_JACCARD_GE && (p.den < 1 || p.num > p.den))
            return fail(HB_ERR_ARG, "hb_add_md: token Jaccard needs 0 <= num <= den, den >= 1");
        if (p.kind == HB_P_CONST_EQ && (p.side < 0 || p.side > 1 || (p.value_len > 0 && !p.value)))
            return fail(HB_ERR_ARG, "hb_add_md: a constant needs side 0 or 1 and its bytes");
        hb_predicate n = normalize(p);
        if (p.kind == HB_P_CONST_EQ) {
            c->consts.emplace_back(static_cast<const char *>(p.value ? p.value : ""), (size_t)p.value_len);
            n.value = c->consts.back().data();
        }
        v.push_back(n);
    }
    c->md_raw.push_back(v);
    c->planned = false;
    invalidate_encoding(c);
    if (md_id_out) *md_id_out = (int32_t)c->md_raw.size() - 1;
    return HB_OK;
}

extern "C" hb_status hb_clear_mds(hb_ctx *c) {
    if (!c) return fail(HB_ERR_ARG, "hb_clear_mds: ctx is NULL");
    c->md_raw.clear();
    c->consts.clear();
    c->planned = false;
    invalidate_encoding(c);
    return HB_OK;
}

// ===================================================================== plan
namespace hb {

bool is_self(hb_ctx *c) { return c->side[1].cols.empty() && c->side[1].n == 0; }

static hb_status check_column(hb_ctx *c, int side, int col, int want_type, const char *what) {
    const SideData &S = c->side[side];
    if (col >= (int)S.cols.size())
        return fail(HB_ERR_ARG, std::string(what) + ": column " + std::to_string(col) + " does not exist in " +
                                    (side ? "S" : "R"));
    if (want_type >= 0 && S.cols[col].type != want_type)
        return fail(HB_ERR_ARG, std::string(what) + ": column " + std::to_string(col) + " has the wrong type");
    return HB_OK;
}

// A predicate whose verdict can change when the pair's two tuples exchange
// roles: a constant on one of them, containment, or two different columns.
static bool asymmetric(const hb_predicate &p) {
    return p.kind == HB_P_CONST_EQ || p.kind == HB_P_CONTAIN_GE || p.col_t != p.col_s;
}

// The MD with its two tuple variables exchanged: a self-join pair {i, j}
// (i < j) is a candidate when some MD is a witness at (t_i, t_j) or at
// (t_j, t_i), and an MD's witness at (t_j, t_i) is its transpose's at
// (t_i, t_j), so evaluating every MD and the transpose of every asymmetric
// one at (t_i, t_j) gives the self-join result.
static std::vector<hb_predicate> transpose(const std::vector<hb_predicate> &md) {
    std::vector<hb_predicate> out = md;
    for (hb_predicate &p : out) {
        std::swap(p.col_t, p.col_s);
        if (p.kind == HB_P_CONST_EQ || p.kind == HB_P_CONTAIN_GE) p.side ^= 1;
    }
    return out;
}

// distinct predicates, equality keys, feature groups and the record layout
static hb_status build_layout(hb_ctx *c, bool job_key) {
    const bool self = is_self(c);
    const int rs = self ? 0 : 1;
    c->preds.clear();
    c->md_preds.clear();
    c->eqkeys.clear();
    c->groups.clear();
    std::vector<std::vector<hb_predicate>> mds = c->md_raw;
    if (self) {
        const size_t n0 = mds.size();
        for (size_t m = 0; m < n0; m++) {
            bool asym = false;
            for (const hb_predicate &p : mds[m]) asym = asym || asymmetric(p);
            if (asym) mds.push_back(transpose(mds[m]));
        }
        if ((int)mds.size() > HB_MAX_MDS)
            return fail(HB_ERR_ARG, "at most 64 MDs, counting the transposed copy of each asymmetric MD");
    }
    c->n_user_mds = (int)c->md_raw.size();
    for (auto &md : mds) {
        std::vector<int> ids;
        for (auto &p : md) {
            if (self && p.col_t != p.col_s && p.kind != HB_P_EQ && p.kind != HB_P_CONST_EQ)
                return fail(HB_ERR_ARG, "in a self-join only equality compares two different columns (col_t != col_s)");
            const char *what = "predicate";
            switch (p.kind) {
            case HB_P_CONST_EQ: {
                const int sd = p.side == 0 ? 0 : rs, col = p.side == 0 ? p.col_t : p.col_s;
                HB_TRY(check_column(c, sd, col, -1, what));
                const int ty = c->side[sd].cols[col].type;
                if (ty == HB_COL_FP32 || (ty == HB_COL_INT32 && p.value_len != 4))
                    return fail(HB_ERR_ARG, "a constant compares a string column (value bytes) or an int32 column "
                                            "(4 value bytes)");
                break;
            }
            case HB_P_CONTAIN_GE:
            case HB_P_TOKEN_JACCARD_GE:
                HB_TRY(check_column(c, 0, p.col_t, HB_COL_STRING, what));
                HB_TRY(check_column(c, rs, p.col_s, HB_COL_STRING, what));
                break;
            case HB_P_EQ: {
                HB_TRY(check_column(c, 0, p.col_t, -1, what));
                HB_TRY(check_column(c, rs, p.col_s, -1, what));
                int tt = c->side[0].cols[p.col_t].type, ts = c->side[rs].cols[p.col_s].type;
                if (tt != ts || tt == HB_COL_FP32)
                    return fail(HB_ERR_ARG, "equality compares two string or two int32 columns");
                break;
            }
            case HB_P_EQ_PREFIX:
            case HB_P_ED_LE:
            case HB_P_JACCARD_GE:
                HB_TRY(check_column(c, 0, p.col_t, HB_COL_STRING, what));
                HB_TRY(check_column(c, rs, p.col_s, HB_COL_STRING, what));
                break;
            case HB_P_ABSDIFF_LE:
                HB_TRY(check_column(c, 0, p.col_t, HB_COL_FP32, what));
                HB_TRY(check_column(c, rs, p.col_s, HB_COL_FP32, what));
                break;
            }
            int id = -1;
            for (size_t k = 0; k < c->preds.size(); k++)
                if (same_pred(c->preds[k].p, p)) id = (int)k;
            if (id < 0) {
                if ((int)c->preds.size() >= HB_MAX_PREDS) return fail(HB_ERR_ARG, "too many distinct predicates");
                PredInfo pi;
                pi.p = p;
                id = (int)c->preds.size();
                c->preds.push_back(pi);
            }
            ids.push_back(id);
        }
        c->md_preds.push_back(ids);
    }
    // equality keys (in a self-join an equality across two columns is checked per pair instead)
    for (auto &pi : c->preds) {
        if (pi.p.kind != HB_P_EQ && pi.p.kind != HB_P_EQ_PREFIX) continue;
        if (self && pi.p.col_t != pi.p.col_s) continue;
        EqKey k{pi.p.col_t, pi.p.col_s, pi.p.kind == HB_P_EQ_PREFIX ? pi.p.k : -1};
        int e = -1;
        for (size_t j = 0; j < c->eqkeys.size(); j++)
            if (c->eqkeys[j].col_t == k.col_t && c->eqkeys[j].col_s == k.col_s && c->eqkeys[j].prefix == k.prefix)
                e = (int)j;
        if (e < 0) {
            e = (int)c->eqkeys.size();
            c->eqkeys.push_back(k);
        }
        pi.eq_index = e;
    }
    c->n_eq_total = (int)c->eqkeys.size() + (job_key ? 1 : 0);
    c->layout_part_m = c->part_m;
    if (c->part_m) {
        // Section 5.3 partitions: key e's partition under its hash function in
        // word n_eq + e, next to the exact codes (which the rules still test)
        if (job_key) return fail(HB_ERR_STATE, "partitioned blocking runs on hb_block / hb_block_device only");
        c->n_eq_total = 2 * (int)c->eqkeys.size();
        if (c->n_eq_total > MAX_EQ) return fail(HB_ERR_ARG, "at most 8 distinct equality keys when partitioned");
    }
    if (c->n_eq_total > MAX_EQ) return fail(HB_ERR_ARG, "at most 16 distinct equality keys");
    int word = c->n_eq_total;
    for (int pid = 0; pid < (int)c->preds.size(); pid++) {
        PredInfo &pi = c->preds[pid];
        if (pi.eq_index >= 0) continue;
        const hb_predicate &p = pi.p;
        int kind = OP_ABS, q = 0, tokens = 0, ct = p.col_t, cs = p.col_s;
        switch (p.kind) {
        case HB_P_ED_LE: kind = OP_ED; break;
        case HB_P_JACCARD_GE:
        case HB_P_CONTAIN_GE: kind = OP_JAC; q = p.q; break;   // containment reads the q-gram group
        case HB_P_TOKEN_JACCARD_GE: kind = OP_JAC; tokens = 1; break;
        case HB_P_EQ:   // two columns of one relation: codes of both in one dictionary
            kind = OP_EQX;
            ct = std::min(p.col_t, p.col_s);
            cs = std::max(p.col_t, p.col_s);
            break;
        case HB_P_CONST_EQ:   // a flag word per (side's column, constant)
            kind = OP_CONST;
            if (self) ct = cs = p.col_t;
            else if (p.side == 0) cs = -1;
            else ct = -1;
            break;
        default: break;
        }
        int g = -1;
        for (size_t j = 0; j < c->groups.size() && g < 0; j++) {
            const FeatGroup &G = c->groups[j];
            if (G.kind != kind || G.col_t != ct || G.col_s != cs || G.q != q || G.tokens != tokens) continue;
            if (kind == OP_CONST) {
                const hb_predicate &o = c->preds[G.pred].p;
                if (o.value_len != p.value_len || memcmp(o.value, p.value, p.value_len) != 0) continue;
            }
            g = (int)j;
        }
        if (g < 0) {
            FeatGroup G{kind, ct, cs, q, word};
            G.tokens = tokens;
            G.pred = pid;
            word += kind == OP_ED ? FEAT_ED_WORDS : kind == OP_JAC ? FEAT_JAC_WORDS : kind == OP_EQX ? 2 : 1;
            g = (int)c->groups.size();
            c->groups.push_back(G);
        }
        pi.group = g;
    }
    c->W = (word + 3) & ~3;
    c->HW = (c->n_eq_total + (int)c->groups.size() + 3) & ~3;
    if (c->HW > 64) return fail(HB_ERR_ARG, "too many distinct predicate columns");
    if (c->W > 252) return fail(HB_ERR_ARG, "record too wide: too many distinct predicate columns");
    // equality sets and the MDs that can own pairs
    const int n_md = (int)c->md_preds.size();
    c->eqset.assign(n_md, 0);
    c->eqonly = 0;
    for (int m = 0; m < n_md; m++) {
        uint16_t s = job_key ? (uint16_t)(1u << c->eqkeys.size()) : 0;   // (cross-column equalities are ops)
        bool has_other = false;
        for (int id : c->md_preds[m]) {
            if (c->preds[id].eq_index >= 0) s |= (uint16_t)(1u << c->preds[id].eq_index);
            else has_other = true;
        }
        c->eqset[m] = s;
        if (!has_other) c->eqonly |= 1ull << m;
    }
    c->active.clear();
    for (int m = 0; m < n_md; m++) {
        bool dominated = false;
        for (int j = 0; j < m; j++)
            if ((c->eqset[j] & c->eqset[m]) == c->eqset[j]) dominated = true;   // eqset_j subset of eqset_m
        if (!dominated) c->active.push_back(m);
    }
    c->lut.clear();
    if (c->n_eq_total <= LUT_MAX_EQ) {
        c->lut.assign((size_t)1 << c->n_eq_total, 0);
        for (uint32_t E = 0; E < c->lut.size(); E++)
            for (int m = 0; m < n_md; m++)
                if ((E & c->eqset[m]) == c->eqset[m]) c->lut[E] |= 1ull << m;
    }
    c->batch_layout = job_key;
    return HB_OK;
}

// Section 4.2 statistics: sp from LSH bucket counts on a sample, cost from an
// operation-count model over sampled string lengths.
static hb_status plan_stats(hb_ctx *c, std::vector<double> &sp, std::vector<double> &cost) {
    const int P = (int)c->preds.size();
    sp.assign(P, 1.0);
    cost.assign(P, 1.0);
    const SideData &R = c->side[0];
    if (P == 0 || R.n == 0) return HB_OK;
    const int K = 1024;
    const int n_samples = (int)std::min<int64_t>(R.n, 65536);
    const int n_keep = std::min(n_samples, 4096);
    std::vector<SampleSpec> specs(P);
    for (int p = 0; p < P; p++) {
        const hb_predicate &q = c->preds[p].p;
        // a constant on S's tuple (R x S) has no R column: its value distribution is not sampled
        const int ci = (q.kind == HB_P_CONST_EQ && q.side == 1 && !is_self(c)) ? 0 : q.col_t;
        const DevCol &col = R.cols[ci];
        SampleSpec s{};
        // sampled like the basic kind they resemble: constants and cross-column equality by value,
        // containment and word-token Jaccard by a MinHash over q-grams
        s.kind = q.kind == HB_P_CONST_EQ ? HB_P_EQ
                 : (q.kind == HB_P_CONTAIN_GE || q.kind == HB_P_TOKEN_JACCARD_GE) ? HB_P_JACCARD_GE : q.kind;
        s.type = col.type;
        s.bytes = col.bytes;
        s.off = col.off;
        s.vals = col.vals;
        s.valid = col.valid;
        s.prefix = q.kind == HB_P_EQ_PREFIX ? q.k : -1;
        s.q = (q.kind == HB_P_JACCARD_GE || q.kind == HB_P_CONTAIN_GE) ? q.q : 3;
        s.delta = q.delta;
        specs[p] = s;
    }
    Buf tmp;
    size_t bytes = sizeof(SampleSpec) * P + sizeof(uint32_t) * ((size_t)P * K + 2 * (size_t)P * n_keep) + 1024;
    HB_TRY(grow(c, tmp, bytes));
    char *base = static_cast<char *>(tmp.p);
    SampleSpec *d_specs = reinterpret_cast<SampleSpec *>(base);
    uint32_t *hist = reinterpret_cast<uint32_t *>(base + ((sizeof(SampleSpec) * P + 255) & ~size_t(255)));
    uint32_t *lens = hist + (size_t)P * K;
    uint32_t *grams = lens + (size_t)P * n_keep;
    HB_CUDA(cudaMemcpyAsync(d_specs, specs.data(), sizeof(SampleSpec) * P, cudaMemcpyHostToDevice, c->stream));
    HB_CUDA(cudaMemsetAsync(hist, 0, sizeof(uint32_t) * (size_t)P * K, c->stream));
    lsh_hist(d_specs, P, R.n, n_samples, K, hist, lens, grams, n_keep, c->stream);
    std::vector<uint32_t> h((size_t)P * K + 2 * (size_t)P * n_keep);
    HB_CUDA(cudaMemcpyAsync(h.data(), hist, sizeof(uint32_t) * h.size(), cudaMemcpyDeviceToHost, c->stream));
    HB_CUDA(cudaStreamSynchronize(c->stream));
    free_buf(c, tmp);
    std::vector<double> sd(P, 0.0);
    for (int p = 0; p < P; p++) {
        double n = 0;   // sampled values present: every one is in exactly one bucket
        for (int b = 0; b < K; b++) n += h[(size_t)p * K + b];
        double acc = 0;
        for (int b = 0; b < K; b++) {
            double d = h[(size_t)p * K + b] - n / K;
            acc += d * d;
        }
        sd[p] = std::sqrt(acc / K);
        // operation-count cost model (speed only)
        const hb_predicate &q = c->preds[p].p;
        double mlen = 0, mg = 0;
        int cnt = 0;
        for (int s = 0; s < n_keep; s++) {
            uint32_t L = h[(size_t)P * K + (size_t)p * n_keep + s];
            uint32_t G = h[(size_t)P * K + (size_t)P * n_keep + (size_t)p * n_keep + s];
            if (L == NULL_LEN) continue;
            mlen += L;
            mg += G;
            cnt++;
        }
        if (cnt) {
            mlen /= cnt;
            mg /= cnt;
        }
        switch (q.kind) {
        case HB_P_EQ:
        case HB_P_EQ_PREFIX: cost[p] = 1.0; break;
        case HB_P_ABSDIFF_LE: cost[p] = 2.0; break;
        case HB_P_ED_LE: cost[p] = 4.0 + 0.5 * mlen * (2.0 * q.k + 1.0); break;
        case HB_P_JACCARD_GE:
        case HB_P_CONTAIN_GE: cost[p] = 6.0 + 2.0 * mg; break;
        case HB_P_TOKEN_JACCARD_GE: cost[p] = 6.0 + 2.0 * (mlen / 6.0); break;
        case HB_P_CONST_EQ: cost[p] = 1.0; break;
        }
    }
    // the sampled lengths / gram counts stay for the learned cost model's
    // features, which are summarised only when asked for (ensure_pred_stats)
    c->stat_keep = n_keep;
    c->stat_lens.assign(h.begin() + (size_t)P * K + P, h.begin() + (size_t)P * K + P + (size_t)P * n_keep);
    c->stat_grams.assign(h.begin() + (size_t)P * K + P + (size_t)P * n_keep,
                         h.begin() + (size_t)P * K + P + 2 * (size_t)P * n_keep);
    c->stat_sd = sd;
    c->pred_stats.clear();
    double mx = 0, mc = 0;
    for (int p = 0; p < P; p++) {
        mx = std::max(mx, sd[p]);
        mc = std::max(mc, cost[p]);
    }
    for (int p = 0; p < P; p++) {
        sp[p] = mx > 0 ? std::max(sd[p] / mx, 1e-6) : 1e-6;
        cost[p] = mc > 0 ? std::max(cost[p] / mc, 1e-6) : 1e-6;
    }
    c->plain_sp = sp;
    c->plain_cost = cost;
    return HB_OK;
}

void ensure_pred_stats(hb_ctx *c) {
    const int P = (int)c->preds.size();
    const int n_keep = c->stat_keep;
    if ((int)c->pred_stats.size() == P || (int)c->stat_sd.size() != P) return;
    c->pred_stats.assign(P, std::vector<float>(10, 0.f));
    for (int p = 0; p < P; p++) {
        std::vector<double> Ls, Gs;
        int nulls = 0;
        for (int s = 0; s < n_keep; s++) {
            const uint32_t L = c->stat_lens[(size_t)p * n_keep + s];
            const uint32_t G = c->stat_grams[(size_t)p * n_keep + s];
            if (L == NULL_LEN) {
                nulls++;
                continue;
            }
            Ls.push_back(L);
            Gs.push_back(G);
        }
        std::vector<float> st(10, 0.f);
        if (!Ls.empty()) {
            std::sort(Ls.begin(), Ls.end());
            double m = 0, v = 0, gm = 0, gv = 0;
            for (double x : Ls) m += x;
            m /= Ls.size();
            for (double x : Ls) v += (x - m) * (x - m);
            for (double x : Gs) gm += x;
            gm /= Gs.size();
            for (double x : Gs) gv += (x - gm) * (x - gm);
            auto q = [&](double f) { return Ls[std::min(Ls.size() - 1, (size_t)(f * (Ls.size() - 1) + 0.5))]; };
            st = {(float)m, (float)std::sqrt(v / Ls.size()), (float)q(0.1), (float)q(0.5), (float)q(0.9),
                  (float)Ls.back(), (float)gm, (float)std::sqrt(gv / Gs.size()), 0.f, 0.f};
        }
        st[8] = n_keep ? (float)nulls / (float)n_keep : 0.f;
        st[9] = (float)c->stat_sd[p];
        c->pred_stats[p] = st;
    }
}

// Section 5.3 "Data partitioning": one hash function per child of the root
// of the execution tree, built from the predicate on that root edge.  The
// equality predicates of an MD are its block keys and head its path, so an
// MD's root edge is its first equality key in written order; an MD without
// one hangs from a similarity root, whose partitions may pull all others (the
// section's remark): that branch is one partition of all tuples.  Each branch
// becomes a grouping MD (after the rules' MDs) whose only key is the branch's
// partition word: the grouping MDs alone own pairs (the lowest branch that
// puts both tuples in one partition), and the program still tests every
// rule, so the result is the plain blocking result.
static hb_status add_partition_groups(hb_ctx *c) {
    const int n_md = (int)c->md_preds.size();
    const int n_eq = (int)c->eqkeys.size();
    c->branch_key.clear();
    c->branch_pred.clear();
    for (int m = 0; m < n_md; m++) {
        int key = -1, pred = -1;
        for (int id : c->md_preds[m])
            if (c->preds[id].eq_index >= 0) {
                key = c->preds[id].eq_index;
                pred = id;
                break;
            }
        bool seen = false;
        for (int k : c->branch_key) seen |= k == key;
        if (!seen) {
            c->branch_key.push_back(key);
            c->branch_pred.push_back(pred);
        }
    }
    const int nb = (int)c->branch_key.size();
    if (n_md + nb > MAX_MD) return fail(HB_ERR_ARG, "rules plus partition branches exceed 64");
    c->eqset.resize(n_md);
    c->group_mds = 0;
    c->active.clear();
    for (int b = 0; b < nb; b++) {
        const int k = c->branch_key[b];
        c->eqset.push_back(k >= 0 ? (uint16_t)(1u << (n_eq + k)) : (uint16_t)0);
        c->group_mds |= 1ull << (n_md + b);
        c->active.push_back(n_md + b);
    }
    c->lut.clear();
    if (c->n_eq_total <= LUT_MAX_EQ) {
        c->lut.assign((size_t)1 << c->n_eq_total, 0);
        for (uint32_t E = 0; E < c->lut.size(); E++)
            for (int m = 0; m < (int)c->eqset.size(); m++)
                if ((E & c->eqset[m]) == c->eqset[m]) c->lut[E] |= 1ull << m;
    }
    return HB_OK;
}

static hb_status finish_plan(hb_ctx *c, int mode, const std::vector<double> &sp, const std::vector<double> &cost) {
    const int P = (int)c->preds.size();
    const int n_md = (int)c->md_preds.size();
    std::vector<uint8_t> skip(P, 0);
    for (int p = 0; p < P; p++) skip[p] = c->preds[p].eq_index >= 0 ? 1 : 0;
    std::vector<int> program;
    std::vector<int> cp(n_md, -1);
    std::vector<int> md_order;
    if (mode == HB_PLAN_GIVEN_ORDER || mode == HB_PLAN_RANDOM) {
        std::vector<int> mds(n_md);
        std::iota(mds.begin(), mds.end(), 0);
        std::vector<std::vector<int>> order(n_md);
        for (int m = 0; m < n_md; m++) order[m] = c->md_preds[m];
        if (mode == HB_PLAN_RANDOM) {
            std::mt19937_64 rng(c->opt.seed ^ 0x5DEECE66Dull);
            std::shuffle(mds.begin(), mds.end(), rng);
            for (auto &o : order) std::shuffle(o.begin(), o.end(), rng);
        }
        std::vector<int> pos(P, -1);
        for (int m : mds) {
            md_order.push_back(m);
            for (int p : order[m])
                if (!skip[p] && pos[p] < 0) {
                    pos[p] = (int)program.size();
                    program.push_back(p);
                }
        }
        for (int m = 0; m < n_md; m++)
            for (int p : c->md_preds[m])
                if (pos[p] > cp[m]) cp[m] = pos[p];
    } else {
        PlanResult R = make_plan(P, sp.data(), cost.data(), c->md_preds, skip);
        program = R.program;
        cp = R.cp;
        md_order = R.md_order;
    }
    if ((int)program.size() > MAX_OPS) return fail(HB_ERR_ARG, "too many distinct non-equality predicates");
    c->program = program;
    c->ops.clear();
    for (size_t k = 0; k < program.size(); k++) {
        const PredInfo &pi = c->preds[program[k]];
        const FeatGroup &G = c->groups[pi.group];
        Op op{};
        op.kind = (uint8_t)(pi.p.kind == HB_P_CONTAIN_GE ? OP_CONT : G.kind);
        op.feat = (uint8_t)G.word;
        op.hot = (uint8_t)(c->n_eq_total + pi.group);
        op.k = (uint8_t)(pi.p.kind == HB_P_ED_LE ? pi.p.k : 0);
        op.num = pi.p.num;
        op.den = pi.p.den;
        op.delta = pi.p.delta;
        if (op.kind == OP_EQX) {   // t-side code word, s-side code word (the group holds min(col), max(col))
            const bool lo_first = pi.p.col_t <= pi.p.col_s;
            op.feat = (uint8_t)(G.word + (lo_first ? 0 : 1));
            op.k = (uint8_t)(G.word + (lo_first ? 1 : 0));
        } else if (op.kind == OP_CONST) {
            op.num = (uint32_t)pi.p.side;
        } else if (op.kind == OP_CONT) {
            op.k = (uint8_t)pi.p.side;
        }
        for (int m = 0; m < n_md; m++) {
            for (int p : c->md_preds[m])
                if (p == program[k]) op.need |= 1ull << m;
            if (cp[m] == (int)k) op.cp |= 1ull << m;
        }
        c->ops.push_back(op);
    }
    // hot record (what phases 1 and 1b of the evaluation read from shared
    // memory): the equality codes and the filter operand (length, gram count
    // or value) of each MD's first program predicate; then, while the record
    // stays within HOT_BUDGET words, the signature words of those predicates,
    // the filter operands of each MD's second predicate and their signatures
    // (MDs by decreasing estimated pass rate of their first predicate)
    c->hot_map.clear();
    for (int e = 0; e < c->n_eq_total; e++) c->hot_map.push_back(e);
    std::vector<int> hot_word(c->groups.size(), -1), hot_bins(c->groups.size(), -1);
    std::vector<std::array<int, 2>> mdops(n_md, std::array<int, 2>{-1, -1});
    for (int m = 0; m < n_md; m++) {
        int n = 0;
        for (size_t k = 0; k < c->ops.size() && n < 2; k++)
            if (c->ops[k].need & (1ull << m)) mdops[m][n++] = (int)k;
    }
    auto group_of = [&](int k) { return c->preds[program[k]].group; };
    // only edit distance, Jaccard and |a-b| have filter operands and screens
    auto screenable = [&](int k) { const int kd = c->ops[k].kind; return kd == OP_ED || kd == OP_JAC || kd == OP_ABS; };
    for (int m = 0; m < n_md; m++) {
        if (mdops[m][0] < 0 || !screenable(mdops[m][0])) continue;
        const int g = group_of(mdops[m][0]);
        if (hot_word[g] < 0) {
            hot_word[g] = (int)c->hot_map.size();
            c->hot_map.push_back(c->groups[g].word);
        }
    }
    // the signature words of a predicate: one for edit distance (8 character
    // bins), two for Jaccard (64-bit gram presence mask)
    auto add_bins = [&](int k) {
        const int g = group_of(k);
        const FeatGroup &G = c->groups[g];
        const int nb = !screenable(k) ? 0 : G.kind == OP_ED ? 1 : G.kind == OP_JAC ? 2 : 0;
        const int w0 = G.kind == OP_ED ? FEAT_ED_SIG : FEAT_JAC_MASK;
        if (nb == 0 || hot_word[g] < 0 || hot_bins[g] >= 0 || (int)c->hot_map.size() + nb > HOT_BUDGET) return;
        hot_bins[g] = (int)c->hot_map.size();
        for (int w = 0; w < nb; w++) c->hot_map.push_back(G.word + w0 + w);
    };
    // the optional words go first to the MDs whose first predicate lets the
    // most pairs through (largest estimated pass rate sp): their survivors
    // gain the most from a screen in shared memory
    std::vector<int> by_pass(n_md);
    std::iota(by_pass.begin(), by_pass.end(), 0);
    auto pass_of = [&](int m) { return (mdops[m][0] >= 0 && !sp.empty()) ? sp[program[mdops[m][0]]] : 0.0; };
    std::stable_sort(by_pass.begin(), by_pass.end(), [&](int x, int y) { return pass_of(x) > pass_of(y); });
    for (int m : by_pass)
        if (mdops[m][0] >= 0) add_bins(mdops[m][0]);
    for (int m : by_pass) {
        if (mdops[m][1] < 0 || !screenable(mdops[m][1])) continue;
        const int g = group_of(mdops[m][1]);
        if (hot_word[g] < 0 && (int)c->hot_map.size() + 1 <= HOT_BUDGET) {
            hot_word[g] = (int)c->hot_map.size();
            c->hot_map.push_back(c->groups[g].word);
        }
    }
    for (int m : by_pass)
        if (mdops[m][1] >= 0) add_bins(mdops[m][1]);
    while (c->hot_map.size() % 4) c->hot_map.push_back(-1);
    c->HW = (int)c->hot_map.size();
    for (size_t k = 0; k < c->ops.size(); k++) {
        const int g = group_of((int)k);
        c->ops[k].hot = (hot_word[g] < 0 || !screenable((int)k)) ? 255 : (uint8_t)hot_word[g];
        c->ops[k].hot2 = (hot_bins[g] < 0 || !screenable((int)k)) ? 255 : (uint8_t)hot_bins[g];
    }
    hb_plan_info &I = c->info;
    memset(&I, 0, sizeof(I));
    I.mode = mode;
    I.n_preds = P;
    I.n_ops = (int)program.size();
    I.n_eq = (int)c->eqkeys.size();
    I.n_mds = n_md;
    for (size_t k = 0; k < program.size(); k++) I.op_pred[k] = program[k];
    for (size_t k = 0; k < md_order.size() && k < HB_MAX_MDS; k++) I.md_order[k] = md_order[k];
    for (int p = 0; p < P; p++) {
        I.sp[p] = sp.empty() ? 0 : sp[p];
        I.cost[p] = cost.empty() ? 0 : cost[p];
        I.pred_md[p] = -1;
        for (int m = 0; m < n_md && I.pred_md[p] < 0; m++)
            for (int q : c->md_preds[m])
                if (q == p) I.pred_md[p] = m;
    }
    int tile = c->opt.tile ? c->opt.tile : 32;
    c->tile = tile;
    I.tile = tile;
    I.record_words = c->W;
    I.hot_words = c->HW;
    c->group_mds = 0;
    if (c->part_m) {
        HB_TRY(add_partition_groups(c));
        I.n_branches = (int32_t)c->branch_key.size();
        for (size_t b = 0; b < c->branch_pred.size() && b < HB_MAX_MDS; b++) I.branch_pred[b] = c->branch_pred[b];
    }
    c->planned = true;
    return HB_OK;
}


hb_status do_plan(hb_ctx *c, int mode, bool job_key) {
    if (c->md_raw.empty()) return fail(HB_ERR_STATE, "hb_plan: no MD added");
    if (c->side[0].cols.empty() && c->side[0].n == 0) return fail(HB_ERR_STATE, "hb_plan: relation R not loaded");
    if (mode < 0 || mode > 5) return fail(HB_ERR_ARG, "hb_plan: unknown mode");
    cudaSetDevice(c->device);
    auto t0 = std::chrono::steady_clock::now();
    bool relayout = !c->planned || c->batch_layout != job_key || c->preds.empty() || c->layout_part_m != c->part_m;
    if (relayout) {
        invalidate_encoding(c);
        HB_TRY(build_layout(c, job_key));
    }
    std::vector<double> sp, cost;
    HB_TRY(plan_stats(c, sp, cost));
    int applied = mode;
    if (mode == HB_PLAN_LEARNED) {
        // the features come from an instrumented run of a row sample, which
        // needs a program: the rule- and data-aware plan serves provisionally
        // (and stays when the model is missing or its output is unusable)
        HB_TRY(finish_plan(c, HB_PLAN_RULE_DATA, sp, cost));
        bool ok = false;
        std::vector<double> lsp = sp, lcost = cost;
        HB_TRY(learned_stats(c, lsp, lcost, ok));
        if (ok) {
            sp = lsp;
            cost = lcost;
        } else {
            applied = HB_PLAN_RULE_DATA;
        }
    } else if (mode == HB_PLAN_COST_FIRST) {
        for (auto &x : sp) x = 0.5;
    } else if (mode == HB_PLAN_SEL_FIRST) {
        for (auto &x : cost) x = 1.0;
    }
    HB_TRY(finish_plan(c, applied, sp, cost));
    c->info.mode = applied;
    auto t1 = std::chrono::steady_clock::now();
    c->stats.ms_plan = std::chrono::duration<double, std::milli>(t1 - t0).count();
    return HB_OK;
}

}  // namespace hb

extern "C" hb_status hb_set_partitions(hb_ctx *c, uint32_t m) {
    if (!c) return fail(HB_ERR_ARG, "hb_set_partitions: ctx is NULL");
    if (m > (1u << 31)) return fail(HB_ERR_ARG, "hb_set_partitions: m above 2^31");
    if (m != c->part_m) {
        c->part_m = m;
        c->planned = false;   // the record layout changes: plan (and encode) again
    }
    return HB_OK;
}

extern "C" hb_status hb_set_shard(hb_ctx *c, int32_t rank, int32_t world) {
    if (!c) return fail(HB_ERR_ARG, "hb_set_shard: ctx is NULL");
    if (world < 1 || rank < 0 || rank >= world) return fail(HB_ERR_ARG, "hb_set_shard: need 0 <= rank < world");
    c->shard_rank = (uint32_t)rank;
    c->shard_world = (uint32_t)world;
    return HB_OK;
}

extern "C" hb_status hb_merge_pairs(const hb_pair *const *lists, const int64_t *counts, int32_t k, hb_pair *out) {
    if (k < 0 || (k > 0 && (!lists || !counts))) return fail(HB_ERR_ARG, "hb_merge_pairs: lists or counts is NULL");
    int64_t total = 0;
    for (int32_t l = 0; l < k; l++) {
        if (counts[l] < 0 || (counts[l] > 0 && !lists[l])) return fail(HB_ERR_ARG, "hb_merge_pairs: bad list");
        total += counts[l];
    }
    if (total > 0 && !out) return fail(HB_ERR_ARG, "hb_merge_pairs: out is NULL");
    // a binary heap of (next pair, list) ordered by (tid1, tid2, list)
    auto key = [](const hb_pair &p) { return ((uint64_t)p.tid1 << 32) | (uint64_t)p.tid2; };
    std::vector<std::pair<uint64_t, int32_t>> heap;
    std::vector<int64_t> pos(k > 0 ? k : 1, 0);
    for (int32_t l = 0; l < k; l++)
        if (counts[l] > 0) heap.push_back({key(lists[l][0]), l});
    auto greater = [](const std::pair<uint64_t, int32_t> &a, const std::pair<uint64_t, int32_t> &b) { return a > b; };
    std::make_heap(heap.begin(), heap.end(), greater);
    int64_t o = 0;
    while (!heap.empty()) {
        std::pop_heap(heap.begin(), heap.end(), greater);
        const int32_t l = heap.back().second;
        heap.pop_back();
        out[o++] = lists[l][pos[l]++];
        if (pos[l] < counts[l]) {
            heap.push_back({key(lists[l][pos[l]]), l});
            std::push_heap(heap.begin(), heap.end(), greater);
        }
    }
    return HB_OK;
}

extern "C" hb_status hb_plan(hb_ctx *c, int32_t mode, hb_plan_info *info_out) {
    if (!c) return fail(HB_ERR_ARG, "hb_plan: ctx is NULL");
    HB_TRY(do_plan(c, mode, false));
    if (info_out) *info_out = c->info;
    return HB_OK;
}

// ===================================================================== encode
namespace hb {

__global__ void k_job_codes(const int64_t *job_rows, int n_jobs, int64_t n, uint32_t *rec, int W, int word) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int lo = 0, hi = n_jobs;   // job_rows[lo] <= i < job_rows[hi]
    while (hi - lo > 1) {
        int mid = (lo + hi) >> 1;
        if (job_rows[mid] <= i) lo = mid;
        else hi = mid;
    }
    rec[i * W + word] = (uint32_t)lo;
}

// Side streams of the context (created on first use): the encoder and the
// block builder run independent work on them, forked from and joined to the
// context's stream with events.
static hb_status ensure_lanes(hb_ctx *c, int lanes) {
    if ((int)c->md_lanes.size() < lanes) c->md_lanes.resize(lanes);
    if (!c->md_fork) HB_CUDA(cudaEventCreateWithFlags(&c->md_fork, cudaEventDisableTiming));
    for (int l = 0; l < lanes; l++) {
        hb_ctx::MdLane &L = c->md_lanes[l];
        if (!L.stream) HB_CUDA(cudaStreamCreateWithFlags(&L.stream, cudaStreamNonBlocking));
        if (!L.done) HB_CUDA(cudaEventCreateWithFlags(&L.done, cudaEventDisableTiming));
    }
    return HB_OK;
}

hb_status encode_side(hb_ctx *c, int side) {
    SideData &S = c->side[side];
    if (S.encoded && S.hot_map == c->hot_map) return HB_OK;
    c->batch_graph_key.clear();   // a captured batch sequence holds the old records
    if (S.encoded) {
        // a new plan staged other filter operands: repack the hot records only
        if (S.hot) cudaFreeAsync(S.hot, c->stream);
        S.hot = nullptr;
        S.encoded = false;   // until the repack is done
        void *q = nullptr;
        HB_TRY(dmalloc(c, &q, sizeof(uint32_t) * (size_t)c->HW * (size_t)(S.n > 0 ? S.n : 1) + 64));
        S.hot = static_cast<uint32_t *>(q);
        hot_pack(S.rec, c->W, S.n, S.hot, c->HW, c->hot_map.data(), c->stream);
        S.hot_map = c->hot_map;
        S.encoded = true;
        HB_CUDA(cudaGetLastError());
        return HB_OK;
    }
    free_side_encoding(c, S);   // whatever an earlier, failed encoding left
    const int64_t n = S.n;
    const int W = c->W;
    void *p = nullptr;
    HB_TRY(dmalloc(c, &p, sizeof(uint32_t) * (size_t)W * (size_t)(n > 0 ? n : 1) + 64));
    S.rec = static_cast<uint32_t *>(p);
    HB_CUDA(cudaMemsetAsync(S.rec, 0, sizeof(uint32_t) * (size_t)W * (size_t)(n > 0 ? n : 1), c->stream));
    // equality codes, written into the records
    if (side == 0) {
        free_dicts(c);
        c->dict.assign(c->eqkeys.size(), nullptr);
        c->dict_cap.assign(c->eqkeys.size(), 0);
    }
    // Independent encoding tasks (each equality key's dictionary, each edit-distance,
    // |a-b| and q-gram feature group) write disjoint words of the records; they
    // run below on up to MD_LANES side streams at once.  Their buffers are
    // allocated here on the context's stream, before the fork.
    struct EncTask {
        int kind;   // 0: equality key, 1: feature group
        size_t idx;
        double cost;
        int lane;
    };
    std::vector<EncTask> tasks;
    for (size_t e = 0; e < c->eqkeys.size(); e++) {
        const EqKey &k = c->eqkeys[e];
        if (side == 0) {
            uint64_t cap = pow2_at_least(std::max<uint64_t>(2 * (uint64_t)n, 1024));
            HB_TRY(dmalloc(c, &p, sizeof(uint64_t) * cap));
            c->dict[e] = static_cast<uint64_t *>(p);
            c->dict_cap[e] = cap;
        }
        const DevCol &col = S.cols[side == 0 ? k.col_t : k.col_s];
        tasks.push_back({0, e, (double)n + (col.type == HB_COL_STRING ? (double)col.nbytes : 0.0), 0});
    }
    // feature groups
    S.grams.assign(c->groups.size(), nullptr);
    S.gram_len.assign(c->groups.size(), 0);
    Buf flag;
    HB_TRY(grow(c, flag, 16));
    HB_CUDA(cudaMemsetAsync(flag.p, 0, 16, c->stream));
    for (size_t g = 0; g < c->groups.size(); g++) {
        const FeatGroup &G = c->groups[g];
        if (G.kind == OP_CONST) {
            // the flag word of the side the constant names (the other side's word stays 0)
            const int ci = side == 0 ? G.col_t : G.col_s;
            if (ci < 0) continue;
            const hb_predicate &q = c->preds[G.pred].p;
            Buf cv;
            HB_TRY(grow(c, cv, q.value_len + 8));
            HB_CUDA(cudaMemcpyAsync(cv.p, q.value, q.value_len, cudaMemcpyHostToDevice, c->stream));
            const_feature(S.cols[ci], as<uint8_t>(cv), q.value_len, S.rec, W, G.word, c->stream);
            HB_CUDA(cudaStreamSynchronize(c->stream));   // the constant's host bytes were read
            free_buf(c, cv);
            continue;
        }
        const DevCol &col = S.cols[side == 0 ? G.col_t : G.col_s];
        if (G.kind == OP_EQX) {
            // two columns of one relation (self-join): both coded in the first column's dictionary
            const DevCol &A = S.cols[G.col_t], &B = S.cols[G.col_s];
            const uint64_t cap = pow2_at_least(std::max<uint64_t>(2 * (uint64_t)n, 1024));
            Buf table;
            HB_TRY(grow(c, table, sizeof(uint64_t) * cap));
            dict_build(A, -1, as<uint64_t>(table), cap, S.rec + G.word, W, c->stream);
            dict_probe(B, -1, A, -1, as<uint64_t>(table), cap, S.rec + G.word + 1, W, c->stream);
            free_buf(c, table);
            continue;
        }
        if (G.kind == OP_JAC && G.tokens) {
            // word tokens: exact codes from R's token dictionary (S's tokens probe it), then per
            // string the sorted unique code list and its Jaccard feature words
            HB_TRY(grow(c, c->w_jac, tok_scratch_bytes(n)));
            Buf toff;
            HB_TRY(grow(c, toff, sizeof(uint32_t) * (size_t)(n + 2)));
            const int64_t T = tok_count(col, as<uint32_t>(toff), c->w_jac.p, c->w_jac.bytes, c->stream);
            if (T >= (1ll << 29)) return fail(HB_ERR_ARG, "more than 2^29 word tokens in a column");
            void *ts = nullptr, *tl = nullptr;
            HB_TRY(dmalloc(c, &ts, sizeof(uint32_t) * (size_t)(T + 1)));
            HB_TRY(dmalloc(c, &tl, sizeof(uint32_t) * (size_t)(T + 1)));
            HB_TRY(dmalloc(c, &p, sizeof(uint32_t) * (size_t)(T + 4)));
            S.grams[g] = static_cast<uint32_t *>(p);
            S.gram_len[g] = (uint64_t)T + 4;
            tok_fill(col, as<uint32_t>(toff), static_cast<uint32_t *>(ts), static_cast<uint32_t *>(tl), c->stream);
            if (c->tok.size() < c->groups.size()) c->tok.resize(c->groups.size());
            hb_ctx::TokDict &D = c->tok[g];
            if (side == 0) {
                D.cap = pow2_at_least(std::max<uint64_t>(2 * (uint64_t)T, 1024));
                void *tb = nullptr;
                HB_TRY(dmalloc(c, &tb, sizeof(uint64_t) * D.cap));
                D.table = static_cast<uint64_t *>(tb);
                D.start = static_cast<uint32_t *>(ts);
                D.len = static_cast<uint32_t *>(tl);
                D.bytes = col.bytes;
                tok_insert(col.bytes, D.start, D.len, T, D.table, D.cap, S.grams[g], c->stream);
            } else {
                if (!D.table) return fail(HB_ERR_STATE, "R's word tokens are not encoded");
                tok_probe(col.bytes, static_cast<uint32_t *>(ts), static_cast<uint32_t *>(tl), T, D.bytes, D.start,
                          D.len, D.table, D.cap, S.grams[g], c->stream);
            }
            tok_lists(col, as<uint32_t>(toff), static_cast<uint32_t *>(ts), static_cast<uint32_t *>(tl), S.grams[g],
                      S.rec, W, G.word, as<unsigned int>(flag), c->stream);
            if (side != 0) {
                cudaFreeAsync(ts, c->stream);
                cudaFreeAsync(tl, c->stream);
            }
            free_buf(c, toff);
            continue;
        }
        if (G.kind == OP_ED) {
            tasks.push_back({1, g, (double)col.nbytes, 0});
        } else if (G.kind == OP_ABS) {
            tasks.push_back({1, g, 0.5 * (double)n, 0});
        } else {
            HB_TRY(dmalloc(c, &p, sizeof(uint32_t) * (col.nbytes + 4)));
            S.grams[g] = static_cast<uint32_t *>(p);
            S.gram_len[g] = col.nbytes + 4;
            tasks.push_back({1, g, 4.0 * (double)col.nbytes + (double)n, 0});
        }
    }
    // longest first, each onto the least loaded lane
    const int lanes = std::min((int)tasks.size(), MD_LANES);
    std::sort(tasks.begin(), tasks.end(), [](const EncTask &a, const EncTask &b) { return a.cost > b.cost; });
    {
        double load[MD_LANES] = {0, 0, 0, 0};
        for (EncTask &t : tasks) {
            int best = 0;
            for (int l = 1; l < lanes; l++)
                if (load[l] < load[best]) best = l;
            t.lane = best;
            load[best] += t.cost;
        }
    }
    const bool forked = lanes >= 2;
    if (forked) {
        HB_TRY(ensure_lanes(c, lanes));
        for (const EncTask &t : tasks)
            if (t.kind == 1 && c->groups[t.idx].kind == OP_JAC)
                HB_TRY(grow(c, c->md_lanes[t.lane].jac, jac_scratch_bytes(n)));
        HB_CUDA(cudaEventRecord(c->md_fork, c->stream));
        for (int l = 0; l < lanes; l++) HB_CUDA(cudaStreamWaitEvent(c->md_lanes[l].stream, c->md_fork, 0));
    } else {
        for (const EncTask &t : tasks)
            if (t.kind == 1 && c->groups[t.idx].kind == OP_JAC) HB_TRY(grow(c, c->w_jac, jac_scratch_bytes(n)));
    }
    for (const EncTask &t : tasks) {
        cudaStream_t st = forked ? c->md_lanes[t.lane].stream : c->stream;
        if (t.kind == 0) {
            const size_t e = t.idx;
            const EqKey &k = c->eqkeys[e];
            if (side == 0)
                dict_build(S.cols[k.col_t], k.prefix, c->dict[e], c->dict_cap[e], S.rec + e, W, st);
            else
                dict_probe(S.cols[k.col_s], k.prefix, c->side[0].cols[k.col_t], k.prefix, c->dict[e],
                           c->dict_cap[e], S.rec + e, W, st);
            if (c->part_m)
                part_feature(S.cols[side == 0 ? k.col_t : k.col_s], k.prefix, c->part_m, S.rec, W,
                             (int)(c->eqkeys.size() + e), st);
            continue;
        }
        const size_t g = t.idx;
        const FeatGroup &G = c->groups[g];
        const DevCol &col = S.cols[side == 0 ? G.col_t : G.col_s];
        if (G.kind == OP_ED) {
            ed_features(col, S.rec, W, G.word, st);
        } else if (G.kind == OP_ABS) {
            abs_feature(col, S.rec, W, G.word, st);
        } else {
            void *scratch = forked ? c->md_lanes[t.lane].jac.p : c->w_jac.p;
            jac_features_impl(col, G.q, S.rec, W, G.word, S.grams[g], scratch, as<unsigned int>(flag), c->n_sm, st);
        }
    }
    if (forked) {
        for (int l = 0; l < lanes; l++) {
            HB_CUDA(cudaEventRecord(c->md_lanes[l].done, c->md_lanes[l].stream));
            HB_CUDA(cudaStreamWaitEvent(c->stream, c->md_lanes[l].done, 0));
        }
    }
    unsigned int too_long = 0;
    HB_CUDA(cudaMemcpyAsync(&too_long, flag.p, sizeof(unsigned int), cudaMemcpyDeviceToHost, c->stream));
    HB_CUDA(cudaStreamSynchronize(c->stream));
    free_buf(c, flag);
    HB_CUDA(cudaGetLastError());
    if (too_long) return fail(HB_ERR_ARG, "a string compared by Jaccard or containment has more than 8192 grams or tokens");
    if (c->batch_layout && side == 0) {
        // the job id is one more equality key held by every MD: blocks never span jobs
        const int n_jobs = (int)c->job_rows.size() - 1;
        if (n_jobs < 1 || c->job_rows.back() != n) return fail(HB_ERR_STATE, "batch layout without job rows");
        Buf jr;
        HB_TRY(grow(c, jr, sizeof(int64_t) * c->job_rows.size()));
        HB_CUDA(cudaMemcpyAsync(jr.p, c->job_rows.data(), sizeof(int64_t) * c->job_rows.size(),
                                cudaMemcpyHostToDevice, c->stream));
        if (n > 0) {
            HB_LAUNCHED(1);
            k_job_codes<<<(unsigned)((n + 255) / 256), 256, 0, c->stream>>>(as<int64_t>(jr), n_jobs, n, S.rec, W,
                                                                            c->n_eq_total - 1);
        }
        free_buf(c, jr);
    }
    {
        HB_TRY(dmalloc(c, &p, sizeof(uint32_t) * (size_t)c->HW * (size_t)(n > 0 ? n : 1) + 64));
        S.hot = static_cast<uint32_t *>(p);
        hot_pack(S.rec, W, n, S.hot, c->HW, c->hot_map.data(), c->stream);
        S.hot_map = c->hot_map;
        HB_CUDA(cudaGetLastError());
    }
    S.encoded = true;
    return HB_OK;
}

}  // namespace hb

// ===================================================================== blocking
namespace hb {


// counters layout (u64 words): 0 tile_counter, 1 out_count, 2 cand_count, 3 n_blocks (u32), 4 overflow (u32)
hb_status build_blocks(hb_ctx *c, const uint32_t *rec_r, int64_t n_r, const uint32_t *rec_s, int64_t n_s,
                              bool self, unsigned long long *ctr, uint32_t &block_cap) {
    const int W = c->W;
    const uint64_t H = pow2_at_least(std::max<uint64_t>(2 * (uint64_t)std::max<int64_t>(n_r, 1), 1024));
    const int na = (int)c->active.size();
    // member lists of all active MDs side by side, addressed with 32 bits
    if (!member_addressing_fits(na, std::max(n_r, n_s)))
        return fail(HB_ERR_ARG, "rows x active MDs exceed the 32-bit member addressing");
    const uint64_t per_md = self ? (uint64_t)(n_r / 2 + 1) : (uint64_t)std::min<int64_t>(n_r, n_s) + 1;
    const uint64_t bc = std::min<uint64_t>(per_md * (uint64_t)std::max(na, 1), 0xFFFFFFF0ull);
    block_cap = (uint32_t)bc;
    HB_TRY(grow(c, c->w_members_r, sizeof(uint32_t) * (size_t)std::max<int64_t>(n_r, 1) * std::max(na, 1)));
    if (!self)
        HB_TRY(grow(c, c->w_members_s, sizeof(uint32_t) * (size_t)std::max<int64_t>(n_s, 1) * std::max(na, 1)));
    HB_TRY(grow(c, c->w_blocks, sizeof(BlockDesc) * (size_t)bc));
    HB_TRY(grow(c, c->w_tiles, sizeof(uint64_t) * ((size_t)bc + 1)));
    HB_TRY(grow(c, c->w_prefix, sizeof(uint64_t) * ((size_t)bc + 1)));
    HB_TRY(grow(c, c->w_scan, scan_tmp_bytes((int64_t)bc + 1)));
    uint32_t *n_blocks = reinterpret_cast<uint32_t *>(ctr + 3);
    unsigned int *overflow = reinterpret_cast<unsigned int *>(ctr + 4);
    uint32_t *n_packed = reinterpret_cast<uint32_t *>(ctr + 6);
    uint32_t *small_total = reinterpret_cast<uint32_t *>(ctr + 7);
    if (self) HB_TRY(grow(c, c->w_small, sizeof(uint32_t) * (size_t)bc));
    // The MDs are independent: up to 4 lanes (side streams with scratch of their
    // own) build them at once, forked from and joined to the context's stream;
    // block descriptors, tile counts and small-block ranges are claimed with
    // atomics.  MD a runs on lane a % lanes.
    const int lanes = std::min(std::max(na, 1), MD_LANES);
    HB_TRY(ensure_lanes(c, lanes));
    for (int l = 0; l < lanes; l++) {
        hb_ctx::MdLane &L = c->md_lanes[l];
        HB_TRY(grow(c, L.table, sizeof(uint64_t) * H));
        HB_TRY(grow(c, L.slot_r, sizeof(uint32_t) * (size_t)(n_r + 1)));
        HB_TRY(grow(c, L.count_r, sizeof(uint32_t) * (H + 1)));
        HB_TRY(grow(c, L.start_r, sizeof(uint32_t) * (H + 1)));
        HB_TRY(grow(c, L.cursor, sizeof(uint32_t) * (H + 1)));
        HB_TRY(grow(c, L.scan, scan_tmp_bytes((int64_t)H + 1)));
        if (self) HB_TRY(grow(c, L.meta, sizeof(uint32_t) * SMALL_META_WORDS));
        if (c->shard_world > 1) HB_TRY(grow(c, L.minrow, sizeof(uint32_t) * (H + 1)));
        if (!self) {
            HB_TRY(grow(c, L.slot_s, sizeof(uint32_t) * (size_t)(n_s + 1)));
            HB_TRY(grow(c, L.count_s, sizeof(uint32_t) * (H + 1)));
            HB_TRY(grow(c, L.start_s, sizeof(uint32_t) * (H + 1)));
        }
    }
    HB_CUDA(cudaEventRecord(c->md_fork, c->stream));
    for (int l = 0; l < lanes; l++) HB_CUDA(cudaStreamWaitEvent(c->md_lanes[l].stream, c->md_fork, 0));
    for (int a = 0; a < na; a++) {
        const int m = c->active[a];
        hb_ctx::MdLane &L = c->md_lanes[a % lanes];
        cudaStream_t st = L.stream;
        int32_t words[MAX_EQ];
        int nk = 0;
        for (int e = 0; e < c->n_eq_total; e++)
            if (c->eqset[m] & (1u << e)) words[nk++] = e;
        group_build(rec_r, W, n_r, words, nk, as<uint64_t>(L.table), H, as<uint32_t>(L.slot_r), st);
        HB_CUDA(cudaMemsetAsync(L.count_r.p, 0, sizeof(uint32_t) * (H + 1), st));
        count_slots(as<uint32_t>(L.slot_r), n_r, as<uint32_t>(L.count_r), st);
        scan_exclusive_u32(as<uint32_t>(L.count_r), as<uint32_t>(L.start_r), (int64_t)H, nullptr, L.scan.p,
                           L.scan.bytes, st);
        HB_CUDA(cudaMemsetAsync(L.cursor.p, 0, sizeof(uint32_t) * (H + 1), st));
        uint32_t *mem_r = as<uint32_t>(c->w_members_r) + (size_t)a * (size_t)std::max<int64_t>(n_r, 1);
        scatter_slots(as<uint32_t>(L.slot_r), n_r, as<uint32_t>(L.start_r), as<uint32_t>(L.cursor), mem_r, st);
        if (self && c->shard_world > 1)
            shard_filter(as<uint32_t>(L.slot_r), n_r, as<uint32_t>(L.count_r), nullptr, as<uint32_t>(L.minrow), H,
                         (uint32_t)m, c->shard_rank, c->shard_world, st);
        if (self) {
            emit_blocks_packed(as<uint32_t>(L.count_r), as<uint32_t>(L.start_r), H, (uint32_t)m,
                               (uint32_t)((size_t)a * (size_t)std::max<int64_t>(n_r, 1)), c->tile,
                               as<BlockDesc>(c->w_blocks), as<uint64_t>(c->w_tiles), n_blocks, n_packed, block_cap,
                               overflow, as<uint32_t>(L.meta), as<uint32_t>(c->w_small), block_cap, small_total,
                               c->n_sm, st);
        } else {
            group_probe(rec_s, n_s, rec_r, W, words, nk, as<uint64_t>(L.table), H, as<uint32_t>(L.slot_s), st);
            HB_CUDA(cudaMemsetAsync(L.count_s.p, 0, sizeof(uint32_t) * (H + 1), st));
            count_slots(as<uint32_t>(L.slot_s), n_s, as<uint32_t>(L.count_s), st);
            scan_exclusive_u32(as<uint32_t>(L.count_s), as<uint32_t>(L.start_s), (int64_t)H, nullptr, L.scan.p,
                               L.scan.bytes, st);
            HB_CUDA(cudaMemsetAsync(L.cursor.p, 0, sizeof(uint32_t) * (H + 1), st));
            uint32_t *mem_s = as<uint32_t>(c->w_members_s) + (size_t)a * (size_t)std::max<int64_t>(n_s, 1);
            scatter_slots(as<uint32_t>(L.slot_s), n_s, as<uint32_t>(L.start_s), as<uint32_t>(L.cursor), mem_s, st);
            if (c->shard_world > 1)
                shard_filter(as<uint32_t>(L.slot_r), n_r, as<uint32_t>(L.count_r), as<uint32_t>(L.count_s),
                             as<uint32_t>(L.minrow), H, (uint32_t)m, c->shard_rank, c->shard_world, st);
            emit_blocks(as<uint32_t>(L.count_r), as<uint32_t>(L.start_r), as<uint32_t>(L.count_s),
                        as<uint32_t>(L.start_s), H, (uint32_t)m, 0,
                        (uint32_t)((size_t)a * (size_t)std::max<int64_t>(n_r, 1)),
                        (uint32_t)((size_t)a * (size_t)std::max<int64_t>(n_s, 1)), c->tile, as<BlockDesc>(c->w_blocks),
                        as<uint64_t>(c->w_tiles), n_blocks, block_cap, overflow, st);
        }
    }
    for (int l = 0; l < lanes; l++) {
        HB_CUDA(cudaEventRecord(c->md_lanes[l].done, c->md_lanes[l].stream));
        HB_CUDA(cudaStreamWaitEvent(c->stream, c->md_lanes[l].done, 0));
    }
    clamp_blocks(n_blocks, block_cap, c->stream);
    scan_exclusive_u64(as<uint64_t>(c->w_tiles), as<uint64_t>(c->w_prefix), (int64_t)bc, n_blocks, c->w_scan.p,
                       c->w_scan.bytes, c->stream);
    HB_CUDA(cudaGetLastError());
    return HB_OK;
}

EvalParams make_params(hb_ctx *c, const uint32_t *rec_r, const uint32_t *rec_s, int side_s, bool self,
                              unsigned long long *ctr, int key_bits_s) {
    EvalParams P;
    memset(&P, 0, sizeof(P));
    P.n_ops = (int)c->ops.size();
    P.n_eq = c->n_eq_total;
    P.W = c->W;
    P.HW = c->HW;
    P.hot_r = c->side[0].hot;
    P.hot_s = self ? c->side[0].hot : c->side[side_s].hot;
    for (int m = 0; m < MAX_MD; m++) P.first_op[m] = -1;
    for (int m = 0; m < (int)c->md_preds.size(); m++)
        for (int k = (int)c->ops.size() - 1; k >= 0; k--)
            if (c->ops[k].need & (1ull << m)) P.first_op[m] = (int8_t)k;
    const int n_all = (int)c->eqset.size();   // the rules' MDs, then any grouping MDs
    for (int m = 0; m < n_all; m++) {
        uint64_t base = 0;
        for (int j = 0; j < n_all; j++)
            if ((c->eqset[j] & ~c->eqset[m]) == 0) base |= 1ull << j;
        P.base_alive[m] = base;
        int nb = 0;
        bool filterable = (base & c->eqonly) == 0;
        for (int j = 0; j < n_all && filterable; j++) {
            if (!(base & (1ull << j))) continue;
            const int f = P.first_op[j];
            if (f < 0 || c->ops[f].hot == 255) {   // no staged filter operand: no phase-1 filter
                filterable = false;
                break;
            }
            bool seen = false;
            for (int i = 0; i < nb; i++) seen |= P.base_op[m][i] == f;
            if (seen) continue;
            if (nb == 4) filterable = false;
            else P.base_op[m][nb++] = (uint8_t)f;
        }
        P.base_nops[m] = filterable ? (uint8_t)nb : 255;
    }
    // the general phase 1: some active MD's blocks have 2..4 distinct base
    // filters or 4 varying equality keys
    P.keymask = c->n_eq_total >= 32 ? 0xffffffffu : ((1u << c->n_eq_total) - 1u);
    if (c->group_mds) {   // only the keys some MD holds: the rules' codes and the branches' partitions
        P.keymask = 0;
        for (uint16_t e : c->eqset) P.keymask |= e;
    }
    P.multi = 0;
    for (int m : c->active) {
        const int ko = __builtin_popcount(P.keymask & ~(unsigned)c->eqset[m]);
        P.multi |= ((P.base_nops[m] >= 2 && P.base_nops[m] <= 4) || ko == 4) ? 1 : 0;
    }
    memset(P.screen_op, 255, sizeof(P.screen_op));
    P.refine = 0;
    for (int m = 0; m < (int)c->md_preds.size(); m++) {
        int n = 0;
        for (size_t k = 0; k < c->ops.size() && n < 2; k++) {
            if (!(c->ops[k].need & (1ull << m))) continue;
            if (c->ops[k].hot != 255) {
                P.screen_op[m][n] = (uint8_t)k;
                // the screen adds to phase 1's filter only with a second
                // predicate or with bins in the hot record
                if (n == 1 || c->ops[k].hot2 != 255) P.refine = 1;
            }
            n++;
        }
    }
    P.self_join = self ? 1 : 0;
    P.n_md = (int)c->eqset.size();
    P.use_lut = c->lut.empty() ? 0 : 1;
    P.group_mds = c->group_mds;
    P.owner_mds = c->group_mds ? c->group_mds : ~0ull;

    P.tile = c->tile;
    P.key_bits_s = key_bits_s;
    P.eqonly = c->eqonly;
    for (int m = 0; m < P.n_md; m++) P.eqset[m] = c->eqset[m];
    for (size_t k = 0; k < c->ops.size(); k++) {
        P.ops[k] = c->ops[k];
        const PredInfo &pi = c->preds[c->program[k]];
        const FeatGroup &G = c->groups[pi.group];
        if (G.kind == OP_ED) {
            P.ptr_r[k] = c->side[0].cols[G.col_t].bytes;
            P.ptr_s[k] = self ? c->side[0].cols[G.col_t].bytes : c->side[side_s].cols[G.col_s].bytes;
            P.len_r[k] = c->side[0].cols[G.col_t].nbytes;
            P.len_s[k] = self ? P.len_r[k] : c->side[side_s].cols[G.col_s].nbytes;
        } else if (G.kind == OP_JAC) {   // q-gram or word-token code lists (Jaccard, containment)
            P.ptr_r[k] = c->side[0].grams[pi.group];
            P.ptr_s[k] = self ? c->side[0].grams[pi.group] : c->side[side_s].grams[pi.group];
            P.len_r[k] = c->side[0].gram_len[pi.group];
            P.len_s[k] = self ? P.len_r[k] : c->side[side_s].gram_len[pi.group];
        }
    }
    P.rec_r = rec_r;
    P.rec_s = rec_s;
    P.lut = P.use_lut ? as<uint64_t>(c->w_lut) : nullptr;
    P.members_r = as<uint32_t>(c->w_members_r);
    P.members_s = self ? as<uint32_t>(c->w_members_r) : as<uint32_t>(c->w_members_s);
    P.small = self ? as<uint32_t>(c->w_small) : nullptr;
    P.n_r = (uint64_t)c->side[0].n;
    P.n_s = self ? P.n_r : (uint64_t)c->side[side_s].n;
    P.members_r_len = c->w_members_r.bytes / 4;
    P.members_s_len = self ? P.members_r_len : c->w_members_s.bytes / 4;
    P.small_len = self ? c->w_small.bytes / 4 : 0;
    P.blocks = as<BlockDesc>(c->w_blocks);
    P.n_blocks = reinterpret_cast<const uint32_t *>(ctr + 3);
    P.tile_prefix = as<uint64_t>(c->w_prefix);
    P.tile_counter = ctr + 0;
    P.out = as<uint64_t>(c->w_out);
    P.out_count = ctr + 1;
    P.out_cap = (uint64_t)c->out_cap;
    P.cand_count = ctr + 2;
    P.exam_count = ctr + 5;
    P.claim = c->claim;
    P.log = as<unsigned long long>(c->w_log);
    return P;
}

hb_status ensure_ready(hb_ctx *c, bool job_key) {
    if (!c->planned || c->batch_layout != job_key) HB_TRY(do_plan(c, HB_PLAN_RULE_DATA, job_key));
    HB_TRY(encode_side(c, 0));
    if (!is_self(c)) HB_TRY(encode_side(c, 1));
    HB_TRY(grow(c, c->w_counters, 64 * sizeof(unsigned long long)));
    if (!c->lut.empty()) {
        HB_TRY(grow(c, c->w_lut, sizeof(uint64_t) * c->lut.size()));
        HB_CUDA(cudaMemcpyAsync(c->w_lut.p, c->lut.data(), sizeof(uint64_t) * c->lut.size(), cudaMemcpyHostToDevice,
                                c->stream));
    }
    HB_TRY(grow(c, c->w_log, sizeof(unsigned long long) * MAX_OPS * 8));
    return HB_OK;
}


// blocks -> evaluation -> sorted packed keys; result keys in *sorted, count in res
hb_status block_eval_sort(hb_ctx *c, const uint32_t *rec_r, int64_t n_r, const uint32_t *rec_s,
                                 int64_t n_s, bool self, int side_s, int key_bits, int key_bits_s, int logging,
                                 RunResult &res, uint64_t **sorted, Timer *tm) {
    unsigned long long *ctr = as<unsigned long long>(c->w_counters);
    HB_CUDA(cudaMemsetAsync(ctr, 0, 64 * sizeof(unsigned long long), c->stream));
    if (logging) HB_CUDA(cudaMemsetAsync(c->w_log.p, 0, sizeof(unsigned long long) * MAX_OPS * 8, c->stream));
    uint32_t block_cap = 0;
    HB_TRY(build_blocks(c, rec_r, n_r, rec_s, n_s, self, ctr, block_cap));
    if (tm) tm->mark();
    if (c->out_cap == 0) c->out_cap = c->opt.out_capacity > 0 ? c->opt.out_capacity : std::max<int64_t>(1 << 20, n_r);
    HB_TRY(grow(c, c->w_out, sizeof(uint64_t) * (size_t)c->out_cap));
    const size_t smem = eval_smem_bytes(c->HW, c->n_eq_total, c->lut.empty() ? 0 : 1, c->tile);
    int bps = eval_blocks_per_sm(c->tile, logging, smem);
    if (bps < 1) return fail(HB_ERR_ARG, "record too wide for the evaluation kernel's shared memory");
    const int grid = bps * c->n_sm;
    for (int attempt = 0; attempt < 2; attempt++) {
        EvalParams P = make_params(c, rec_r, rec_s, side_s, self, ctr, key_bits_s);
        P.profile = logging == 2 ? 1 : 0;   // 1: instrumented plan; 2: instrumented, no early exit
        HB_CUDA(launch_eval(P, grid, smem, logging ? 1 : 0, c->stream));
        if (tm && attempt == 0) tm->mark();
        unsigned long long h[8];
        HB_CUDA(cudaMemcpyAsync(h, ctr, sizeof(h), cudaMemcpyDeviceToHost, c->stream));
        HB_CUDA(cudaStreamSynchronize(c->stream));
        if (h[4]) return fail(HB_ERR_INTERNAL, "block list overflow");
        res.n_out = (int64_t)h[1];
        res.cand = (int64_t)h[2];
        res.blocks = (int64_t)(uint32_t)h[3];
        res.examined = (int64_t)h[5];
        res.real_blocks = res.blocks - (int64_t)(uint32_t)h[6] + (int64_t)(uint32_t)h[7];
        if (res.n_out <= c->out_cap) break;
        // the slab was too small: grow it to the exact count and evaluate again
        c->out_cap = res.n_out + res.n_out / 8 + 1024;
        HB_TRY(grow(c, c->w_out, sizeof(uint64_t) * (size_t)c->out_cap));
        HB_CUDA(cudaMemsetAsync(ctr, 0, 3 * sizeof(unsigned long long), c->stream));
        HB_CUDA(cudaMemsetAsync(ctr + 5, 0, sizeof(unsigned long long), c->stream));
        if (logging) HB_CUDA(cudaMemsetAsync(c->w_log.p, 0, sizeof(unsigned long long) * MAX_OPS * 8, c->stream));
    }
    {
        uint64_t t = 0;
        HB_CUDA(cudaMemcpyAsync(&t, as<uint64_t>(c->w_prefix) + res.blocks, sizeof(uint64_t), cudaMemcpyDeviceToHost,
                                c->stream));
        HB_CUDA(cudaStreamSynchronize(c->stream));
        res.tiles = (int64_t)t;
    }
    HB_TRY(grow(c, c->w_alt, sizeof(uint64_t) * (size_t)std::max<int64_t>(res.n_out, 1)));
    HB_TRY(grow(c, c->w_sort, radix_tmp_bytes(std::max<int64_t>(res.n_out, 1))));
    radix_sort_u64(as<uint64_t>(c->w_out), as<uint64_t>(c->w_alt), res.n_out, nullptr, key_bits, c->w_sort.p,
                   c->w_sort.bytes, c->stream, sorted);
    HB_CUDA(cudaGetLastError());
    if (tm) tm->mark();
    return HB_OK;
}

hb_status deliver(hb_ctx *c, const uint64_t *keys, int64_t n, int key_bits_s, bool to_host, hb_pair **out) {
    HB_TRY(grow(c, c->w_pairs, sizeof(hb_pair) * (size_t)std::max<int64_t>(n, 1)));
    pack_pairs(keys, n, key_bits_s, as<hb_pair>(c->w_pairs), c->stream);
    if (!to_host) {
        *out = as<hb_pair>(c->w_pairs);
        HB_CUDA(cudaStreamSynchronize(c->stream));
        return HB_OK;
    }
    hb_pair *h = static_cast<hb_pair *>(malloc(sizeof(hb_pair) * (size_t)std::max<int64_t>(n, 1)));
    if (!h) return fail(HB_ERR_OOM, "host allocation of the result failed");
    if (n > 0) {
        cudaError_t e = cudaMemcpyAsync(h, c->w_pairs.p, sizeof(hb_pair) * (size_t)n, cudaMemcpyDeviceToHost, c->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
        if (e != cudaSuccess) {
            free(h);
            return fail(HB_ERR_CUDA, std::string("result copy: ") + cudaGetErrorString(e));
        }
    }
    *out = h;
    return HB_OK;
}

static hb_status run_block(hb_ctx *c, hb_pair **out, int64_t *n_out, bool to_host) {
    if (!out || !n_out) return fail(HB_ERR_ARG, "hb_block: output pointers are NULL");
    *out = nullptr;
    *n_out = 0;
    if (c->side[0].cols.empty() && c->side[0].n == 0) return fail(HB_ERR_STATE, "hb_block: relation R not loaded");
    cudaSetDevice(c->device);
    auto w0 = std::chrono::steady_clock::now();
    Timer tm(c->stream);
    tm.mark();
    HB_TRY(ensure_ready(c, false));
    tm.mark();
    const bool self = is_self(c);
    const int64_t nr = c->side[0].n, ns = self ? nr : c->side[1].n;
    const int kbs = bits_for((uint64_t)std::max<int64_t>(ns, 2));
    const int kb = kbs + bits_for((uint64_t)std::max<int64_t>(nr, 2));
    RunResult res;
    uint64_t *sorted = nullptr;
    HB_TRY(block_eval_sort(c, c->side[0].rec, nr, self ? c->side[0].rec : c->side[1].rec, ns, self, 1, kb, kbs, 0,
                           res, &sorted, &tm));
    HB_TRY(check_bounds(c, "hb_block"));
    HB_TRY(deliver(c, sorted, res.n_out, kbs, to_host, out));
    tm.mark();
    HB_CUDA(cudaStreamSynchronize(c->stream));
    *n_out = res.n_out;
    hb_stats &S = c->stats;
    S.candidate_pairs = res.cand;
    S.emitted_pairs = res.n_out;
    S.tiles = res.tiles;
    S.blocks = res.real_blocks;
    S.examined_pairs = res.examined;
    S.ms_encode = tm.ms(0, 1);
    S.ms_block_build = tm.ms(1, 2);
    S.ms_eval = tm.ms(2, 3);
    S.ms_sort = tm.ms(3, 4);
    S.ms_d2h = tm.ms(4, 5);
    S.ms_total = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - w0).count();
    S.tile = c->tile;
    S.n_mds = (int)c->md_preds.size();
    return HB_OK;
}

}  // namespace hb

extern "C" hb_status hb_block(hb_ctx *c, hb_pair **pairs_out, int64_t *n_out) {
    if (!c) return fail(HB_ERR_ARG, "hb_block: ctx is NULL");
    return run_block(c, pairs_out, n_out, true);
}

extern "C" hb_status hb_block_device(hb_ctx *c, hb_pair **dev_pairs_out, int64_t *n_out) {
    if (!c) return fail(HB_ERR_ARG, "hb_block_device: ctx is NULL");
    return run_block(c, dev_pairs_out, n_out, false);
}

extern "C" void hb_free_pairs(hb_pair *pairs) { free(pairs); }

extern "C" hb_status hb_get_stats(const hb_ctx *c, hb_stats *out) {
    if (!c || !out) return fail(HB_ERR_ARG, "hb_get_stats: NULL argument");
    *out = c->stats;
    size_t tot = 0;
    for (int s = 0; s < 2; s++) {
        for (auto &col : c->side[s].cols) tot += col.nbytes + (col.off ? 4 * (col.n + 1) : 0) + (col.vals ? 4 * col.n : 0);
        if (c->side[s].rec) tot += (size_t)4 * c->W * c->side[s].n;
    }
    const Buf *bufs[] = {&c->w_slot_r, &c->w_slot_s, &c->w_count_s, &c->w_start_s, &c->w_cursor, &c->w_members_r,
                         &c->w_members_s, &c->w_blocks, &c->w_tiles, &c->w_prefix, &c->w_scan, &c->w_out,
                         &c->w_alt, &c->w_sort, &c->w_pairs, &c->w_small, &c->w_jac, &c->w_lut, &c->w_log,
                         &c->w_chunk[0], &c->w_chunk[1]};
    for (const Buf *b : bufs) tot += b->bytes;
    for (const hb_ctx::MdLane &L : c->md_lanes) {
        const Buf *lb[] = {&L.table, &L.slot_r, &L.count_r, &L.start_r, &L.cursor, &L.slot_s, &L.count_s,
                           &L.start_s, &L.scan, &L.meta, &L.jac, &L.minrow};
        for (const Buf *b : lb) tot += b->bytes;
    }
    out->device_bytes = (int64_t)tot;
    out->kernel_launches = (int64_t)g_kernel_launches.load();
    return HB_OK;
}
