// Columnar encoder: exact dictionary codes for equality keys, per-string
// features for edit distance and q-gram Jaccard, and the packed per-tuple
// record (array of structs, W 32-bit words) that the evaluation kernel stages.
#include <cuda_runtime.h>
#include <stdint.h>

#include "hb_internal.h"

namespace hb {
namespace {

constexpr int ENC_THREADS = 256;

__device__ __forceinline__ uint64_t mix64(uint64_t x) {
    x ^= x >> 33;
    x *= 0xff51afd7ed558ccdull;
    x ^= x >> 33;
    x *= 0xc4ceb9fe1a85ec53ull;
    x ^= x >> 33;
    return x;
}

__device__ __forceinline__ uint64_t hash_bytes(const uint8_t *p, uint32_t len) {
    uint64_t h = 0x9E3779B97F4A7C15ull ^ (uint64_t)len;
    uint32_t i = 0;
    for (; i + 4 <= len; i += 4) {
        uint32_t w = (uint32_t)p[i] | ((uint32_t)p[i + 1] << 8) | ((uint32_t)p[i + 2] << 16) |
                     ((uint32_t)p[i + 3] << 24);
        h = (h ^ w) * 0x100000001B3ull;
        h ^= h >> 29;
    }
    for (; i < len; i++) h = (h ^ p[i]) * 0x100000001B3ull;
    return mix64(h);
}

struct View {
    const uint8_t *bytes;
    const uint32_t *off;
    const int32_t *i32;
    const uint8_t *valid;
    int32_t type;
    int32_t prefix;
};

__host__ __device__ inline View make_view(const DevCol &c, int prefix) {
    View v;
    v.bytes = c.bytes;
    v.off = c.off;
    v.i32 = static_cast<const int32_t *>(c.vals);
    v.valid = c.valid;
    v.type = c.type;
    v.prefix = prefix;
    return v;
}

__device__ __forceinline__ void view_str(const View &v, int64_t i, const uint8_t *&p, uint32_t &len) {
    uint32_t a = v.off[i], b = v.off[i + 1];
    p = v.bytes + a;
    len = b - a;
    if (v.prefix >= 0 && len > (uint32_t)v.prefix) len = (uint32_t)v.prefix;
}

__device__ __forceinline__ uint64_t view_hash(const View &v, int64_t i) {
    if (v.type == HB_COL_STRING) {
        const uint8_t *p;
        uint32_t len;
        view_str(v, i, p, len);
        return hash_bytes(p, len);
    }
    return mix64((uint64_t)(uint32_t)v.i32[i] * 0x9E3779B97F4A7C15ull + 1);
}

__device__ __forceinline__ bool view_equal(const View &a, int64_t i, const View &b, int64_t j) {
    if (a.type == HB_COL_STRING) {
        const uint8_t *p, *q;
        uint32_t lp, lq;
        view_str(a, i, p, lp);
        view_str(b, j, q, lq);
        if (lp != lq) return false;
        for (uint32_t k = 0; k < lp; k++)
            if (p[k] != q[k]) return false;
        return true;
    }
    return a.i32[i] == b.i32[j];
}

// Insert every present value into an open-addressing table whose slots hold
// (32-bit hash << 32 | representative row); the code of a value is its slot.
// Two values share a slot only after a byte-exact comparison.
__global__ void k_dict_insert(View v, int64_t n, uint64_t *table, uint64_t mask, uint32_t *codes, int64_t stride) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    if (v.valid && !v.valid[i]) {
        codes[i * stride] = NULL_CODE;
        return;
    }
    uint64_t h = view_hash(v, i);
    uint32_t h32 = (uint32_t)(h >> 32);
    uint64_t mine = ((uint64_t)h32 << 32) | (uint64_t)(uint32_t)i;
    uint64_t slot = h & mask;
    for (uint64_t probe = 0; probe <= mask; probe++) {
        uint64_t cur = table[slot];
        if (cur == EMPTY_SLOT) {
            uint64_t prev = atomicCAS(reinterpret_cast<unsigned long long *>(table + slot),
                                      (unsigned long long)EMPTY_SLOT, (unsigned long long)mine);
            if (prev == EMPTY_SLOT) {
                codes[i * stride] = (uint32_t)slot;
                return;
            }
            cur = prev;
        }
        if ((uint32_t)(cur >> 32) == h32 && view_equal(v, i, v, (int64_t)(uint32_t)cur)) {
            codes[i * stride] = (uint32_t)slot;
            return;
        }
        slot = (slot + 1) & mask;
    }
    codes[i * stride] = NULL_CODE;   // unreachable: the table has at least twice as many slots as rows
}

// Codes for the other relation: the slot of an equal value of the owner, or NOMATCH.
__global__ void k_dict_probe(View v, int64_t n, View owner, const uint64_t *table, uint64_t mask, uint32_t *codes,
                             int64_t stride) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    if (v.valid && !v.valid[i]) {
        codes[i * stride] = NULL_CODE;
        return;
    }
    uint64_t h = view_hash(v, i);
    uint32_t h32 = (uint32_t)(h >> 32);
    uint64_t slot = h & mask;
    for (uint64_t probe = 0; probe <= mask; probe++) {
        uint64_t cur = table[slot];
        if (cur == EMPTY_SLOT) break;
        if ((uint32_t)(cur >> 32) == h32 && view_equal(v, i, owner, (int64_t)(uint32_t)cur)) {
            codes[i * stride] = (uint32_t)slot;
            return;
        }
        slot = (slot + 1) & mask;
    }
    codes[i * stride] = NOMATCH_CODE;
}

// Section 5.3 data partitioning: the partition of a row's value under one
// root-edge hash function, 32-bit FNV-1a (offset basis 2166136261, prime
// 16777619) of the value's bytes (a string's bytes or its prefix, an int32's
// four little-endian bytes) modulo m; a missing value is in no partition.
__global__ void k_part_key(View v, int64_t n, uint32_t m, uint32_t *rec, int W, int word) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    uint32_t out = NULL_CODE;
    if (!v.valid || v.valid[i]) {
        uint32_t h = 2166136261u;
        if (v.type == HB_COL_STRING) {
            const uint8_t *p;
            uint32_t len;
            view_str(v, i, p, len);
            for (uint32_t k = 0; k < len; k++) h = (h ^ p[k]) * 16777619u;
        } else {
            const uint32_t x = (uint32_t)v.i32[i];
            for (int k = 0; k < 4; k++) h = (h ^ ((x >> (8 * k)) & 255u)) * 16777619u;
        }
        out = h % m;
    }
    rec[i * W + word] = out;
}

// length, byte offset and 16 saturating 8-bit counts of (byte & 15)
__global__ void k_ed_features(const uint8_t *bytes, const uint32_t *off, const uint8_t *valid, int64_t n,
                              uint32_t *rec, int W, int feat) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    uint32_t *r = rec + i * W + feat;
    if (valid && !valid[i]) {
        r[0] = NULL_LEN;
        r[1] = 0;
        r[2] = r[3] = r[4] = r[5] = r[6] = 0;
        return;
    }
    uint32_t a = off[i], b = off[i + 1];
    uint32_t cnt[4] = {0, 0, 0, 0};
    uint32_t sig = 0;   // 8 nibbles: counts of bytes with (byte & 7) == nibble index, saturating at 15
    for (uint32_t k = a; k < b; k++) {
        const uint32_t by = bytes[k];
        uint32_t bin = by & 15u;
        uint32_t word = bin >> 2, sh = (bin & 3u) * 8u;
        uint32_t cur = (cnt[word] >> sh) & 255u;
        if (cur < 255u) cnt[word] += 1u << sh;
        const uint32_t ns = (by & 7u) * 4u;
        if (((sig >> ns) & 15u) < 15u) sig += 1u << ns;
    }
    r[0] = b - a;
    r[1] = a;
    r[2] = cnt[0];
    r[3] = cnt[1];
    r[4] = cnt[2];
    r[5] = cnt[3];
    r[FEAT_ED_SIG] = sig;
}

__global__ void k_abs_feature(const float *vals, const uint8_t *valid, int64_t n, uint32_t *rec, int W, int feat) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    rec[i * W + feat] = (valid && !valid[i]) ? 0x7FC00000u : __float_as_uint(vals[i]);
}

__device__ __forceinline__ uint32_t gram_at(const uint8_t *p, uint32_t k, int q) {
    uint32_t g = 0;
    for (int t = 0; t < q; t++) g = (g << 8) | p[k + t];
    return g;
}

__device__ __forceinline__ uint32_t gram_bin(uint32_t g) { return (g * 0x9E3779B1u) >> 27; }
// 6-bit hash bin of a gram for the 64-bit presence mask
__device__ __forceinline__ uint32_t gram_bit(uint32_t g) { return (g * 0x9E3779B1u) >> 26; }

constexpr int QG_MID = 256;        // grams per string handled by one warp
constexpr int QG_LONG_MAX = 8192;  // grams per string handled by one block

// Strings are handed to the sorting threads in order of their gram count
// (buckets 0..64, one more for longer strings), so that the threads of a warp
// sort lists of one length: the insertion sort's cost is then the average, not
// the warp's longest string.  The order only affects speed: every string
// writes its own output slot.
constexpr int QG_BUCKETS = 66;

__device__ __forceinline__ uint32_t gram_bucket(uint32_t g) { return g < 65u ? g : 65u; }

__global__ void k_gram_counts(const uint32_t *off, const uint8_t *valid, int64_t n, int q, uint32_t *cnt,
                              uint32_t *bucket_count) {
    __shared__ uint32_t h[QG_BUCKETS];
    for (int t = threadIdx.x; t < QG_BUCKETS; t += blockDim.x) h[t] = 0;
    __syncthreads();
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) {
        uint32_t len = off[i + 1] - off[i];
        const uint32_t g = (valid && !valid[i]) ? 0u : (len >= (uint32_t)q ? len - (uint32_t)q + 1u : 0u);
        cnt[i] = g;
        atomicAdd(&h[gram_bucket(g)], 1u);
    }
    __syncthreads();
    for (int t = threadIdx.x; t < QG_BUCKETS; t += blockDim.x)
        if (h[t]) atomicAdd(&bucket_count[t], h[t]);
}

// exclusive scan of the bucket counts (one warp)
__global__ void k_bucket_scan(const uint32_t *bucket_count, uint32_t *bucket_cursor) {
    const int lane = threadIdx.x;
    uint32_t carry = 0;
    for (int b0 = 0; b0 < QG_BUCKETS; b0 += 32) {
        const int b = b0 + lane;
        const uint32_t v = b < QG_BUCKETS ? bucket_count[b] : 0u;
        uint32_t incl = v;
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t u = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += u;
        }
        if (b < QG_BUCKETS) bucket_cursor[b] = carry + incl - v;
        carry += __shfl_sync(0xffffffffu, incl, 31);
    }
}

// ent[bucket start + rank] = (string, byte offset, length, first gram slot):
// a block reserves one range per bucket
__global__ void k_bucket_scatter(const uint32_t *cnt, const uint32_t *off, const uint32_t *gstart, int64_t n,
                                 uint32_t *bucket_cursor, uint4 *ent) {
    __shared__ uint32_t h[QG_BUCKETS], base[QG_BUCKETS];
    for (int t = threadIdx.x; t < QG_BUCKETS; t += blockDim.x) h[t] = 0;
    __syncthreads();
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    uint32_t b = 0, rank = 0;
    if (i < n) {
        b = gram_bucket(cnt[i]);
        rank = atomicAdd(&h[b], 1u);
    }
    __syncthreads();
    for (int t = threadIdx.x; t < QG_BUCKETS; t += blockDim.x)
        base[t] = h[t] ? atomicAdd(&bucket_cursor[t], h[t]) : 0u;
    __syncthreads();
    if (i < n) {
        const uint32_t a = off[i];
        ent[base[b] + rank] = make_uint4((uint32_t)i, a, off[i + 1] - a, gstart[i]);
    }
}

__device__ void write_gram_feature(uint32_t *r, uint32_t ucount, uint32_t start, const uint32_t *g) {
    uint32_t sig[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    for (uint32_t k = 0; k < ucount; k++) {
        uint32_t bin = gram_bin(g[k]);
        uint32_t word = bin >> 2, sh = (bin & 3u) * 8u;
        uint32_t cur = (sig[word] >> sh) & 255u;
        if (cur < 255u) sig[word] += 1u << sh;
    }
    uint64_t mask = 0;
    for (uint32_t k = 0; k < ucount; k++) mask |= 1ull << gram_bit(g[k]);
    r[0] = ucount;
    r[1] = start;
#pragma unroll
    for (int k = 0; k < 8; k++) r[2 + k] = sig[k];
    r[FEAT_JAC_MASK] = (uint32_t)mask;
    r[FEAT_JAC_MASK + 1] = (uint32_t)(mask >> 32);
}

// One string's grams sorted by a group of G lanes holding E grams each (up to
// E*G grams; E = 4 or 8): a bitonic network over the E*G elements, element
// e = E * (lane in group) + j.  Partners at a distance below E sit in the same
// lane (a compare-exchange in registers), farther ones in another lane of the
// group (a shuffle).  The unique grams are compacted (per-lane counts summed
// over the group with ballots of their bits) and written in order; their 32
// bin counts (at most 64 grams, so no 8-bit count saturates) and 64-bit
// presence mask are summed in the warp's shared words.  e is the string's entry
// (id, byte offset, length, first gram slot); a[0..2] are the lane's bytes
// E*gl .. E*gl+11 of the string, byte t of the window in byte t % 4 of a[t / 4]
// (loaded beforehand; bytes past the string's end are never part of a gram
// that is kept).  Gram j is bytes j .. j+q-1 of the window, the first byte
// most significant: one byte permutation (selector sel[j % 4]) of the word
// pair that holds it, masked to q bytes.
template <int G, int E>
__device__ __forceinline__ void grams_group(int q, uint32_t qmask, const uint32_t (&sel)[4], bool has, uint4 e,
                                            const uint32_t (&a)[3], uint32_t *grams, uint64_t gcap, uint32_t *rec,
                                            int W, int feat, uint32_t *acc) {
    const int lane = threadIdx.x & 31;
    const int gl = lane & (G - 1), gi = lane / G;
    const uint32_t i = e.x, gs = e.w;
    const uint32_t g = has ? e.z - (uint32_t)q + 1u : 0u;   // strings of this class have 1..E*G grams
    const uint32_t k0 = (uint32_t)(E * gl);
    uint32_t v[E];
#pragma unroll
    for (int j = 0; j < E; j++) {
        const uint32_t x = __byte_perm(a[j >> 2], a[(j >> 2) + 1], sel[j & 3]) & qmask;
        v[j] = k0 + j < g ? x : 0xFFFFFFFFu;
    }
#pragma unroll
    for (int size = 2; size <= E * G; size <<= 1) {
#pragma unroll
        for (int stride = size / 2; stride > 0; stride >>= 1) {
            if (stride < E) {
#pragma unroll
                for (int j = 0; j < E; j++) {
                    const int p = j ^ stride;
                    if (p > j) {
                        // direction from the element's bit `size`: within the lane below E, else the lane's
                        const bool up = size < E ? ((j & size) == 0) : ((k0 & (uint32_t)size) == 0u);
                        const uint32_t lo = min(v[j], v[p]), hi = max(v[j], v[p]);
                        v[j] = up ? lo : hi;
                        v[p] = up ? hi : lo;
                    }
                }
            } else {
                const int ls = stride / E;
                const bool up = (k0 & (uint32_t)size) == 0u;
                const bool keep_min = ((gl & ls) == 0) == up;
#pragma unroll
                for (int j = 0; j < E; j++) {
                    const uint32_t p = __shfl_xor_sync(0xffffffffu, v[j], ls);
                    v[j] = keep_min ? min(v[j], p) : max(v[j], p);
                }
            }
        }
    }
    // unique flags: an element differs from the one before it (lane gl-1's last for j = 0)
    const uint32_t prev = __shfl_up_sync(0xffffffffu, v[E - 1], 1);
    bool u[E];
    uint32_t cnt = 0;
#pragma unroll
    for (int j = 0; j < E; j++) {
        u[j] = k0 + j < g && (j > 0 ? v[j] != v[j - 1] : (gl == 0 || v[0] != prev));
        cnt += u[j] ? 1u : 0u;
    }
    // the group's exclusive prefix of the per-lane counts (0..E) from ballots of their bits
    const uint32_t gbits = (G == 32 ? 0xffffffffu : ((1u << G) - 1u)) << (gi * G);
    const uint32_t lower = gbits & ((1u << lane) - 1u);
    uint32_t pre = 0, ucount = 0;
    constexpr int CNT_BITS = E == 8 ? 4 : E == 4 ? 3 : 2;
#pragma unroll
    for (int b = 0; b < CNT_BITS; b++) {
        const uint32_t bal = __ballot_sync(0xffffffffu, (cnt >> b) & 1u);
        pre += (uint32_t)__popc(bal & lower) << b;
        ucount += (uint32_t)__popc(bal & gbits) << b;
    }
    uint32_t *sh = acc + gi * 10;
    for (int w = gl; w < 10; w += G) sh[w] = 0u;
    __syncwarp();
#pragma unroll
    for (int j = 0; j < E; j++) {
        if (u[j]) {
            grams[HB_IDX((uint64_t)gs + pre, gcap, 20)] = v[j];
            pre++;
            // feature words: 8 words of 32 8-bit bin counts, then the 64-bit mask
            const uint32_t bin = gram_bin(v[j]), bit = gram_bit(v[j]);
            atomicAdd(sh + (bin >> 2), 1u << ((bin & 3u) * 8u));
            atomicOr(sh + 8 + (bit >> 5), 1u << (bit & 31u));
        }
    }
    __syncwarp();
    if (has) {
        uint32_t *r = rec + (size_t)i * W + feat;
        for (int w = gl; w < FEAT_JAC_WORDS; w += G) r[w] = w == 0 ? ucount : w == 1 ? gs : sh[w - 2];
    }
    __syncwarp();
}

// Strings in bucket order (by gram count), in six classes: no grams (null or
// shorter than q; a thread each), 1-8, 9-16, 17-32 and 33-64 grams (groups of
// 2, 2, 4 and 8 lanes with 4, 8, 8 and 8 grams to a lane: 16, 16, 8 and 4
// strings per warp), and more than 64 grams (a thread each, handed to the
// per-warp and per-block kernels).  bucket_end[b] is the end of bucket b in the
// order.  Warps walk the classes' groups with a grid stride; the entries of the
// group two steps ahead and the bytes of the next are loaded before a group is
// sorted, so the two dependent loads of a string overlap the sorting.
constexpr int QG_COOP_THREADS = 256;

struct CoopStep {
    int c;          // class (-1: past the end)
    uint32_t pos;   // this lane's entry
    bool has;       // pos lies in the class
};

__device__ __forceinline__ CoopStep coop_step(uint32_t w, const uint32_t (&lo)[7], const uint32_t (&wstart)[7],
                                              int lane) {
    CoopStep st{-1, 0u, false};
    if (w >= wstart[6]) return st;
    int c = 0;
#pragma unroll
    for (int k = 1; k < 6; k++) c += w >= wstart[k] ? 1 : 0;
    uint32_t lo_c = 0, hi_c = 0, ws_c = 0;
#pragma unroll
    for (int k = 0; k < 6; k++)
        if (k == c) {
            lo_c = lo[k];
            hi_c = lo[k + 1];
            ws_c = wstart[k];
        }
    const uint32_t wc = w - ws_c;
    uint32_t pos;
    if (c == 0 || c == 5) pos = lo_c + wc * 32u + (uint32_t)lane;
    else if (c == 1 || c == 2) pos = lo_c + wc * 16u + (uint32_t)(lane >> 1);
    else if (c == 3) pos = lo_c + wc * 8u + (uint32_t)(lane >> 2);
    else pos = lo_c + wc * 4u + (uint32_t)(lane >> 3);
    st.c = c;
    st.pos = pos;
    st.has = pos < hi_c;
    return st;
}

__device__ __forceinline__ uint4 coop_entry(const CoopStep &st, const uint4 *ent) {
    return st.has ? ent[st.pos] : make_uint4(0u, 0u, 0u, 0u);
}

// the lane's 12-byte window E*gl .. E*gl+11 of its string (group classes only,
// lanes holding at least one gram): four aligned words from the column's byte
// array, shifted into place (byte arrays start 4-byte aligned and are padded
// by 16 bytes, so the words past a string's end stay in bounds)
__device__ __forceinline__ void coop_words(const CoopStep &st, uint4 e, const uint8_t *bytes, int q,
                                           uint32_t (&a)[3]) {
    const int lane = threadIdx.x & 31;
    const int G = st.c <= 2 ? 2 : st.c == 3 ? 4 : 8;
    const int E = st.c == 1 ? 4 : 8;
    const uint32_t k0 = (uint32_t)(E * (lane & (G - 1)));
    a[0] = a[1] = a[2] = 0u;
    if (st.has && st.c >= 1 && st.c <= 4 && k0 + (uint32_t)q <= e.z) {
        const uint32_t at = e.y + k0;
        const uint32_t *wp = reinterpret_cast<const uint32_t *>(bytes) + (at >> 2);
        const uint32_t w0 = __ldg(wp), w1 = __ldg(wp + 1), w2 = __ldg(wp + 2), w3 = __ldg(wp + 3);
        const uint32_t s = 8u * (at & 3u);
        a[0] = __funnelshift_r(w0, w1, s);
        a[1] = __funnelshift_r(w1, w2, s);
        a[2] = __funnelshift_r(w2, w3, s);
    }
}

__global__ void __launch_bounds__(QG_COOP_THREADS) k_grams_coop(const uint8_t *bytes, const uint8_t *valid, int64_t n,
                                                                int q, const uint4 *ent, const uint32_t *bucket_end,
                                                                uint32_t *grams, uint64_t gcap, uint32_t *rec, int W,
                                                                int feat, uint32_t *mid_list, unsigned int *n_mid,
                                                                uint32_t *long_list, unsigned int *n_long) {
    __shared__ uint32_t acc_all[QG_COOP_THREADS / 32][160];
    uint32_t *acc = acc_all[threadIdx.x >> 5];
    const int lane = threadIdx.x & 31;
    // byte selectors of a gram starting at window byte p (mod 4): result byte m
    // (m < q) = window byte p + q - 1 - m; the bytes from q up are masked off
    uint32_t sel[4];
#pragma unroll
    for (int p = 0; p < 4; p++) {
        uint32_t x = 0;
        for (int m = 0; m < q; m++) x |= (uint32_t)((p + q - 1 - m) & 7) << (4 * m);
        sel[p] = x;
    }
    const uint32_t qmask = q >= 4 ? 0xFFFFFFFFu : ((1u << (8 * q)) - 1u);
    // class c covers order positions [lo[c], lo[c+1]) and takes per[c] strings per warp
    uint32_t lo[7];
    lo[0] = 0;
    lo[1] = bucket_end[0];
    lo[2] = bucket_end[8];
    lo[3] = bucket_end[16];
    lo[4] = bucket_end[32];
    lo[5] = bucket_end[64];
    lo[6] = (uint32_t)n;
    const uint32_t per[6] = {32, 16, 16, 8, 4, 32};
    uint32_t wstart[7];
    wstart[0] = 0;
#pragma unroll
    for (int c = 0; c < 6; c++) wstart[c + 1] = wstart[c] + (lo[c + 1] - lo[c] + per[c] - 1) / per[c];
    const uint32_t nw = (uint32_t)((gridDim.x * blockDim.x) >> 5);
    uint32_t w = (uint32_t)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    CoopStep A = coop_step(w, lo, wstart, lane);
    uint4 eA = coop_entry(A, ent);
    CoopStep B = coop_step(w + nw, lo, wstart, lane);
    uint4 eB = coop_entry(B, ent);
    uint32_t bA[3];
    coop_words(A, eA, bytes, q, bA);
    while (A.c >= 0) {
        w += nw;
        const CoopStep C = coop_step(w + nw, lo, wstart, lane);
        const uint4 eC = coop_entry(C, ent);
        uint32_t bB[3];
        coop_words(B, eB, bytes, q, bB);
        if (A.c == 0) {
            if (A.has) {
                const uint32_t i = eA.x;
                uint32_t *r = rec + (size_t)i * W + feat;
                const bool null = valid && !valid[i];
                r[0] = null ? NULL_LEN : 0u;
                r[1] = null ? 0u : eA.w;
                for (int k = 2; k < FEAT_JAC_WORDS; k++) r[k] = 0u;
            }
        } else if (A.c == 5) {
            if (A.has) {
                const uint32_t g = eA.z - (uint32_t)q + 1u;
                if (g <= (uint32_t)QG_MID) mid_list[atomicAdd(n_mid, 1u)] = eA.x;
                else long_list[atomicAdd(n_long, 1u)] = eA.x;
            }
        } else if (A.c == 1) {
            grams_group<2, 4>(q, qmask, sel, A.has, eA, bA, grams, gcap, rec, W, feat, acc);
        } else if (A.c == 2) {
            grams_group<2, 8>(q, qmask, sel, A.has, eA, bA, grams, gcap, rec, W, feat, acc);
        } else if (A.c == 3) {
            grams_group<4, 8>(q, qmask, sel, A.has, eA, bA, grams, gcap, rec, W, feat, acc);
        } else {
            grams_group<8, 8>(q, qmask, sel, A.has, eA, bA, grams, gcap, rec, W, feat, acc);
        }
        A = B;
        eA = eB;
#pragma unroll
        for (int t = 0; t < 3; t++) bA[t] = bB[t];
        B = C;
        eB = eC;
    }
}

// Strings with 65..256 grams: one warp per string, bitonic sort in the warp's
// shared memory, the unique grams compacted with warp ballots and counted in
// 32 bins with shared-memory atomics.
__global__ void __launch_bounds__(256) k_grams_mid(const uint8_t *bytes, const uint32_t *off, int q,
                                                  const uint32_t *gstart, uint32_t *grams, uint64_t gcap, uint32_t *rec, int W,
                                                  int feat, const uint32_t *mid_list, const unsigned int *n_mid) {
    __shared__ uint32_t sm[8][QG_MID];
    __shared__ uint32_t bins[8][32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const unsigned lt = (1u << lane) - 1u;
    uint32_t *s = sm[w];
    const unsigned int nm = *n_mid;
    for (unsigned int li = blockIdx.x * 8u + (unsigned)w; li < nm; li += gridDim.x * 8u) {
        const int64_t i = mid_list[li];
        const uint32_t a = off[i], len = off[i + 1] - a;
        const uint32_t g = len - (uint32_t)q + 1u;   // 65 .. QG_MID
        const uint32_t P2 = g <= 128u ? 128u : 256u;
        const uint8_t *p = bytes + a;
        for (uint32_t k = lane; k < P2; k += 32) s[k] = k < g ? gram_at(p, k, q) : 0xFFFFFFFFu;
        bins[w][lane] = 0;
        __syncwarp();
        for (uint32_t size = 2; size <= P2; size <<= 1) {
            for (uint32_t stride = size >> 1; stride > 0; stride >>= 1) {
                for (uint32_t k = lane; k < P2; k += 32) {
                    const uint32_t partner = k ^ stride;
                    if (partner > k) {
                        const bool up = (k & size) == 0;
                        const uint32_t x = s[k], y = s[partner];
                        if ((x > y) == up) {
                            s[k] = y;
                            s[partner] = x;
                        }
                    }
                }
                __syncwarp();
            }
        }
        uint32_t *dst = grams + gstart[i];
        if (!HB_RANGE_OK(gstart[i], g, gcap, 21)) continue;
        uint32_t base = 0;
        uint64_t mask = 0;
        for (uint32_t c0 = 0; c0 < g; c0 += 32) {
            const uint32_t k = c0 + lane;
            const bool keep = k < g && (k == 0 || s[k] != s[k - 1]);
            const unsigned bal = __ballot_sync(0xffffffffu, keep);
            if (keep) {
                dst[base + __popc(bal & lt)] = s[k];
                atomicAdd(&bins[w][gram_bin(s[k])], 1u);
                mask |= 1ull << gram_bit(s[k]);
            }
            base += __popc(bal);
        }
        const uint32_t mlo = __reduce_or_sync(0xffffffffu, (uint32_t)mask);
        const uint32_t mhi = __reduce_or_sync(0xffffffffu, (uint32_t)(mask >> 32));
        __syncwarp();
        uint32_t *r = rec + i * W + feat;
        if (lane < 8) {
            uint32_t word = 0;
#pragma unroll
            for (int j = 0; j < 4; j++) word |= min(bins[w][4 * lane + j], 255u) << (8 * j);
            r[2 + lane] = word;
        }
        if (lane == 0) {
            r[0] = base;
            r[1] = gstart[i];
            r[FEAT_JAC_MASK] = mlo;
            r[FEAT_JAC_MASK + 1] = mhi;
        }
        __syncwarp();
    }
}

// Strings with more grams: one block per string, bitonic sort in shared memory.
__global__ void __launch_bounds__(256) k_grams_long(const uint8_t *bytes, const uint32_t *off, int q,
                                                   const uint32_t *gstart, uint32_t *grams, uint64_t gcap, uint32_t *rec, int W,
                                                   int feat, const uint32_t *long_list, const unsigned int *n_long,
                                                   unsigned int *too_long) {
    __shared__ uint32_t s[QG_LONG_MAX];
    __shared__ uint32_t wcount[8];
    const unsigned int nl = *n_long;
    for (unsigned int li = blockIdx.x; li < nl; li += gridDim.x) {
        const int64_t i = long_list[li];
        const uint32_t a = off[i], len = off[i + 1] - a;
        const uint32_t g = len - (uint32_t)q + 1u;
        uint32_t *r = rec + i * W + feat;
        if (g > (uint32_t)QG_LONG_MAX) {
            if (threadIdx.x == 0) {
                atomicExch(too_long, 1u);
                r[0] = NULL_LEN;
                r[1] = 0;
            }
            continue;
        }
        uint32_t P2 = 1;
        while (P2 < g) P2 <<= 1;
        const uint8_t *p = bytes + a;
        for (uint32_t k = threadIdx.x; k < P2; k += blockDim.x) s[k] = k < g ? gram_at(p, k, q) : 0xFFFFFFFFu;
        __syncthreads();
        for (uint32_t size = 2; size <= P2; size <<= 1) {
            for (uint32_t stride = size >> 1; stride > 0; stride >>= 1) {
                for (uint32_t k = threadIdx.x; k < P2; k += blockDim.x) {
                    uint32_t partner = k ^ stride;
                    if (partner > k) {
                        bool up = (k & size) == 0;
                        uint32_t x = s[k], y = s[partner];
                        if ((x > y) == up) {
                            s[k] = y;
                            s[partner] = x;
                        }
                    }
                }
                __syncthreads();
            }
        }
        // unique: a block-wide compaction in index order
        uint32_t *dst = grams + gstart[i];
        if (!HB_RANGE_OK(gstart[i], g, gcap, 22)) continue;
        uint32_t base = 0;
        for (uint32_t c0 = 0; c0 < g; c0 += blockDim.x) {
            uint32_t k = c0 + threadIdx.x;
            bool keep = k < g && (k == 0 || s[k] != s[k - 1]);
            unsigned bal = __ballot_sync(0xffffffffu, keep);
            int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
            if (lane == 0) wcount[w] = __popc(bal);
            __syncthreads();
            uint32_t before = 0, total = 0;
            for (int t = 0; t < (int)(blockDim.x >> 5); t++) {
                if (t < w) before += wcount[t];
                total += wcount[t];
            }
            if (keep) dst[base + before + __popc(bal & ((1u << lane) - 1u))] = s[k];
            base += total;
            __syncthreads();
        }
        if (threadIdx.x == 0) write_gram_feature(r, base, gstart[i], dst);
        __syncthreads();
    }
}

struct HotMap {
    int32_t w[64];
};

// A thread per (row, hot word): a block holds whole rows, so the hot records
// are written contiguously and each row's record is read by neighbouring lanes.
__global__ void k_hot_pack(const uint32_t *rec, int W, int64_t n, uint32_t *hot, int HW, HotMap map) {
    __shared__ int32_t m[64];
    if (threadIdx.x < 64) m[threadIdx.x] = map.w[threadIdx.x];
    __syncthreads();
    const int rpb = (int)blockDim.x / HW;
    const int lr = (int)threadIdx.x / HW, h = (int)threadIdx.x - lr * HW;
    const int64_t i = (int64_t)blockIdx.x * rpb + lr;
    if (lr >= rpb || i >= n) return;
    const int w = m[h];
    hot[i * HW + h] = w >= 0 ? rec[i * W + w] : 0u;
}

// ---- constants: one flag word per (column, constant) ----
__global__ void k_const_flag(View v, int64_t n, const uint8_t *cval, uint32_t clen, uint32_t *rec, int W, int feat) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    uint32_t f = 0;
    if (!v.valid || v.valid[i]) {
        if (v.type == HB_COL_STRING) {
            const uint8_t *p;
            uint32_t len;
            view_str(v, i, p, len);
            f = len == clen ? 1u : 0u;
            for (uint32_t k = 0; k < len && f; k++) f = p[k] == cval[k] ? 1u : 0u;
        } else {
            int32_t want = (int32_t)((uint32_t)cval[0] | ((uint32_t)cval[1] << 8) | ((uint32_t)cval[2] << 16) |
                                     ((uint32_t)cval[3] << 24));
            f = v.i32[i] == want ? 1u : 0u;
        }
    }
    rec[i * W + feat] = f;
}

// ---- word tokens: the maximal runs of bytes other than the space 0x20 ----
__global__ void k_tok_count(const uint8_t *bytes, const uint32_t *off, const uint8_t *valid, int64_t n,
                            uint32_t *cnt) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    uint32_t t = 0;
    if (!valid || valid[i]) {
        bool in = false;
        for (uint32_t k = off[i]; k < off[i + 1]; k++) {
            const bool word = bytes[k] != 0x20;
            t += (word && !in) ? 1u : 0u;
            in = word;
        }
    }
    cnt[i] = t;
}

__global__ void k_tok_fill(const uint8_t *bytes, const uint32_t *off, const uint8_t *valid, int64_t n,
                           const uint32_t *toff, uint32_t *tstart, uint32_t *tlen) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n || (valid && !valid[i])) return;
    uint32_t t = toff[i], k = off[i];
    const uint32_t e = off[i + 1];
    while (k < e) {
        while (k < e && bytes[k] == 0x20) k++;
        const uint32_t a = k;
        while (k < e && bytes[k] != 0x20) k++;
        if (k > a) {
            tstart[t] = a;
            tlen[t] = k - a;
            t++;
        }
    }
}

struct TokView {
    const uint8_t *bytes;
    const uint32_t *start, *len;
};

__device__ __forceinline__ bool tok_equal(const TokView &a, int64_t i, const TokView &b, int64_t j) {
    const uint32_t la = a.len[i];
    if (la != b.len[j]) return false;
    const uint8_t *p = a.bytes + a.start[i], *q = b.bytes + b.start[j];
    for (uint32_t k = 0; k < la; k++)
        if (p[k] != q[k]) return false;
    return true;
}

// exact token dictionary: slots hold (32-bit hash << 32 | representative token);
// a token's code is its slot (byte-exact comparison on equal hashes)
__global__ void k_tok_insert(TokView v, int64_t T, uint64_t *table, uint64_t mask, uint32_t *codes) {
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= T) return;
    const uint64_t h = hash_bytes(v.bytes + v.start[t], v.len[t]);
    const uint32_t h32 = (uint32_t)(h >> 32);
    const uint64_t mine = ((uint64_t)h32 << 32) | (uint64_t)(uint32_t)t;
    uint64_t slot = h & mask;
    for (uint64_t probe = 0; probe <= mask; probe++) {
        uint64_t cur = table[slot];
        if (cur == EMPTY_SLOT) {
            const uint64_t prev = atomicCAS(reinterpret_cast<unsigned long long *>(table + slot),
                                            (unsigned long long)EMPTY_SLOT, (unsigned long long)mine);
            if (prev == EMPTY_SLOT) {
                codes[t] = (uint32_t)slot;
                return;
            }
            cur = prev;
        }
        if ((uint32_t)(cur >> 32) == h32 && tok_equal(v, t, v, (int64_t)(uint32_t)cur)) {
            codes[t] = (uint32_t)slot;
            return;
        }
        slot = (slot + 1) & mask;
    }
    codes[t] = NOMATCH_CODE;   // unreachable: the table has at least twice as many slots as tokens
}

// the other relation's tokens: the slot of an equal token of the owner, or NOMATCH
__global__ void k_tok_probe(TokView v, int64_t T, TokView owner, const uint64_t *table, uint64_t mask,
                            uint32_t *codes) {
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= T) return;
    const uint64_t h = hash_bytes(v.bytes + v.start[t], v.len[t]);
    const uint32_t h32 = (uint32_t)(h >> 32);
    uint64_t slot = h & mask;
    for (uint64_t probe = 0; probe <= mask; probe++) {
        const uint64_t cur = table[slot];
        if (cur == EMPTY_SLOT) break;
        if ((uint32_t)(cur >> 32) == h32 && tok_equal(v, t, owner, (int64_t)(uint32_t)cur)) {
            codes[t] = (uint32_t)slot;
            return;
        }
        slot = (slot + 1) & mask;
    }
    codes[t] = NOMATCH_CODE;
}

// Per string: tokens that no owner token equals get codes local to the string
// (0x80000000 | position of the string's first equal token: such tokens meet
// no token of the other relation, so only their identity within the string
// matters), then the codes are sorted, made unique and summarised like q-grams.
__global__ void k_tok_lists(const uint8_t *bytes, const uint8_t *valid, int64_t n, const uint32_t *toff,
                            const uint32_t *tstart, const uint32_t *tlen, uint32_t *codes, uint32_t *rec, int W,
                            int feat, unsigned int *too_long) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    uint32_t *r = rec + i * W + feat;
    if (valid && !valid[i]) {
        r[0] = NULL_LEN;
        r[1] = 0;
        for (int k = 2; k < FEAT_JAC_WORDS; k++) r[k] = 0;
        return;
    }
    const uint32_t a = toff[i], b = toff[i + 1];
    if (b - a > 8192u) {
        atomicExch(too_long, 1u);
        r[0] = NULL_LEN;
        r[1] = 0;
        return;
    }
    TokView v{bytes, tstart, tlen};
    for (uint32_t t = a; t < b; t++) {
        if (codes[t] != NOMATCH_CODE) continue;
        uint32_t code = 0x80000000u | (t - a);
        for (uint32_t u = a; u < t; u++)
            if (codes[u] >= 0x80000000u && codes[u] != NOMATCH_CODE && tok_equal(v, t, v, u)) {
                code = codes[u];
                break;
            }
        codes[t] = code;
    }
    for (uint32_t t = a + 1; t < b; t++) {   // insertion sort (a string holds few tokens)
        const uint32_t x = codes[t];
        uint32_t u = t;
        while (u > a && codes[u - 1] > x) {
            codes[u] = codes[u - 1];
            u--;
        }
        codes[u] = x;
    }
    uint32_t m = a;
    for (uint32_t t = a; t < b; t++)
        if (t == a || codes[t] != codes[m - 1]) codes[m++] = codes[t];
    write_gram_feature(r, m - a, a, codes + a);
}

inline unsigned blocks_for(int64_t n, int t) { return (unsigned)((n + t - 1) / t > 0 ? (n + t - 1) / t : 1); }

}  // namespace

void dict_build(const DevCol &c, int prefix, uint64_t *table, uint64_t cap, uint32_t *codes, int64_t stride,
                cudaStream_t s) {
    cudaMemsetAsync(table, 0xFF, cap * sizeof(uint64_t), s);
    if (c.n == 0) return;
    HB_LAUNCHED(1);
    k_dict_insert<<<blocks_for(c.n, ENC_THREADS), ENC_THREADS, 0, s>>>(make_view(c, prefix), c.n, table, cap - 1,
                                                                      codes, stride);
}
void dict_probe(const DevCol &probe, int prefix, const DevCol &owner, int owner_prefix, const uint64_t *table,
                uint64_t cap, uint32_t *codes, int64_t stride, cudaStream_t s) {
    if (probe.n == 0) return;
    HB_LAUNCHED(1);
    k_dict_probe<<<blocks_for(probe.n, ENC_THREADS), ENC_THREADS, 0, s>>>(
        make_view(probe, prefix), probe.n, make_view(owner, owner_prefix), table, cap - 1, codes, stride);
}

void hot_pack(const uint32_t *rec, int W, int64_t n, uint32_t *hot, int HW, const int32_t *map, cudaStream_t s) {
    if (n == 0) return;
    HotMap m;
    for (int h = 0; h < 64; h++) m.w[h] = h < HW ? map[h] : -1;
    HB_LAUNCHED(1);
    const int rpb = HW >= ENC_THREADS ? 1 : ENC_THREADS / HW;   // rows per block
    k_hot_pack<<<(unsigned)((n + rpb - 1) / rpb), (unsigned)(rpb * HW), 0, s>>>(rec, W, n, hot, HW, m);
}

void part_feature(const DevCol &c, int prefix, uint32_t m, uint32_t *rec, int W, int word, cudaStream_t s) {
    if (c.n == 0) return;
    HB_LAUNCHED(1);
    k_part_key<<<blocks_for(c.n, ENC_THREADS), ENC_THREADS, 0, s>>>(make_view(c, prefix), c.n, m, rec, W, word);
}

void ed_features(const DevCol &c, uint32_t *rec, int W, int feat, cudaStream_t s) {
    if (c.n == 0) return;
    HB_LAUNCHED(1);
    k_ed_features<<<blocks_for(c.n, ENC_THREADS), ENC_THREADS, 0, s>>>(c.bytes, c.off, c.valid, c.n, rec, W, feat);
}

void const_feature(const DevCol &c, const uint8_t *cval_dev, uint32_t clen, uint32_t *rec, int W, int feat,
                   cudaStream_t s) {
    if (c.n == 0) return;
    HB_LAUNCHED(1);
    k_const_flag<<<blocks_for(c.n, ENC_THREADS), ENC_THREADS, 0, s>>>(make_view(c, -1), c.n, cval_dev, clen, rec, W,
                                                                     feat);
}

size_t tok_scratch_bytes(int64_t n) { return (size_t)(n + 1) * 4 + scan_tmp_bytes(n + 1) + 4096; }

int64_t tok_count(const DevCol &c, uint32_t *toff, void *scratch, size_t scratch_bytes, cudaStream_t s) {
    if (c.n == 0) return 0;
    uint32_t *cnt = static_cast<uint32_t *>(scratch);
    void *tmp = static_cast<char *>(scratch) + (((size_t)(c.n + 1) * 4 + 255) & ~(size_t)255);
    HB_LAUNCHED(1);
    k_tok_count<<<blocks_for(c.n, ENC_THREADS), ENC_THREADS, 0, s>>>(c.bytes, c.off, c.valid, c.n, cnt);
    cudaMemsetAsync(cnt + c.n, 0, 4, s);
    scan_exclusive_u32(cnt, toff, c.n + 1, nullptr, tmp, scratch_bytes - (((size_t)(c.n + 1) * 4 + 255) & ~(size_t)255), s);
    uint32_t total = 0;
    cudaMemcpyAsync(&total, toff + c.n, 4, cudaMemcpyDeviceToHost, s);
    cudaStreamSynchronize(s);
    return (int64_t)total;
}

void tok_fill(const DevCol &c, const uint32_t *toff, uint32_t *tstart, uint32_t *tlen, cudaStream_t s) {
    if (c.n == 0) return;
    HB_LAUNCHED(1);
    k_tok_fill<<<blocks_for(c.n, ENC_THREADS), ENC_THREADS, 0, s>>>(c.bytes, c.off, c.valid, c.n, toff, tstart, tlen);
}

void tok_insert(const uint8_t *bytes, const uint32_t *tstart, const uint32_t *tlen, int64_t T, uint64_t *table,
                uint64_t cap, uint32_t *codes, cudaStream_t s) {
    cudaMemsetAsync(table, 0xFF, cap * sizeof(uint64_t), s);
    if (T == 0) return;
    HB_LAUNCHED(1);
    k_tok_insert<<<blocks_for(T, ENC_THREADS), ENC_THREADS, 0, s>>>(TokView{bytes, tstart, tlen}, T, table, cap - 1,
                                                                   codes);
}

void tok_probe(const uint8_t *bytes, const uint32_t *tstart, const uint32_t *tlen, int64_t T, const uint8_t *obytes,
               const uint32_t *ostart, const uint32_t *olen, const uint64_t *table, uint64_t cap, uint32_t *codes,
               cudaStream_t s) {
    if (T == 0) return;
    HB_LAUNCHED(1);
    k_tok_probe<<<blocks_for(T, ENC_THREADS), ENC_THREADS, 0, s>>>(TokView{bytes, tstart, tlen}, T,
                                                                  TokView{obytes, ostart, olen}, table, cap - 1, codes);
}

void tok_lists(const DevCol &c, const uint32_t *toff, const uint32_t *tstart, const uint32_t *tlen, uint32_t *codes,
               uint32_t *rec, int W, int feat, unsigned int *too_long, cudaStream_t s) {
    if (c.n == 0) return;
    HB_LAUNCHED(1);
    k_tok_lists<<<blocks_for(c.n, 128), 128, 0, s>>>(c.bytes, c.valid, c.n, toff, tstart, tlen, codes, rec, W, feat,
                                                    too_long);
}

void abs_feature(const DevCol &c, uint32_t *rec, int W, int feat, cudaStream_t s) {
    if (c.n == 0) return;
    HB_LAUNCHED(1);
    k_abs_feature<<<blocks_for(c.n, ENC_THREADS), ENC_THREADS, 0, s>>>(static_cast<const float *>(c.vals), c.valid,
                                                                      c.n, rec, W, feat);
}

size_t jac_scratch_bytes(int64_t n) {
    return (size_t)(n + 1) * 4 * 4 + (size_t)(n + 1) * 16 + 16 + 2 * QG_BUCKETS * 4 + scan_tmp_bytes(n) + 4096;
}

// scratch: jac_scratch_bytes(n); grams: capacity >= nbytes of the column (one gram per byte at most)
void jac_features_impl(const DevCol &c, int q, uint32_t *rec, int W, int feat, uint32_t *grams, void *scratch,
                       unsigned int *too_long, int n_sm, cudaStream_t s) {
    const int64_t n = c.n;
    if (n == 0) return;
    uint32_t *cnt = static_cast<uint32_t *>(scratch);
    uint32_t *gstart = cnt + (n + 1);
    uint32_t *long_list = gstart + (n + 1);
    uint32_t *mid_list = long_list + (n + 1);
    uint4 *ent = reinterpret_cast<uint4 *>((reinterpret_cast<uintptr_t>(mid_list + (n + 1)) + 15) & ~uintptr_t(15));
    uint32_t *bucket_count = reinterpret_cast<uint32_t *>(ent + (n + 1));
    uint32_t *bucket_cursor = bucket_count + QG_BUCKETS;
    unsigned int *n_long = bucket_cursor + QG_BUCKETS;
    unsigned int *n_mid = n_long + 1;
    void *stmp = reinterpret_cast<void *>((reinterpret_cast<uintptr_t>(n_long + 4) + 255) & ~uintptr_t(255));
    // n_long, n_mid and the bucket counts are zeroed together
    cudaMemsetAsync(bucket_count, 0, sizeof(uint32_t) * (2 * QG_BUCKETS + 2), s);
    HB_LAUNCHED(4);
    k_gram_counts<<<blocks_for(n, ENC_THREADS), ENC_THREADS, 0, s>>>(c.off, c.valid, n, q, cnt, bucket_count);
    scan_exclusive_u32(cnt, gstart, n, nullptr, stmp, 0, s);
    k_bucket_scan<<<1, 32, 0, s>>>(bucket_count, bucket_cursor);
    k_bucket_scatter<<<blocks_for(n, ENC_THREADS), ENC_THREADS, 0, s>>>(cnt, c.off, gstart, n, bucket_cursor, ent);
    k_grams_coop<<<(unsigned)(n_sm * 8), QG_COOP_THREADS, 0, s>>>(c.bytes, c.valid, n, q, ent, bucket_cursor, grams,
                                                                  c.nbytes, rec, W, feat, mid_list, n_mid, long_list,
                                                                  n_long);
    HB_LAUNCHED(1);
    k_grams_mid<<<(unsigned)(n_sm * 8), 256, 0, s>>>(c.bytes, c.off, q, gstart, grams, c.nbytes, rec, W, feat,
                                                     mid_list, n_mid);
    HB_LAUNCHED(1);
    k_grams_long<<<(unsigned)(n_sm * 4), 256, 0, s>>>(c.bytes, c.off, q, gstart, grams, c.nbytes, rec, W, feat,
                                                      long_list, n_long, too_long);
}

HB_ERROR_READER(checked_error_encode)

}  // namespace hb
