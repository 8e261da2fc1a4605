// Pair evaluation: the hot loop of blocking.
//
// Work items are tiles of a block's pair space (T x T tuples, the upper
// triangle for a self-join), or packed tiles holding several small self-join
// blocks side by side.  A persistent grid of warps claims tiles (up to 16 per
// claim) from one atomic counter (task stealing in the form of a shared queue,
// Section 5.2).  Each warp works on one tile at a time; consecutive tiles of a
// claim mostly share their row band, whose staged records are then kept, and
// the next tile's member ids are loaded while the current one is evaluated:
//
//  phase 1 (every pair, branch-light): the warp stages the tile's "hot"
//    records (equality codes, the filter operand of each MD's first predicate
//    and, within a word budget, bins and second-predicate operands) in shared
//    memory, rows tuple-major and columns word-major; lane = row, loop over
//    the columns 4 at a time.  For every pair:
//      - equality keys: bit e of E is set when both tuples hold the same
//        present code of key e; the MDs whose keys are all in E are alive;
//      - owner check: the pair is handled only in the block of the lowest
//        alive MD, so each pair is evaluated once however many blocks hold it;
//      - when the alive MDs are exactly those alive in every pair of the
//        block, the cheap necessary condition of each one's first predicate
//        (length / size filter, or the |a-b| test itself) rejects most pairs
//        at once: a pair survives if one of them passes;
//    the owner / keep decisions come from per-tile tables indexed by the
//    combination of other-key matches, applied to per-row match masks, and a
//    filter is a per-row interval test; each lane collects its kept columns
//    in a bit mask, and one warp prefix sum per tile turns the masks into a
//    per-warp survivor list.
//  phase 1b (when the hot record holds more than phase 1 used): each survivor
//    is screened with the staged necessary conditions of every alive MD's
//    first two predicates (shared memory only; the survivors whose alive set
//    is the block's base set first, with warp-uniform ops) and the rest join
//    a per-warp ring spanning tiles, so phase 2 always runs 32 pairs at a time.
//  phase 2 (survivors, 32 at a time, all lanes busy): the sequential execution
//    path of Section 5.1 on the full records: non-equality predicates in plan
//    order, each evaluated once per pair and its result applied to every MD
//    holding it ("Reusing computation"), skipped when no alive MD needs it,
//    with a checkpoint after each MD's last predicate; witnessed pairs are
//    compacted with a warp ballot and one atomic.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <type_traits>

#include "hb_internal.h"

namespace hb {
namespace {

constexpr int EV_THREADS = 256;
constexpr int EV_WARPS = EV_THREADS / 32;
constexpr int LOG_FIELDS = 6;   // evaluated, passed, cycles, stage-1 passes, stage-2 passes, core work

struct LogAcc {
    unsigned long long *s;   // shared [MAX_OPS * LOG_FIELDS] or null
};

// warp-aggregated add of per-lane values to one shared counter (the index is
// uniform over the active lanes)
__device__ __forceinline__ void log_add(LogAcc &lg, int idx, unsigned v) {
    const unsigned m = __activemask();
    const unsigned s = __reduce_add_sync(m, v);
    if ((threadIdx.x & 31) == __ffs(m) - 1) atomicAdd(&lg.s[idx], (unsigned long long)s);
}

// Bag distance over the 8 character bins of two signatures (4-bit counts of
// bytes with (byte & 7) == bin, saturating at 15): max of the summed excess
// counts either way.  Every edit changes the bin counts of a string by at most
// one unit removed and one added, so this is a lower bound of the edit
// distance; a saturated count differs from another by at most their true
// difference, so the bound stays valid.
__device__ __forceinline__ unsigned sig_bag(uint32_t a, uint32_t b) {
    const uint32_t m = 0x0F0F0F0Fu;
    const uint32_t al = a & m, ah = (a >> 4) & m, bl = b & m, bh = (b >> 4) & m;
    const unsigned p1 = __dp4a(__vsubus4(al, bl), 0x01010101u, __dp4a(__vsubus4(ah, bh), 0x01010101u, 0u));
    const unsigned p2 = __dp4a(__vsubus4(bl, al), 0x01010101u, __dp4a(__vsubus4(bh, ah), 0x01010101u, 0u));
    return max(p1, p2);
}

// Upper bound of |A n B| from the sizes and the 64-bit presence masks of the
// grams' hash bins: each bin that A occupies and B does not holds a gram of A
// outside B (distinct bins, distinct grams), and likewise the other way.
__device__ __forceinline__ uint32_t mask_common_ub(uint32_t na, uint64_t ma, uint32_t nb, uint64_t mb) {
    return min(na - (uint32_t)__popcll(ma & ~mb), nb - (uint32_t)__popcll(mb & ~ma));
}

// ---- edit distance <= K: Ukkonen-banded Wagner-Fischer, band of 2K+1 cells ----
// D[i][j] is kept for |i - j| <= K only (other cells exceed K); values are
// clamped at K+1.  Returns false as soon as a whole band row exceeds K.
template <int K>
__device__ __forceinline__ bool ed_band_fixed(const uint8_t *a, int la, const uint8_t *b, int lb, uint32_t &rows) {
    constexpr int BW = 2 * K + 1;
    constexpr int BIG = K + 1;
    int Bd[BW];
    int win[BW];   // win[d] = b[j - 1] for j = i + d - K (text byte on the band), -1 outside
#pragma unroll
    for (int d = 0; d < BW; d++) {
        int j = d - K;
        Bd[d] = (j >= 0 && j <= lb) ? j : BIG;
        int jj = 1 + d - K;   // row 1
        win[d] = (jj >= 1 && jj <= lb) ? (int)b[jj - 1] : -1;
    }
    int i = 1;
    for (; i <= la; i++) {
        const int ai = a[i - 1];
        int left = BIG, rowmin = BIG;
#pragma unroll
        for (int d = 0; d < BW; d++) {
            const int j = i + d - K;
            int v;
            if (j < 0 || j > lb) {
                v = BIG;
            } else if (j == 0) {
                v = i < BIG ? i : BIG;
            } else {
                int sub = Bd[d] + (ai != win[d] ? 1 : 0);
                int del = (d + 1 < BW) ? Bd[d + 1] + 1 : BIG;
                int ins = left + 1;
                v = min(sub, min(del, ins));
                v = v < BIG ? v : BIG;
            }
            Bd[d] = v;
            left = v;
            rowmin = min(rowmin, v);
        }
        if (rowmin > K) {
            rows += i;
            return false;
        }
        // slide the text window to row i + 1
#pragma unroll
        for (int d = 0; d + 1 < BW; d++) win[d] = win[d + 1];
        {
            int jj = i + 1 + (BW - 1) - K;
            win[BW - 1] = (jj >= 1 && jj <= lb) ? (int)b[jj - 1] : -1;
        }
    }
    rows += la;
    const int dfin = lb - la + K;
    return Bd[dfin] <= K;
}

constexpr int KMAX_GENERIC = 31;

__device__ bool ed_band_generic(const uint8_t *a, int la, const uint8_t *b, int lb, int K, uint32_t &rows) {
    const int BW = 2 * K + 1;
    const int BIG = K + 1;
    int Bd[2 * KMAX_GENERIC + 1];
    for (int d = 0; d < BW; d++) {
        int j = d - K;
        Bd[d] = (j >= 0 && j <= lb) ? j : BIG;
    }
    for (int i = 1; i <= la; i++) {
        const int ai = a[i - 1];
        int left = BIG, rowmin = BIG;
        for (int d = 0; d < BW; d++) {
            const int j = i + d - K;
            int v;
            if (j < 0 || j > lb) {
                v = BIG;
            } else if (j == 0) {
                v = i < BIG ? i : BIG;
            } else {
                int sub = Bd[d] + (ai != (int)b[j - 1] ? 1 : 0);
                int del = (d + 1 < BW) ? Bd[d + 1] + 1 : BIG;
                int ins = left + 1;
                v = min(sub, min(del, ins));
                v = v < BIG ? v : BIG;
            }
            Bd[d] = v;
            left = v;
            rowmin = min(rowmin, v);
        }
        if (rowmin > K) {
            rows += i;
            return false;
        }
    }
    rows += la;
    return Bd[lb - la + K] <= K;
}

__device__ __forceinline__ bool ed_le(const uint8_t *a, int la, const uint8_t *b, int lb, int k, uint32_t &rows) {
    switch (k) {
    case 0: {
        for (int i = 0; i < la; i++)
            if (a[i] != b[i]) return false;   // la == lb here
        rows += la;
        return true;
    }
    case 1: return ed_band_fixed<1>(a, la, b, lb, rows);
    case 2: return ed_band_fixed<2>(a, la, b, lb, rows);
    case 3: return ed_band_fixed<3>(a, la, b, lb, rows);
    case 4: return ed_band_fixed<4>(a, la, b, lb, rows);
    default: return ed_band_generic(a, la, b, lb, k, rows);
    }
}


template <bool LOG>
__device__ __forceinline__ bool eval_op(const EvalParams &P, int k, const uint32_t *__restrict__ a,
                                        const uint32_t *__restrict__ b, LogAcc &lg) {
    const Op &op = P.ops[k];
    const int f = op.feat;
    if (op.kind == OP_ABS) {
        const float x = __uint_as_float(__ldg(a + f)), y = __uint_as_float(__ldg(b + f));
        return fabsf(x - y) <= op.delta;
    }
    if (op.kind == OP_ED) {
        const uint32_t la = __ldg(a + f), lb = __ldg(b + f);
        if (la == NULL_LEN || lb == NULL_LEN) return false;
        const uint32_t d = la > lb ? la - lb : lb - la;
        if (d > op.k) return false;
        if (LOG) log_add(lg, k * LOG_FIELDS + 3, 1u);
        // bag distance over 16 character bins is a lower bound of the edit distance
        unsigned p1 = 0, p2 = 0;
#pragma unroll
        for (int w = 0; w < 4; w++) {
            const unsigned x = __ldg(a + f + 2 + w), y = __ldg(b + f + 2 + w);
            p1 = __dp4a(__vsubus4(x, y), 0x01010101u, p1);
            p2 = __dp4a(__vsubus4(y, x), 0x01010101u, p2);
        }
        if (max(p1, p2) > op.k) return false;
        if (LOG) log_add(lg, k * LOG_FIELDS + 4, 1u);
        const uint32_t oa = __ldg(a + f + 1), ob = __ldg(b + f + 1);
        if (!HB_RANGE_OK(oa, la, P.len_r[k], 12) || !HB_RANGE_OK(ob, lb, P.len_s[k], 13)) return false;
        const uint8_t *sa = static_cast<const uint8_t *>(P.ptr_r[k]) + oa;
        const uint8_t *sb = static_cast<const uint8_t *>(P.ptr_s[k]) + ob;
        uint32_t rows = 0;
        const bool r = ed_le(sa, (int)la, sb, (int)lb, op.k, rows);
        if (LOG) log_add(lg, k * LOG_FIELDS + 5, rows * (2u * op.k + 1u));
        return r;
    }
    if (op.kind == OP_EQX) {   // two columns' codes in one dictionary; a missing or unmatched code equals nothing
        const uint32_t x = __ldg(a + f), y = __ldg(b + op.k);
        return x < NOMATCH_CODE && x == y;
    }
    if (op.kind == OP_CONST) return __ldg((op.num ? b : a) + f) != 0u;   // the named tuple's flag word
    const uint32_t na = __ldg(a + f), nb = __ldg(b + f);
    if (na == NULL_LEN || nb == NULL_LEN) return false;
    if (op.kind == OP_CONT) {
        // containment: |A n B| * den >= num * |D|, D the set of side k (0: a's, 1: b's); the
        // size, presence-mask and gram-bin bounds of |A n B| first, then an early-exit merge
        const uint64_t den = op.den;
        const uint64_t need = (uint64_t)op.num * (op.k ? nb : na);
        if ((uint64_t)min(na, nb) * den < need) return false;
        if (LOG) log_add(lg, k * LOG_FIELDS + 3, 1u);
        {
            const uint64_t ma = (uint64_t)__ldg(a + f + FEAT_JAC_MASK) | ((uint64_t)__ldg(a + f + FEAT_JAC_MASK + 1) << 32);
            const uint64_t mb = (uint64_t)__ldg(b + f + FEAT_JAC_MASK) | ((uint64_t)__ldg(b + f + FEAT_JAC_MASK + 1) << 32);
            if ((uint64_t)mask_common_ub(na, ma, nb, mb) * den < need) return false;
        }
        if (na <= 255u && nb <= 255u) {
            unsigned ub = 0;
#pragma unroll
            for (int w = 0; w < 8; w++) ub = __dp4a(__vminu4(__ldg(a + f + 2 + w), __ldg(b + f + 2 + w)), 0x01010101u, ub);
            if ((uint64_t)ub * den < need) return false;
        }
        if (LOG) log_add(lg, k * LOG_FIELDS + 4, 1u);
        const uint64_t imin = (need + den - 1) / den;
        if (imin == 0) return true;
        const uint32_t ga = __ldg(a + f + 1), gb = __ldg(b + f + 1);
        if (!HB_RANGE_OK(ga, na, P.len_r[k], 14) || !HB_RANGE_OK(gb, nb, P.len_s[k], 15)) return false;
        const uint32_t *A = static_cast<const uint32_t *>(P.ptr_r[k]) + ga;
        const uint32_t *B = static_cast<const uint32_t *>(P.ptr_s[k]) + gb;
        uint32_t i = 0, j = 0, I = 0;
        bool res = false;
        while (i < na && j < nb) {
            const uint32_t x = __ldg(A + i), y = __ldg(B + j);
            I += (x == y) ? 1u : 0u;
            i += (x <= y) ? 1u : 0u;
            j += (y <= x) ? 1u : 0u;
            if (I >= imin) {
                res = true;
                break;
            }
            if ((uint64_t)I + min(na - i, nb - j) < imin) break;
        }
        if (LOG) log_add(lg, k * LOG_FIELDS + 5, i + j);
        return res;
    }
    // OP_JAC (q-gram or word-token code sets)
    const uint64_t num = op.num, den = op.den;
    const uint32_t mn = min(na, nb), mx = max(na, nb);
    if ((uint64_t)mn * den < num * mx) return false;   // J <= min/max
    if (LOG) log_add(lg, k * LOG_FIELDS + 3, 1u);
    const uint64_t dn = den + num;
    const uint64_t need = num * ((uint64_t)na + nb);   // I*(den+num) >= num*(|A|+|B|)
    {
        const uint64_t ma = (uint64_t)__ldg(a + f + FEAT_JAC_MASK) | ((uint64_t)__ldg(a + f + FEAT_JAC_MASK + 1) << 32);
        const uint64_t mb = (uint64_t)__ldg(b + f + FEAT_JAC_MASK) | ((uint64_t)__ldg(b + f + FEAT_JAC_MASK + 1) << 32);
        if ((uint64_t)mask_common_ub(na, ma, nb, mb) * dn < need) return false;
    }
    if (na <= 255u && nb <= 255u) {
        unsigned ub = 0;   // sum over 32 gram bins of min(count_a, count_b) >= |A n B|
#pragma unroll
        for (int w = 0; w < 8; w++) ub = __dp4a(__vminu4(__ldg(a + f + 2 + w), __ldg(b + f + 2 + w)), 0x01010101u, ub);
        if ((uint64_t)ub * dn < need) return false;
    }
    if (LOG) log_add(lg, k * LOG_FIELDS + 4, 1u);
    const uint64_t imin = (need + dn - 1) / dn;
    if (imin == 0) return true;
    const uint32_t ga = __ldg(a + f + 1), gb = __ldg(b + f + 1);
    if (!HB_RANGE_OK(ga, na, P.len_r[k], 14) || !HB_RANGE_OK(gb, nb, P.len_s[k], 15)) return false;
    const uint32_t *A = static_cast<const uint32_t *>(P.ptr_r[k]) + ga;
    const uint32_t *B = static_cast<const uint32_t *>(P.ptr_s[k]) + gb;
    uint32_t i = 0, j = 0, I = 0;
    bool res = false;
    while (i < na && j < nb) {
        const uint32_t x = __ldg(A + i), y = __ldg(B + j);
        I += (x == y) ? 1u : 0u;
        i += (x <= y) ? 1u : 0u;
        j += (y <= x) ? 1u : 0u;
        if (I >= imin) {
            res = true;
            break;
        }
        if ((uint64_t)I + min(na - i, nb - j) < imin) break;
    }
    if (LOG) log_add(lg, k * LOG_FIELDS + 5, i + j);
    return res;
}

template <bool LOG>
__device__ __forceinline__ bool run_program(const EvalParams &P, uint64_t alive, const uint32_t *a,
                                            const uint32_t *b, LogAcc &lg) {
    // profile mode (logging only): evaluate every predicate the initially alive
    // MDs hold, without early exit; the verdict is unchanged
    const bool prof = LOG && P.profile;
    alive &= ~P.group_mds;
    const uint64_t alive0 = alive;
    bool hit = (alive & P.eqonly) != 0;
    if (hit && !prof) return true;
    for (int k = 0; k < P.n_ops; k++) {
        const uint64_t need = P.ops[k].need;
        if ((prof ? alive0 : alive) & need) {
            long long c0 = 0;
            if (LOG) c0 = clock64();
            const bool r = eval_op<LOG>(P, k, a, b, lg);
            if (LOG) {
                log_add(lg, k * LOG_FIELDS + 0, 1u);
                log_add(lg, k * LOG_FIELDS + 1, r ? 1u : 0u);
                log_add(lg, k * LOG_FIELDS + 2, (unsigned)min(clock64() - c0, 0x7fffffffll));
            }
            if (!r) alive &= ~need;
        }
        if (alive & P.ops[k].cp) {
            if (!prof) return true;
            hit = true;
        }
        if (!alive && !prof) return false;
    }
    return hit;
}

__device__ __forceinline__ void decode_tile(uint64_t q, uint32_t nr, uint32_t ns, int self_join, int T, uint32_t &ti,
                                            uint32_t &tj) {
    if (!self_join) {
        const uint64_t nts = (ns + T - 1) / T;
        ti = (uint32_t)(q / nts);
        tj = (uint32_t)(q % nts);
        return;
    }
    const int64_t nt = (nr + T - 1) / T;
    // row i holds nt - i tiles; start(i) = i*nt - i*(i-1)/2
    const float b2 = 2.0f * (float)nt + 1.0f;
    int64_t i = (int64_t)floorf((b2 - sqrtf(fmaxf(b2 * b2 - 8.0f * (float)q, 0.0f))) * 0.5f);
    if (i < 0) i = 0;
    if (i > nt - 1) i = nt - 1;
    auto start = [&](int64_t r) { return r * nt - r * (r - 1) / 2; };
    while (i + 1 < nt && start(i + 1) <= (int64_t)q) i++;
    while (i > 0 && start(i) > (int64_t)q) i--;
    ti = (uint32_t)i;
    tj = (uint32_t)(i + ((int64_t)q - start(i)));
}

// largest b in [0, nb) with prefix[b] <= t, searched 32 ways per round
__device__ __forceinline__ uint32_t find_block(const uint64_t *prefix, uint32_t nb, uint64_t t, int lane) {
    uint32_t lo = 0, hi = nb;   // prefix[lo] <= t < prefix[hi]
    while (hi - lo > 1) {
        const uint32_t step = (hi - lo + 31) / 32;
        const uint32_t idx = lo + (uint32_t)lane * step;
        const bool le = idx < hi && prefix[idx] <= t;
        const unsigned m = __ballot_sync(0xffffffffu, le);
        const uint32_t L = 31 - __clz(m);
        const uint32_t nlo = lo + L * step;
        hi = min(hi, nlo + step);
        lo = nlo;
    }
    return lo;
}

__device__ __forceinline__ uint64_t alive_of(const EvalParams &P, const uint64_t *lut, uint32_t E) {
    if (P.use_lut) return lut[E];
    uint64_t alive = 0;
    for (int m = 0; m < P.n_md; m++) alive |= ((E & P.eqset[m]) == P.eqset[m]) ? (1ull << m) : 0ull;
    return alive;
}

// the cheap necessary condition of a predicate on the staged filter operands
// (length filter of edit distance, size filter of Jaccard, |a-b| <= delta
// itself); word w of the column record is hc[w * cs]
__device__ __forceinline__ bool first_filter(const Op &op, const uint32_t *hr, const uint32_t *hc, int cs) {
    const uint32_t x = hr[op.hot], y = hc[op.hot * cs];
    if (op.kind == OP_ED) return x != NULL_LEN && y != NULL_LEN && (x > y ? x - y : y - x) <= op.k;
    if (op.kind == OP_JAC)
        return x != NULL_LEN && y != NULL_LEN && (uint64_t)min(x, y) * op.den >= (uint64_t)op.num * max(x, y);
    return fabsf(__uint_as_float(x) - __uint_as_float(y)) <= op.delta;
}

// phase-1 filter forms of one tile
enum : int { F_NONE = 0, F_RANGE = 1, F_ABS = 2 };

__device__ __forceinline__ int pop(uint32_t x) { return __popc(x); }
__device__ __forceinline__ int pop(uint64_t x) { return __popcll(x); }
__device__ __forceinline__ int first_bit(uint32_t x) { return __ffs(x) - 1; }
__device__ __forceinline__ int first_bit(uint64_t x) { return __ffsll((long long)x) - 1; }

// columns c of row r that form a pair of the tile: c < nc, and c > r on a
// diagonal tile of a self-join; on a packed tile (pn > 0) c must also lie in
// r's block [pn * (r / pn), pn * (r / pn + 1))
template <typename Mask>
__device__ __forceinline__ Mask valid_cols(int r, int nr, int nc, bool diag, int pn) {
    constexpr int BITS = 8 * (int)sizeof(Mask);
    if (r >= nr) return 0;
    if (pn) nc = (r / pn + 1) * pn;   // packed tile: columns of r's own block only
    Mask v = nc >= BITS ? ~(Mask)0 : (((Mask)1 << nc) - (Mask)1);
    if (diag) v &= ~((((Mask)2) << r) - (Mask)1);
    return v;
}

// The length filter of edit distance (|x - y| <= k) and the size filter of
// Jaccard (min(x,y) * den >= num * max(x,y)) both hold exactly for y in an
// interval [lo, hi] around the row's operand x: y passes iff y - lo <= hi - lo
// in unsigned arithmetic (a missing y, 0xFFFFFFFF, never does since hi stays
// below it).  x itself must be present.
__device__ __forceinline__ void filter_range(const Op &op, uint32_t x, uint32_t &lo, uint32_t &span) {
    uint64_t l, h;
    if (op.kind == OP_ED) {
        l = x >= op.k ? x - op.k : 0u;
        h = (uint64_t)x + op.k;
    } else {
        // l = ceil(num * x / den), h = floor(x * den / num): a float estimate,
        // then exact integer correction
        const uint64_t a = (uint64_t)op.num * x, b = (uint64_t)op.den * x;
        const float ratio = (float)op.num / (float)op.den;
        uint64_t q = (uint64_t)fmaxf((float)x * ratio - 2.0f, 0.0f);
        while (q * op.den < a) q++;
        while (q > 0 && (q - 1) * op.den >= a) q--;
        l = q;
        if (op.num == 0) {
            h = 0xFFFFFFFEull;
        } else {
            const float est = (float)x / ratio;
            if (est > 8.0e9f) {   // above 2^32 whatever the rounding: the cap below applies
                h = 0xFFFFFFFEull;
            } else {
                uint64_t e = (uint64_t)fmaxf(est - 2.0f, 0.0f);
                while ((e + 1) * op.num <= b) e++;
                while (e > 0 && e * op.num > b) e--;
                h = e;
            }
        }
    }
    if (h > 0xFFFFFFFEull) h = 0xFFFFFFFEull;
    lo = (uint32_t)l;
    span = (uint32_t)(h - l);
}

// Phase 1 of one row (lane) of a tile, as bit masks over the tile's columns
// (visited 8 at a time, 4 in p1_row, whose smaller unrolled body measured
// faster: the tile's side is a multiple of 8, and bits past nc are cleared by
// the valid mask).
//
// p1_keys: bit c of em[i] = the row's code of the i-th varying equality key
// (okey[i]) equals column c's.
template <int KO, int T, typename Mask>
__device__ __forceinline__ void p1_keys(const uint32_t *__restrict__ hr, const uint32_t *__restrict__ hcols, int nc,
                                        const int *okey, Mask *em) {
    uint32_t rk[KO > 0 ? KO : 1];
    const uint32_t *ck[KO > 0 ? KO : 1];
#pragma unroll
    for (int i = 0; i < KO; i++) {
        const uint32_t x = hr[okey[i]];
        rk[i] = x < NOMATCH_CODE ? x : 0xFFFFFFFDu;   // a missing code matches no column code
        ck[i] = hcols + okey[i] * T;
        em[i] = 0;
    }
    if (KO == 0) return;
    for (int c0 = 0; c0 < nc; c0 += 8) {
        uint32_t ec[KO > 0 ? KO : 1];
#pragma unroll
        for (int i = 0; i < KO; i++) ec[i] = 0;
#pragma unroll
        for (int u = 0; u < 8; u++)
#pragma unroll
            for (int i = 0; i < KO; i++)
                if (ck[i][c0 + u] == rk[i]) ec[i] |= 1u << u;
#pragma unroll
        for (int i = 0; i < KO; i++) em[i] |= (Mask)ec[i] << c0;
    }
}

// p1_filter: bit c = the cheap necessary condition of op holds for (row, column
// c): an interval test on the column's operand (F_RANGE: edit-distance length
// or Jaccard size filter; none passes a missing row operand) or |a - b| <= delta
// (F_ABS).
template <int FK, int T, typename Mask>
__device__ __forceinline__ Mask p1_filter(const uint32_t *__restrict__ hr, const uint32_t *__restrict__ hcols,
                                          int nc, const Op &op) {
    const uint32_t *cf = hcols + op.hot * T;
    const uint32_t x = hr[op.hot];
    uint32_t lo = 0, span = 0;
    if (FK == F_RANGE) {
        if (x == NULL_LEN) return 0;
        filter_range(op, x, lo, span);
    }
    const float xf = __uint_as_float(x), dl = op.delta;
    Mask fm = 0;
    for (int c0 = 0; c0 < nc; c0 += 8) {
        uint32_t fc = 0;
#pragma unroll
        for (int u = 0; u < 8; u++) {
            const uint32_t y = cf[c0 + u];
            const bool pass = FK == F_RANGE ? y - lo <= span : fabsf(xf - __uint_as_float(y)) <= dl;
            if (pass) fc |= 1u << u;
        }
        fm |= (Mask)fc << c0;
    }
    return fm;
}

// p1_combine: the tile's decisions applied to whole masks.  For each
// combination cb of other-key matches, own8 bit cb = the pair is owned, kf8
// bit cb = it is kept even when every base filter fails (an owned pair is kept
// when one passes: fm).  Returns the row's surviving columns; owned = its
// owned (candidate) pairs; extra = the survivors of kf8 combinations (more MDs
// alive than the block's base set; the others have exactly the base set).
template <int KO, typename Mask>
__device__ __forceinline__ Mask p1_combine(const Mask *em, Mask fm, uint32_t own8, uint32_t kf8, Mask vm,
                                           unsigned &owned, Mask &extra) {
    Mask keep = 0, ext = 0;
    owned = 0;
#pragma unroll
    for (int cb = 0; cb < (1 << KO); cb++) {
        if (!((own8 >> cb) & 1u)) continue;
        Mask mt = vm;
#pragma unroll
        for (int i = 0; i < KO; i++) mt &= ((cb >> i) & 1) ? em[i] : ~em[i];
        owned += (unsigned)pop(mt);
        const bool kf = (kf8 >> cb) & 1u;
        keep |= kf ? mt : (mt & fm);
        ext |= kf ? mt : (Mask)0;
    }
    extra = ext;
    return keep;
}

// p1_row: the same for one row with at most one base filter (FK), in a single
// pass over the columns (keys and filter together), then the decisions of
// p1_combine applied inline; keep_out = surviving columns, extra_out = those
// of kf8 combinations, owned_out = owned (candidate) pairs.
template <int KO, int FK, int T, typename Mask>
__device__ __forceinline__ void p1_row(const uint32_t *__restrict__ hr, const uint32_t *__restrict__ hcols, int nc,
                                       const int *okey, const Op &op0, uint32_t own8, uint32_t kf8, Mask vm,
                                       Mask &keep_out, Mask &extra_out, unsigned &owned_out) {
    uint32_t rk[KO > 0 ? KO : 1];
    const uint32_t *ck[KO > 0 ? KO : 1];
#pragma unroll
    for (int i = 0; i < KO; i++) {
        const uint32_t x = hr[okey[i]];
        rk[i] = x < NOMATCH_CODE ? x : 0xFFFFFFFDu;
        ck[i] = hcols + okey[i] * T;
    }
    const uint32_t *cf = FK != F_NONE ? hcols + op0.hot * T : hcols;
    uint32_t lo = 0, span = 0;
    bool rnull = false;
    float xf = 0.f;
    const float dl = op0.delta;
    if (FK == F_RANGE) {
        const uint32_t x = hr[op0.hot];
        rnull = x == NULL_LEN;
        if (!rnull) filter_range(op0, x, lo, span);
    }
    if (FK == F_ABS) xf = __uint_as_float(hr[op0.hot]);
    Mask em[KO > 0 ? KO : 1];
#pragma unroll
    for (int i = 0; i < KO; i++) em[i] = 0;
    Mask fm = 0;
    if (KO > 0 || FK != F_NONE) {
        for (int c0 = 0; c0 < nc; c0 += 4) {
            uint32_t ec[KO > 0 ? KO : 1], fc = 0;
#pragma unroll
            for (int i = 0; i < KO; i++) ec[i] = 0;
#pragma unroll
            for (int u = 0; u < 4; u++) {
                const int c = c0 + u;
#pragma unroll
                for (int i = 0; i < KO; i++)
                    if (ck[i][c] == rk[i]) ec[i] |= 1u << u;
                if (FK == F_RANGE && cf[c] - lo <= span) fc |= 1u << u;
                if (FK == F_ABS && fabsf(xf - __uint_as_float(cf[c])) <= dl) fc |= 1u << u;
            }
#pragma unroll
            for (int i = 0; i < KO; i++) em[i] |= (Mask)ec[i] << c0;
            fm |= (Mask)fc << c0;
        }
    }
    if (FK == F_NONE) fm = ~(Mask)0;
    if (FK == F_RANGE && rnull) fm = 0;
    Mask keep = 0, ext = 0;
    unsigned owned = 0;
#pragma unroll
    for (int cb = 0; cb < (1 << KO); cb++) {
        if (!((own8 >> cb) & 1u)) continue;
        Mask mt = vm;
#pragma unroll
        for (int i = 0; i < KO; i++) mt &= ((cb >> i) & 1) ? em[i] : ~em[i];
        owned += (unsigned)pop(mt);
        const bool kf = (kf8 >> cb) & 1u;
        keep |= kf ? mt : (mt & fm);
        ext |= kf ? mt : (Mask)0;
    }
    keep_out = keep;
    extra_out = ext;
    owned_out = owned;
}

// A necessary condition of a predicate from the hot records alone: the filter
// operand test and, where its signature words are staged, the bag-distance
// bound of edit distance over the signature's bins or the presence-mask bound
// of Jaccard.  Word w of the column record is hc[w * cs].
__device__ __forceinline__ bool screen(const Op &op, const uint32_t *hr, const uint32_t *hc, int cs) {
    const uint32_t x = hr[op.hot], y = hc[op.hot * cs];
    if (op.kind == OP_ABS) return fabsf(__uint_as_float(x) - __uint_as_float(y)) <= op.delta;
    if (x == NULL_LEN || y == NULL_LEN) return false;
    const int h2 = op.hot2;
    if (op.kind == OP_ED) {
        if ((x > y ? x - y : y - x) > op.k) return false;
        return h2 == 255 || sig_bag(hr[h2], hc[h2 * cs]) <= op.k;
    }
    if ((uint64_t)min(x, y) * op.den < (uint64_t)op.num * max(x, y)) return false;
    if (h2 == 255) return true;
    const uint64_t ma = (uint64_t)hr[h2] | ((uint64_t)hr[h2 + 1] << 32);
    const uint64_t mb = (uint64_t)hc[h2 * cs] | ((uint64_t)hc[(h2 + 1) * cs] << 32);
    return (uint64_t)mask_common_ub(x, ma, y, mb) * ((uint64_t)op.den + op.num) >= (uint64_t)op.num * ((uint64_t)x + y);
}

// per-warp ring of survivors waiting for phase 2: tuple ids and equality-match bits
constexpr int RING_SLOTS = 64;

// phase 2 for one survivor per lane (act): the sequential program on the full
// records; witnessed pairs are compacted with a warp ballot and one atomic.
// Kept out of line: it runs for few pairs, and inlined its code (the banded
// edit-distance variants, the merge) crowds the hot loops' registers and
// instruction cache (measured: C2 evaluation 5.8 -> 3.8 ms out of line)
template <bool LOG>
__device__ __noinline__ void phase2(const EvalParams &P, const uint64_t *lut, bool act, uint32_t ra,
                                       uint32_t cb, uint32_t E, const uint32_t *rec_c, int W, int lane,
                                       unsigned lt, LogAcc &lg) {
    bool hit = false;
    if (act) {
        const uint64_t alive = alive_of(P, lut, E);
        hit = run_program<LOG>(P, alive, P.rec_r + (size_t)HB_IDX(ra, P.n_r, 10) * W,
                               rec_c + (size_t)HB_IDX(cb, P.self_join ? P.n_r : P.n_s, 11) * W, lg);
    }
    const unsigned hm = __ballot_sync(0xffffffffu, hit);
    if (hm) {
        unsigned long long base = 0;
        if (lane == 0) base = atomicAdd(P.out_count, (unsigned long long)__popc(hm));
        base = __shfl_sync(0xffffffffu, base, 0);
        if (hit) {
            const unsigned long long idx = base + __popc(hm & lt);
            uint64_t key;
            if (P.self_join) {
                const uint32_t lo2 = ra < cb ? ra : cb, hi2 = ra < cb ? cb : ra;
                key = ((uint64_t)lo2 << P.key_bits_s) | (uint64_t)hi2;
            } else {
                key = ((uint64_t)(ra + P.row_base) << P.key_bits_s) | (uint64_t)(cb + P.col_base);
            }
            if (idx < P.out_cap) P.out[idx] = key;
        }
    }
}

// MULTI: the general phase 1 for rule sets that need it: blocks with 2..4
// distinct base filters (multi-pass) or 4 varying equality keys.  RING: the
// survivors are screened (phase 1b) and batched through the warp's ring;
// otherwise phase 2 runs per tile.
template <int R, bool LOG, bool MULTI, bool RING>
__global__ void __launch_bounds__(EV_THREADS, 4) k_eval(const __grid_constant__ EvalParams P) {
    extern __shared__ __align__(16) uint32_t smem[];
    constexpr int T = 32 * R;
    constexpr int SURV_CAP = T * T / 4;   // survivor list entries (16-bit) per warp
    using Mask = typename std::conditional<(R == 2), uint64_t, uint32_t>::type;
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int HW = P.HW, HWP = P.HW + 1, W = P.W;
    uint64_t *lut = reinterpret_cast<uint64_t *>(smem);
    const int lut_words = P.use_lut ? 2 * (1 << P.n_eq) : 0;
    uint32_t *wbase = smem + lut_words + wib * (T * HWP + T * HW + 2 * T + SURV_CAP / 2 + 3 * RING_SLOTS);
    uint32_t *hrows = wbase;
    uint32_t *hcols = hrows + T * HWP;
    uint32_t *rid_s = hcols + T * HW;
    uint32_t *cid_s = rid_s + T;
    uint16_t *surv = reinterpret_cast<uint16_t *>(cid_s + T);
    uint32_t *ring_ra = cid_s + T + SURV_CAP / 2;
    uint32_t *ring_cb = ring_ra + RING_SLOTS;
    uint32_t *ring_e = ring_cb + RING_SLOTS;
    int pend = 0;   // survivors in the ring (warp-uniform)
    __shared__ unsigned long long lgs[LOG ? MAX_OPS * LOG_FIELDS : 1];
    LogAcc lg{lgs};
    if (P.use_lut)
        for (int i = threadIdx.x; i < (1 << P.n_eq); i += blockDim.x) lut[i] = P.lut[i];
    if (LOG)
        for (int i = threadIdx.x; i < MAX_OPS * LOG_FIELDS; i += blockDim.x) lgs[i] = 0;
    __syncthreads();

    const uint32_t nb = *P.n_blocks;
    const uint64_t total = P.tile_prefix[nb];
    // tiles per claim: at most P.claim, and few enough that every warp gets about
    // 8 claims (small launches would otherwise end on a few warps' last claims);
    // kept in shared memory, read once per claim
    __shared__ unsigned s_claim;
    if (threadIdx.x == 0) {
        const uint64_t per = total / ((uint64_t)gridDim.x * (blockDim.x >> 5) * 8);
        s_claim = (unsigned)max((uint64_t)1, min((uint64_t)P.claim, per));
    }
    __syncthreads();
    const unsigned lt = (1u << lane) - 1u;
    const uint32_t allkeys = P.keymask;
    const uint32_t *rec_c = P.self_join ? P.rec_r : P.rec_s;
    const uint32_t *hot_c = P.self_join ? P.hot_r : P.hot_s;
    unsigned long long cand = 0, exam = 0;
    // the row band whose hot records are staged (warp-uniform): consecutive
    // tiles of one block share their rows, which are then not staged again
    uint32_t rows_bi = 0xFFFFFFFFu, rows_ti = 0;
    // the tile-level decision tables of the last MD seen (warp-uniform): its
    // varying keys (4 x 8 bits), their count, the owned / base-set masks, its
    // base filter count and the program index of its first base filter
    uint32_t c_m = 0xFFFFFFFFu, c_okey = 0, c_own = 0, c_basem = 0;
    int c_ko = 0, c_nbase = 0, c_op0 = 0;

    for (;;) {
        unsigned long long t0 = 0;
        const unsigned claim = s_claim;
        if (lane == 0) t0 = atomicAdd(P.tile_counter, (unsigned long long)claim);
        t0 = __shfl_sync(0xffffffffu, t0, 0);
        if (t0 >= total) break;
        const uint64_t t1 = min((uint64_t)t0 + (uint64_t)claim, total);
        uint32_t bi = find_block(P.tile_prefix, nb, t0, lane);
        // the next tile of the claim, located one tile ahead (warp-uniform), and
        // its member ids (per lane), loaded while this tile is evaluated
        bool nx_ok = false;
        uint32_t nx_ti = 0, nx_tj = 0, nx_r[R], nx_c[R];
#pragma unroll
        for (int rr = 0; rr < R; rr++) nx_r[rr] = nx_c[rr] = 0;
        for (uint64_t t = t0; t < t1; t++) {
            while (P.tile_prefix[bi + 1] <= t) bi++;
            const BlockDesc B = P.blocks[HB_IDX(bi, nb, 1)];
            // pn > 0: a packed tile of self-join blocks of pn tuples, side by side
            const int pn = (int)B.packed;
            uint32_t ti = 0, tj = 0;
            const bool pre = nx_ok;   // this tile was located, and its member ids loaded, one tile ago
            uint32_t pre_r[R], pre_c[R];
#pragma unroll
            for (int rr = 0; rr < R; rr++) {
                pre_r[rr] = nx_r[rr];
                pre_c[rr] = nx_c[rr];
            }
            if (pre) {
                ti = nx_ti;
                tj = nx_tj;
            } else if (!pn) {
                decode_tile(t - P.tile_prefix[bi], B.n_r, B.n_s, P.self_join, T, ti, tj);
            }
            const bool rows_kept = !pn && bi == rows_bi && ti == rows_ti;
            nx_ok = false;
            if (t + 1 < t1) {
                uint32_t bj = bi;
                while (P.tile_prefix[bj + 1] <= t + 1) bj++;
                const bool same_block = bj == bi;
                const BlockDesc B1 = same_block ? B : P.blocks[HB_IDX(bj, nb, 1)];
                if (!B1.packed) {
                    if (same_block) {
                        // the tile after (ti, tj) in the block's order: along the row band, then
                        // the next band from its diagonal (self-join) or first column band
                        const uint32_t ntc = (B.n_s + T - 1) / T;
                        nx_ti = tj + 1 < ntc ? ti : ti + 1;
                        nx_tj = tj + 1 < ntc ? tj + 1 : (P.self_join ? ti + 1 : 0u);
                    } else {
                        decode_tile(t + 1 - P.tile_prefix[bj], B1.n_r, B1.n_s, P.self_join, T, nx_ti, nx_tj);
                    }
                    const uint32_t nr1 = min((uint32_t)T, B1.n_r - nx_ti * T), nc1 = min((uint32_t)T, B1.n_s - nx_tj * T);
                    const bool same_rows = bj == bi && nx_ti == ti;
#pragma unroll
                    for (int rr = 0; rr < R; rr++) {
                        const uint32_t r = (uint32_t)(rr * 32 + lane);
                        nx_r[rr] = (!same_rows && r < nr1)
                                       ? P.members_r[HB_IDX(B1.start_r + nx_ti * T + r, P.members_r_len, 2)] : 0u;
                        nx_c[rr] = r < nc1 ? P.members_s[HB_IDX(B1.start_s + nx_tj * T + r, P.members_s_len, 5)] : 0u;
                    }
                    nx_ok = true;
                }
            }
            const uint32_t r0 = ti * T, c0 = tj * T;
            const int nr = (int)min((uint32_t)T, B.n_r - r0);
            const int nc = (int)min((uint32_t)T, B.n_s - c0);
            const bool diag = P.self_join && ti == tj;
            const uint32_t m = B.md;
            const uint64_t mbit = 1ull << m;
            const uint64_t below = (mbit - 1ull) & P.owner_mds;
            const uint32_t okeys = allkeys & ~(uint32_t)P.eqset[m];
            const uint64_t base = P.base_alive[m];
            // The equality keys of the owner MD hold for every pair of its block;
            // only the other keys (okeys) vary.  With at most 4 of them, lane l
            // works out, for the l-th combination of other-key matches, whether
            // the owner check passes and whether exactly the block's base MDs are
            // alive; each pair then reads its answer from two bit masks.
            // (depend on the MD alone: worked out again only when it changes)
            if (m != c_m) {
                c_m = m;
                c_nbase = P.base_nops[m];
                c_op0 = (c_nbase != 255 && c_nbase > 0) ? P.base_op[m][0] : 0;
                c_ko = __popc(okeys);
                int ok4[4] = {0, 0, 0, 0};
                uint32_t ok = okeys;
#pragma unroll
                for (int i = 0; i < 4; i++) {
                    if (ok) {
                        ok4[i] = __ffs(ok) - 1;
                        ok &= ok - 1;
                    }
                }
                c_okey = (uint32_t)ok4[0] | ((uint32_t)ok4[1] << 8) | ((uint32_t)ok4[2] << 16) | ((uint32_t)ok4[3] << 24);
                c_own = c_basem = 0;
                if (c_ko <= 4) {
                    uint32_t E = P.eqset[m];
#pragma unroll
                    for (int i = 0; i < 4; i++)
                        if (i < c_ko && ((lane >> i) & 1)) E |= 1u << ok4[i];
                    const bool in = lane < (1 << c_ko);
                    const uint64_t al = in ? alive_of(P, lut, E) : 0ull;
                    c_own = __ballot_sync(0xffffffffu, in && (al & mbit) && !(al & below));
                    c_basem = __ballot_sync(0xffffffffu, in && al == base);
                }
            }
            const int ko = c_ko;
            int okey[4];
#pragma unroll
            for (int i = 0; i < 4; i++) okey[i] = (int)((c_okey >> (8 * i)) & 255u);
            const uint32_t ownmask = c_own, basemask = c_basem;
            const int nbase = c_nbase;
            const Op op0 = P.ops[c_op0];
            // ---- stage the hot records of the tile's rows and columns
            __syncwarp();
#pragma unroll
            for (int rr = 0; rr < R; rr++) {
                const int r = rr * 32 + lane;
                uint32_t pid = 0;   // packed tile: row r = member r % pn of block r / pn; columns alike
                if (pn && r < nr)
                    pid = P.members_r[HB_IDX(P.small[HB_IDX(B.start_r + r / pn, P.small_len, 3)] + r % pn,
                                             P.members_r_len, 4)];
                if (r < nr && !rows_kept) {
                    const uint32_t id =
                        HB_IDX(pn ? pid : pre ? pre_r[rr] : P.members_r[HB_IDX(B.start_r + r0 + r, P.members_r_len, 2)],
                               P.n_r, 6);
                    rid_s[r] = id;
                    const uint4 *src = reinterpret_cast<const uint4 *>(P.hot_r + (size_t)id * HW);
                    uint32_t *dst = hrows + r * HWP;
                    for (int w4 = 0; w4 < (HW >> 2); w4++) {
                        const uint4 v = __ldg(src + w4);
                        dst[4 * w4 + 0] = v.x;
                        dst[4 * w4 + 1] = v.y;
                        dst[4 * w4 + 2] = v.z;
                        dst[4 * w4 + 3] = v.w;
                    }
                }
                if (r < nc) {
                    const uint32_t id =
                        HB_IDX(pn ? pid : pre ? pre_c[rr] : P.members_s[HB_IDX(B.start_s + c0 + r, P.members_s_len, 5)],
                               P.self_join ? P.n_r : P.n_s, 7);
                    cid_s[r] = id;
                    const uint4 *src = reinterpret_cast<const uint4 *>(hot_c + (size_t)id * HW);
                    uint32_t *dst = hcols + r;   // word-major: word w of column c at w * T + c
                    for (int w4 = 0; w4 < (HW >> 2); w4++) {
                        const uint4 v = __ldg(src + w4);
                        dst[(4 * w4 + 0) * T] = v.x;
                        dst[(4 * w4 + 1) * T] = v.y;
                        dst[(4 * w4 + 2) * T] = v.z;
                        dst[(4 * w4 + 3) * T] = v.w;
                    }
                }
            }
            __syncwarp();
            rows_bi = pn ? 0xFFFFFFFFu : bi;
            rows_ti = ti;
            // ---- phase 1: every pair of the tile; lane = row, loop over the
            // columns; each lane collects the kept columns of its rows in a bit mask
            exam += pn ? (unsigned long long)(nr / pn) * (pn * (pn - 1) / 2)
                       : diag ? (unsigned long long)nr * (nr - 1) / 2 : (unsigned long long)nr * nc;
            // the MDs alive for every pair of this block (the owner and those whose
            // keys are a subset of its keys): when no other MD is alive, a pair is
            // rejected if the first predicate of each of them fails its necessary
            // condition; any other owned pair goes on as it is
            const bool filt = !LOG && nbase != 255;
            // kmask: surviving columns of each row; xmask: those whose alive set
            // is more than the block's base set (the rest have exactly the base set)
            Mask kmask[R], xmask[R];
            // fast path: at most 4 varying keys, and at most one base filter unless MULTI
            const bool fast = ko <= (MULTI ? 4 : 3) && (MULTI || !filt || nbase == 1);
            if (fast) {
                const uint32_t own8 = ownmask & 0xffffu;   // bit cb: key-match combination cb is owned
                const uint32_t kf8 = filt ? (own8 & ~basemask) : own8;
                const int fk = !filt ? F_NONE : op0.kind == OP_ABS ? F_ABS : F_RANGE;
#pragma unroll
                for (int rr = 0; rr < R; rr++) {
                    const int r = rr * 32 + lane;
                    const uint32_t *hr = hrows + r * HWP;
                    const Mask vm = valid_cols<Mask>(r, nr, nc, diag, pn);
                    Mask km = 0, xm = 0;
                    unsigned ow = 0;
                    bool done = false;
                    if constexpr (MULTI) {
                        if (filt && nbase != 1) {
                            Mask em[4];
                            switch (ko) {
                            case 0: p1_keys<0, T>(hr, hcols, nc, okey, em); break;
                            case 1: p1_keys<1, T>(hr, hcols, nc, okey, em); break;
                            case 2: p1_keys<2, T>(hr, hcols, nc, okey, em); break;
                            case 3: p1_keys<3, T>(hr, hcols, nc, okey, em); break;
                            default: p1_keys<4, T>(hr, hcols, nc, okey, em); break;
                            }
                            Mask fm = 0;
                            for (int i = 0; i < nbase; i++) {
                                const Op &op = P.ops[P.base_op[m][i]];
                                fm |= op.kind == OP_ABS ? p1_filter<F_ABS, T, Mask>(hr, hcols, nc, op)
                                                        : p1_filter<F_RANGE, T, Mask>(hr, hcols, nc, op);
                            }
                            switch (ko) {
                            case 0: km = p1_combine<0, Mask>(em, fm, own8, kf8, vm, ow, xm); break;
                            case 1: km = p1_combine<1, Mask>(em, fm, own8, kf8, vm, ow, xm); break;
                            case 2: km = p1_combine<2, Mask>(em, fm, own8, kf8, vm, ow, xm); break;
                            case 3: km = p1_combine<3, Mask>(em, fm, own8, kf8, vm, ow, xm); break;
                            default: km = p1_combine<4, Mask>(em, fm, own8, kf8, vm, ow, xm); break;
                            }
                            done = true;
                        } else if (ko == 4) {
                            switch (fk) {
                            case F_NONE: p1_row<4, F_NONE, T>(hr, hcols, nc, okey, op0, own8, kf8, vm, km, xm, ow); break;
                            case F_RANGE: p1_row<4, F_RANGE, T>(hr, hcols, nc, okey, op0, own8, kf8, vm, km, xm, ow); break;
                            default: p1_row<4, F_ABS, T>(hr, hcols, nc, okey, op0, own8, kf8, vm, km, xm, ow); break;
                            }
                            done = true;
                        }
                    }
                    if (!done) switch (ko * 3 + fk) {
                    case 0: p1_row<0, F_NONE, T>(hr, hcols, nc, okey, op0, own8, kf8, vm, km, xm, ow); break;
                    case 1: p1_row<0, F_RANGE, T>(hr, hcols, nc, okey, op0, own8, kf8, vm, km, xm, ow); break;
                    case 2: p1_row<0, F_ABS, T>(hr, hcols, nc, okey, op0, own8, kf8, vm, km, xm, ow); break;
                    case 3: p1_row<1, F_NONE, T>(hr, hcols, nc, okey, op0, own8, kf8, vm, km, xm, ow); break;
                    case 4: p1_row<1, F_RANGE, T>(hr, hcols, nc, okey, op0, own8, kf8, vm, km, xm, ow); break;
                    case 5: p1_row<1, F_ABS, T>(hr, hcols, nc, okey, op0, own8, kf8, vm, km, xm, ow); break;
                    case 6: p1_row<2, F_NONE, T>(hr, hcols, nc, okey, op0, own8, kf8, vm, km, xm, ow); break;
                    case 7: p1_row<2, F_RANGE, T>(hr, hcols, nc, okey, op0, own8, kf8, vm, km, xm, ow); break;
                    case 8: p1_row<2, F_ABS, T>(hr, hcols, nc, okey, op0, own8, kf8, vm, km, xm, ow); break;
                    case 9: p1_row<3, F_NONE, T>(hr, hcols, nc, okey, op0, own8, kf8, vm, km, xm, ow); break;
                    case 10: p1_row<3, F_RANGE, T>(hr, hcols, nc, okey, op0, own8, kf8, vm, km, xm, ow); break;
                    default: p1_row<3, F_ABS, T>(hr, hcols, nc, okey, op0, own8, kf8, vm, km, xm, ow); break;
                    }
                    kmask[rr] = km;
                    xmask[rr] = xm;
                    cand += ow;
                }
            } else {
#pragma unroll
                for (int rr = 0; rr < R; rr++) {
                    const int r = rr * 32 + lane;
                    const uint32_t *hr = hrows + r * HWP;
                    const Mask vm = valid_cols<Mask>(r, nr, nc, diag, pn);
                    Mask km = 0, xm = 0;
                    for (int c = 0; c < nc; c++) {
                        const uint32_t *hc = hcols + c;
                        bool own, isbase;
                        if (ko <= 4) {
                            uint32_t combo = 0;
#pragma unroll
                            for (int i = 0; i < 4; i++)
                                if (i < ko) {
                                    const uint32_t x = hr[okey[i]];
                                    combo |= (x == hc[okey[i] * T] && x < NOMATCH_CODE) ? (1u << i) : 0u;
                                }
                            own = (ownmask >> combo) & 1u;
                            isbase = (basemask >> combo) & 1u;
                        } else {
                            uint32_t E = P.eqset[m];
                            for (uint32_t ok = okeys; ok; ok &= ok - 1) {
                                const int e = __ffs(ok) - 1;
                                const uint32_t x = hr[e];
                                E |= (x == hc[e * T] && x < NOMATCH_CODE) ? (1u << e) : 0u;
                            }
                            const uint64_t alive = alive_of(P, lut, E);
                            own = (alive & mbit) && !(alive & below);
                            isbase = alive == base;
                        }
                        bool keep = own;
                        if (filt && own && isbase) {
                            keep = false;
                            for (int i = 0; i < nbase && !keep; i++) keep = first_filter(P.ops[P.base_op[m][i]], hr, hc, T);
                        }
                        const Mask bit = (Mask)1 << c;
                        if (keep) km |= bit;
                        if (own && !(filt && isbase)) xm |= bit;
                        if (own && (vm & bit)) cand++;
                    }
                    kmask[rr] = km & vm;
                    xmask[rr] = xm & vm;
                }
            }
            // survivors, by class (cls 0: alive set = the block's base set, the
            // same for every pair of the class, so its screens are warp-uniform;
            // cls 1: the others), each in rounds of at most SURV_CAP: a warp
            // prefix sum of the per-lane counts places each lane's kept pairs in
            // the warp's survivor list (a round takes the first SURV_CAP in lane
            // order; the rest stay in the masks for the next round)
#pragma unroll
            for (int rr = 0; rr < R; rr++) kmask[rr] &= ~xmask[rr];
            for (int cls = 0; cls < 2; cls++)
            for (;;) {
            int cnt;
            bool more;
            {
                int my = 0;
#pragma unroll
                for (int rr = 0; rr < R; rr++) my += pop(cls ? xmask[rr] : kmask[rr]);
                int incl = my;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const int v = __shfl_up_sync(0xffffffffu, incl, o);
                    if (lane >= o) incl += v;
                }
                const int tot = __shfl_sync(0xffffffffu, incl, 31);
                if (tot == 0) break;
                cnt = min(tot, SURV_CAP);
                more = tot > SURV_CAP;
                int pos = incl - my;
#pragma unroll
                for (int rr = 0; rr < R; rr++) {
                    Mask mk = cls ? xmask[rr] : kmask[rr];
                    const uint32_t rb = (uint32_t)(rr * 32 + lane) << 6;
                    while (mk && pos < SURV_CAP) {
                        const int c = first_bit(mk);
                        mk &= mk - 1;
                        surv[HB_IDX(pos, SURV_CAP, 8)] = (uint16_t)(rb | (uint32_t)c);
                        pos++;
                    }
                    if (cls) xmask[rr] = mk;
                    else kmask[rr] = mk;
                }
            }
            __syncwarp();
            if constexpr (!RING) {
                // ---- phase 2 per tile: the survivors, one per lane
                for (int s0 = 0; s0 < cnt; s0 += 32) {
                    const int s = s0 + lane;
                    uint32_t E = 0, ra = 0, cb = 0;
                    if (s < cnt) {
                        const uint32_t e16 = surv[s];
                        const int r = (int)(e16 >> 6), c = (int)(e16 & 63u);
                        const uint32_t *hr = hrows + r * HWP, *hc = hcols + c;
                        E = P.eqset[m];   // class 0: its alive set is alive_of(eqset[m]) = the base set
                        if (cls)
                            for (uint32_t ok = okeys; ok; ok &= ok - 1) {
                                const int e = __ffs(ok) - 1;
                                const uint32_t x = hr[e];
                                E |= (x == hc[e * T] && x < NOMATCH_CODE) ? (1u << e) : 0u;
                            }
                        ra = rid_s[r];
                        cb = cid_s[c];
                    }
                    phase2<LOG>(P, lut, s < cnt, ra, cb, E, rec_c, W, lane, lt, lg);
                }
            } else {
            // ---- phase 1b: the survivors, 32 at a time (shared memory only): the
            // equality-match bits, then, unless an MD without non-equality
            // predicates is alive, the staged necessary conditions of each alive
            // MD's first two predicates; a survivor that every alive MD fails is
            // dropped, the others join the warp's ring.  Phase 2 runs whenever
            // the ring holds 32, so that every lane of it has a pair.
            for (int s0 = 0; s0 < cnt; s0 += 32) {
                const int s = s0 + lane;
                bool keep = false;
                uint32_t E = 0, ra = 0, cb = 0;
                if (s < cnt) {
                    const uint32_t e16 = surv[s];
                    const int r = (int)(e16 >> 6), c = (int)(e16 & 63u);
                    const uint32_t *hr = hrows + r * HWP, *hc = hcols + c;
                    // class 0: the base set, whatever other keys match (its MDs all
                    // have filters, so none is equality-only); class 1: from the keys
                    E = P.eqset[m];
                    uint64_t alive = base;
                    if (cls) {
                        for (uint32_t ok = okeys; ok; ok &= ok - 1) {
                            const int e = __ffs(ok) - 1;
                            const uint32_t x = hr[e];
                            E |= (x == hc[e * T] && x < NOMATCH_CODE) ? (1u << e) : 0u;
                        }
                        alive = alive_of(P, lut, E);
                    }
                    {
                        keep = (alive & P.eqonly) != 0;
                        for (uint64_t a = alive & ~P.group_mds; a && !keep; a &= a - 1) {
                            const int j = __ffsll((long long)a) - 1;
                            const int o0 = P.screen_op[j][0], o1 = P.screen_op[j][1];
                            keep = (o0 == 255 || screen(P.ops[o0], hr, hc, T)) &&
                                   (o1 == 255 || screen(P.ops[o1], hr, hc, T));
                        }
                    }
                    ra = rid_s[r];
                    cb = cid_s[c];
                }
                const unsigned km = __ballot_sync(0xffffffffu, keep);
                if (keep) {
                    const int q = pend + __popc(km & lt);
                    const int qc = (int)HB_IDX(q, RING_SLOTS, 9);
                    ring_ra[qc] = ra;
                    ring_cb[qc] = cb;
                    ring_e[qc] = E;
                }
                pend += __popc(km);
                if (pend >= 32) {
                    __syncwarp();
                    phase2<LOG>(P, lut, true, ring_ra[lane], ring_cb[lane], ring_e[lane], rec_c, W, lane, lt, lg);
                    const int rest = pend - 32;
                    uint32_t xa = 0, xb = 0, xe = 0;
                    if (lane < rest) {
                        xa = ring_ra[32 + lane];
                        xb = ring_cb[32 + lane];
                        xe = ring_e[32 + lane];
                    }
                    __syncwarp();
                    if (lane < rest) {
                        ring_ra[lane] = xa;
                        ring_cb[lane] = xb;
                        ring_e[lane] = xe;
                    }
                    pend = rest;
                }
                __syncwarp();
            }
            if (!more) break;
            __syncwarp();
            }
            }
        }
    }
    // the last survivors of this warp
    if (RING && pend > 0) {
        __syncwarp();
        phase2<LOG>(P, lut, lane < pend, ring_ra[lane], ring_cb[lane], ring_e[lane], rec_c, W, lane, lt, lg);
    }
    for (int o = 16; o > 0; o >>= 1) cand += __shfl_xor_sync(0xffffffffu, cand, o);
    if (lane == 0 && cand) atomicAdd(P.cand_count, cand);
    if (lane == 0 && exam) atomicAdd(P.exam_count, exam);
    if (LOG) {
        __syncthreads();
        for (int i = threadIdx.x; i < P.n_ops * LOG_FIELDS; i += blockDim.x)
            if (lgs[i]) atomicAdd(&P.log[i], lgs[i]);
    }
}

// Per-pair timing of one program op (the paper's T_p(t1, t2) that its shallow
// model N learns): each given pair has a warp of its own, whose lane 0
// evaluates op k and records the clock64 cycles (no other lane's divergence
// enters them), the verdict and N's 8 input features (kind one-hot,
// threshold, the two operands, their difference and min/max ratio).
__global__ void k_pair_times(const __grid_constant__ EvalParams P, int k, const uint32_t *pi, const uint32_t *pj,
                             int n, uint32_t *cycles, uint8_t *verdict, float *X) {
    const int t = (int)(((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    if ((threadIdx.x & 31) != 0 || t >= n) return;
    const uint32_t *a = P.rec_r + (size_t)pi[t] * P.W;
    const uint32_t *b = (P.self_join ? P.rec_r : P.rec_s) + (size_t)pj[t] * P.W;
    const Op &op = P.ops[k];
    LogAcc lg{nullptr};
    const long long c0 = clock64();
    const bool r = eval_op<false>(P, k, a, b, lg);
    const long long c1 = clock64();
    cycles[t] = (uint32_t)min(c1 - c0, 0x7fffffffll);
    verdict[t] = r ? 1 : 0;
    float *f = X + (size_t)t * 8;
    f[0] = op.kind == OP_ED ? 1.f : 0.f;
    f[1] = op.kind == OP_JAC ? 1.f : 0.f;
    f[2] = op.kind == OP_ABS ? 1.f : 0.f;
    f[3] = op.kind == OP_ED ? op.k / 8.f : op.kind == OP_JAC ? (float)op.num / (float)op.den : log1pf(op.delta);
    const uint32_t x1 = a[op.feat], x2 = b[op.feat];
    bool miss;
    float o1, o2;
    if (op.kind == OP_ABS) {
        o1 = __uint_as_float(x1);
        o2 = __uint_as_float(x2);
        miss = isnan(o1) || isnan(o2);
    } else {
        miss = x1 == NULL_LEN || x2 == NULL_LEN;
        o1 = (float)x1;
        o2 = (float)x2;
    }
    if (miss) {
        f[4] = f[5] = f[6] = f[7] = -1.f;
        return;
    }
    const float a1 = fabsf(o1), a2 = fabsf(o2), d = fabsf(o1 - o2);
    if (op.kind == OP_ABS) {
        f[4] = log1pf(a1) / 8.f;
        f[5] = log1pf(a2) / 8.f;
        f[6] = log1pf(d) / 8.f;
    } else {
        f[4] = o1 / 64.f;
        f[5] = o2 / 64.f;
        f[6] = d / 64.f;
    }
    const float mx = fmaxf(a1, a2);
    f[7] = mx > 0.f ? fminf(a1, a2) / mx : 0.f;
}

__global__ void k_pack_pairs(const uint64_t *keys, int64_t n, int key_bits_s, hb_pair *out) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const uint64_t k = keys[i];
    hb_pair p;
    p.tid1 = (uint32_t)(k >> key_bits_s);
    p.tid2 = (uint32_t)(k & ((1ull << key_bits_s) - 1ull));
    out[i] = p;
}

}  // namespace

size_t eval_smem_bytes(int HW, int n_eq, int use_lut, int tile) {
    const size_t T = (size_t)tile;
    size_t lut = use_lut ? (size_t)8 << n_eq : 0;
    return lut + (size_t)EV_WARPS * (T * (HW + 1) + T * HW + 2 * T + T * T / 8 + 3 * RING_SLOTS) * 4;
}

template <int R, bool LOG, bool MULTI, bool RING>
static int occupancy1(size_t smem) {
    int nb = 0;
    cudaFuncSetAttribute(k_eval<R, LOG, MULTI, RING>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_eval<R, LOG, MULTI, RING>, EV_THREADS, smem);
    return nb;
}

// the smallest occupancy over the instantiations a launch may pick
template <int R, bool LOG>
static int occupancy(size_t smem) {
    int nb = std::min(occupancy1<R, LOG, false, false>(smem), occupancy1<R, LOG, true, false>(smem));
    if constexpr (!LOG)
        nb = std::min(nb, std::min(occupancy1<R, LOG, false, true>(smem), occupancy1<R, LOG, true, true>(smem)));
    return nb;
}

int eval_blocks_per_sm(int tile, int logging, size_t smem) {
    if (tile == 64) return logging ? occupancy<2, true>(smem) : occupancy<2, false>(smem);
    return logging ? occupancy<1, true>(smem) : occupancy<1, false>(smem);
}

template <int R, bool LOG>
static void launch(const EvalParams &p, bool multi, bool ring, int grid, size_t smem, cudaStream_t s) {
    if constexpr (LOG) {
        if (multi) k_eval<R, true, true, false><<<grid, EV_THREADS, smem, s>>>(p);
        else k_eval<R, true, false, false><<<grid, EV_THREADS, smem, s>>>(p);
    } else {
        if (multi && ring) k_eval<R, false, true, true><<<grid, EV_THREADS, smem, s>>>(p);
        else if (multi) k_eval<R, false, true, false><<<grid, EV_THREADS, smem, s>>>(p);
        else if (ring) k_eval<R, false, false, true><<<grid, EV_THREADS, smem, s>>>(p);
        else k_eval<R, false, false, false><<<grid, EV_THREADS, smem, s>>>(p);
    }
}

cudaError_t launch_eval(const EvalParams &p, int grid, size_t smem, int logging, cudaStream_t s) {
    HB_LAUNCHED(1);
    const bool multi = p.multi != 0, ring = p.refine != 0;
    if (p.tile == 64) {
        if (logging) launch<2, true>(p, multi, ring, grid, smem, s);
        else launch<2, false>(p, multi, ring, grid, smem, s);
    } else {
        if (logging) launch<1, true>(p, multi, ring, grid, smem, s);
        else launch<1, false>(p, multi, ring, grid, smem, s);
    }
    return cudaGetLastError();
}

cudaError_t launch_pair_times(const EvalParams &p, int k, const uint32_t *pi, const uint32_t *pj, int n,
                              uint32_t *cycles, uint8_t *verdict, float *X, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    HB_LAUNCHED(1);
    k_pair_times<<<(unsigned)((n + 3) / 4), 128, 0, s>>>(p, k, pi, pj, n, cycles, verdict, X);   // 4 pairs a block
    return cudaGetLastError();
}

void pack_pairs(const uint64_t *keys, int64_t n, int key_bits_s, hb_pair *out, cudaStream_t s) {
    if (n <= 0) return;
    HB_LAUNCHED(1);
    k_pack_pairs<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(keys, n, key_bits_s, out);
}

HB_ERROR_READER(checked_error_eval)

}  // namespace hb
