// Pair evaluation: the hot loop of blocking.
//
// Work items are tiles of a block's pair space (T x T tuples, upper triangle
// for a self-join).  A persistent grid of warps claims tiles from one atomic
// counter (task stealing in the form of a shared queue, Section 5.2).  A warp
// stages the packed records of its T row tuples and T column tuples in shared
// memory; each lane owns T/32 rows and walks the columns.  For every pair:
//
//   1. equality keys: bit e of E is set when the two tuples carry the same
//      (present) code of key e; the MDs whose equality keys are all in E are
//      alive (they cannot be excluded by an equality predicate);
//   2. owner check: the pair is handled only in the block of the lowest alive
//      MD, so every pair is evaluated once however many blocks contain it;
//   3. the sequential execution path of Section 5.1: non-equality predicates
//      in plan order, each evaluated once per pair (its result applies to
//      every MD holding it: "Reusing computation"), skipped when no alive MD
//      needs it, with a checkpoint after the last predicate of each MD;
//   4. witnessed pairs are compacted with a warp ballot and one atomic.
#include <cuda_runtime.h>
#include <stdint.h>

#include "hb_internal.h"

namespace hb {
namespace {

constexpr int EV_THREADS = 128;
constexpr int EV_WARPS = EV_THREADS / 32;
constexpr int LOG_FIELDS = 6;   // evaluated, passed, cycles, stage-1 passes, stage-2 passes, core work

struct LogAcc {
    unsigned long long *s;   // shared [MAX_OPS * LOG_FIELDS] or null
};

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
__device__ __forceinline__ bool eval_op(const EvalParams &P, int k, const uint32_t *a, const uint32_t *b,
                                        LogAcc &lg) {
    const Op &op = P.ops[k];
    const int f = op.feat;
    if (op.kind == OP_ABS) {
        const float x = __uint_as_float(a[f]), y = __uint_as_float(b[f]);
        return fabsf(x - y) <= op.delta;
    }
    if (op.kind == OP_ED) {
        const uint32_t la = a[f], lb = b[f];
        if (la == NULL_LEN || lb == NULL_LEN) return false;
        const uint32_t d = la > lb ? la - lb : lb - la;
        if (d > op.k) return false;
        if (LOG) atomicAdd(&lg.s[k * LOG_FIELDS + 3], 1ull);
        // bag distance over 16 character bins is a lower bound of the edit distance
        unsigned p1 = 0, p2 = 0;
#pragma unroll
        for (int w = 0; w < 4; w++) {
            const unsigned x = a[f + 2 + w], y = b[f + 2 + w];
            p1 = __dp4a(__vsubus4(x, y), 0x01010101u, p1);
            p2 = __dp4a(__vsubus4(y, x), 0x01010101u, p2);
        }
        if (max(p1, p2) > op.k) return false;
        if (LOG) atomicAdd(&lg.s[k * LOG_FIELDS + 4], 1ull);
        const uint8_t *sa = static_cast<const uint8_t *>(P.ptr_r[k]) + a[f + 1];
        const uint8_t *sb = static_cast<const uint8_t *>(P.ptr_s[k]) + b[f + 1];
        uint32_t rows = 0;
        bool r = ed_le(sa, (int)la, sb, (int)lb, op.k, rows);
        if (LOG) atomicAdd(&lg.s[k * LOG_FIELDS + 5], (unsigned long long)rows * (2ull * op.k + 1ull));
        return r;
    }
    // OP_JAC
    const uint32_t na = a[f], nb = b[f];
    if (na == NULL_LEN || nb == NULL_LEN) return false;
    const uint64_t num = op.num, den = op.den;
    const uint32_t mn = min(na, nb), mx = max(na, nb);
    if ((uint64_t)mn * den < num * mx) return false;   // J <= min/max
    if (LOG) atomicAdd(&lg.s[k * LOG_FIELDS + 3], 1ull);
    const uint64_t dn = den + num;
    const uint64_t need = num * ((uint64_t)na + nb);   // I*(den+num) >= num*(|A|+|B|)
    if (na <= 255u && nb <= 255u) {
        unsigned ub = 0;   // sum over 32 gram bins of min(count_a, count_b) >= |A n B|
#pragma unroll
        for (int w = 0; w < 8; w++) ub = __dp4a(__vminu4(a[f + 2 + w], b[f + 2 + w]), 0x01010101u, ub);
        if ((uint64_t)ub * dn < need) return false;
    }
    if (LOG) atomicAdd(&lg.s[k * LOG_FIELDS + 4], 1ull);
    const uint64_t imin = (need + dn - 1) / dn;
    if (imin == 0) return true;
    const uint32_t *A = static_cast<const uint32_t *>(P.ptr_r[k]) + a[f + 1];
    const uint32_t *B = static_cast<const uint32_t *>(P.ptr_s[k]) + b[f + 1];
    uint32_t i = 0, j = 0, I = 0;
    bool res = false;
    while (i < na && j < nb) {
        const uint32_t x = A[i], y = B[j];
        I += (x == y) ? 1u : 0u;
        i += (x <= y) ? 1u : 0u;
        j += (y <= x) ? 1u : 0u;
        if (I >= imin) {
            res = true;
            break;
        }
        if ((uint64_t)I + min(na - i, nb - j) < imin) break;
    }
    if (LOG) atomicAdd(&lg.s[k * LOG_FIELDS + 5], (unsigned long long)(i + j));
    return res;
}

template <bool LOG>
__device__ __forceinline__ bool run_program(const EvalParams &P, uint64_t alive, const uint32_t *a,
                                            const uint32_t *b, LogAcc &lg) {
    // profile mode (logging only): evaluate every predicate the initially alive
    // MDs hold, without early exit; the verdict is unchanged
    const bool prof = LOG && P.profile;
    const uint64_t alive0 = alive;
    bool hit = (alive & P.eqonly) != 0;
    if (hit && !prof) return true;
    for (int k = 0; k < P.n_ops; k++) {
        const uint64_t need = P.ops[k].need;
        if ((prof ? alive0 : alive) & need) {
            long long c0 = 0;
            if (LOG) c0 = clock64();
            bool r = eval_op<LOG>(P, k, a, b, lg);
            if (LOG) {
                atomicAdd(&lg.s[k * LOG_FIELDS + 0], 1ull);
                atomicAdd(&lg.s[k * LOG_FIELDS + 1], r ? 1ull : 0ull);
                atomicAdd(&lg.s[k * LOG_FIELDS + 2], (unsigned long long)(clock64() - c0));
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
    const double b2 = 2.0 * (double)nt + 1.0;
    int64_t i = (int64_t)floor((b2 - sqrt(b2 * b2 - 8.0 * (double)q)) * 0.5);
    if (i < 0) i = 0;
    if (i > nt - 1) i = nt - 1;
    auto start = [&](int64_t r) { return r * nt - r * (r - 1) / 2; };
    while (i + 1 < nt && start(i + 1) <= (int64_t)q) i++;
    while (i > 0 && start(i) > (int64_t)q) i--;
    ti = (uint32_t)i;
    tj = (uint32_t)(i + ((int64_t)q - start(i)));
}

template <int R, bool LOG>
__global__ void __launch_bounds__(EV_THREADS) k_eval(const __grid_constant__ EvalParams P) {
    extern __shared__ __align__(16) uint32_t smem[];
    constexpr int T = 32 * R;
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int W = P.W, WP = P.W + 1;
    uint64_t *lut = reinterpret_cast<uint64_t *>(smem);
    const int lut_words = P.use_lut ? 2 * (1 << P.n_eq) : 0;
    uint32_t *rows = smem + lut_words + wib * (2 * T * WP);
    uint32_t *cols = rows + T * WP;
    __shared__ unsigned long long lgs[LOG ? MAX_OPS * LOG_FIELDS : 1];
    LogAcc lg{lgs};
    if (P.use_lut)
        for (int i = threadIdx.x; i < (1 << P.n_eq); i += blockDim.x) lut[i] = P.lut[i];
    if (LOG)
        for (int i = threadIdx.x; i < MAX_OPS * LOG_FIELDS; i += blockDim.x) lgs[i] = 0;
    __syncthreads();

    const uint32_t nb = *P.n_blocks;
    const uint64_t total = P.tile_prefix[nb];
    const unsigned lt = (1u << lane) - 1u;
    unsigned long long cand = 0, exam = 0;

    for (;;) {
        unsigned long long t0 = 0;
        if (lane == 0) t0 = atomicAdd(P.tile_counter, (unsigned long long)P.claim);
        t0 = __shfl_sync(0xffffffffu, t0, 0);
        if (t0 >= total) break;
        const uint64_t t1 = min((uint64_t)t0 + (uint64_t)P.claim, total);
        uint32_t lo = 0, hi = nb;
        while (hi - lo > 1) {
            const uint32_t mid = (lo + hi) >> 1;
            if (P.tile_prefix[mid] <= t0) lo = mid;
            else hi = mid;
        }
        uint32_t bi = lo;
        for (uint64_t t = t0; t < t1; t++) {
            while (P.tile_prefix[bi + 1] <= t) bi++;
            const BlockDesc B = P.blocks[bi];
            uint32_t ti, tj;
            decode_tile(t - P.tile_prefix[bi], B.n_r, B.n_s, P.self_join, T, ti, tj);
            const uint32_t r0 = ti * T, c0 = tj * T;
            const int nr = (int)min((uint32_t)T, B.n_r - r0);
            const int nc = (int)min((uint32_t)T, B.n_s - c0);
            const bool diag = P.self_join && ti == tj;
            // stage row and column records (16-byte loads; W is a multiple of 4)
            uint32_t rid[R], cid[R];
#pragma unroll
            for (int rr = 0; rr < R; rr++) {
                const int r = rr * 32 + lane;
                rid[rr] = r < nr ? P.members_r[B.start_r + r0 + r] : 0u;
                cid[rr] = r < nc ? P.members_s[B.start_s + c0 + r] : 0u;
                if (r < nr) {
                    const uint4 *src = reinterpret_cast<const uint4 *>(P.rec_r + (size_t)rid[rr] * W);
                    uint32_t *dst = rows + r * WP;
                    for (int w4 = 0; w4 < (W >> 2); w4++) {
                        const uint4 v = src[w4];
                        dst[4 * w4 + 0] = v.x;
                        dst[4 * w4 + 1] = v.y;
                        dst[4 * w4 + 2] = v.z;
                        dst[4 * w4 + 3] = v.w;
                    }
                }
                if (r < nc) {
                    const uint4 *src = reinterpret_cast<const uint4 *>(
                        (P.self_join ? P.rec_r : P.rec_s) + (size_t)cid[rr] * W);
                    uint32_t *dst = cols + r * WP;
                    for (int w4 = 0; w4 < (W >> 2); w4++) {
                        const uint4 v = src[w4];
                        dst[4 * w4 + 0] = v.x;
                        dst[4 * w4 + 1] = v.y;
                        dst[4 * w4 + 2] = v.z;
                        dst[4 * w4 + 3] = v.w;
                    }
                }
            }
            __syncwarp();
#pragma unroll
            for (int rr = 0; rr < R; rr++) {
                const int r = rr * 32 + lane;
                const bool rv = r < nr;
                const uint32_t *ar = rows + r * WP;
                for (int c = 0; c < nc; c++) {
                    const uint32_t *bc = cols + c * WP;
                    const bool v = rv && (!diag || c > r);
                    uint32_t E = 0;
                    for (int e = 0; e < P.n_eq; e++) {
                        const uint32_t x = ar[e];
                        E |= (x == bc[e] && x < NOMATCH_CODE) ? (1u << e) : 0u;
                    }
                    uint64_t alive;
                    if (P.use_lut) {
                        alive = lut[E];
                    } else {
                        alive = 0;
                        for (int m = 0; m < P.n_md; m++)
                            alive |= ((E & P.eqset[m]) == P.eqset[m]) ? (1ull << m) : 0ull;
                    }
                    const bool own = v && alive != 0 && (uint32_t)(__ffsll((long long)alive) - 1) == B.md;
                    cand += __popc(__ballot_sync(0xffffffffu, own));
                    exam += __popc(__ballot_sync(0xffffffffu, v));
                    bool hit = false;
                    if (own) hit = run_program<LOG>(P, alive, ar, bc, lg);
                    const unsigned hm = __ballot_sync(0xffffffffu, hit);
                    if (hm) {
                        unsigned long long base = 0;
                        if (lane == 0) base = atomicAdd(P.out_count, (unsigned long long)__popc(hm));
                        base = __shfl_sync(0xffffffffu, base, 0);
                        // column id of column c: lane (c % 32) holds it in cid[c / 32]
                        uint32_t mycid = 0;
#pragma unroll
                        for (int q = 0; q < R; q++)
                            if (q == c / 32) mycid = cid[q];
                        const uint32_t colid = __shfl_sync(0xffffffffu, mycid, c & 31);
                        if (hit) {
                            const unsigned long long idx = base + __popc(hm & lt);
                            uint64_t key;
                            if (P.self_join) {
                                const uint32_t x = rid[rr], y = colid;
                                const uint32_t lo2 = x < y ? x : y, hi2 = x < y ? y : x;
                                key = ((uint64_t)lo2 << P.key_bits_s) | (uint64_t)hi2;
                            } else {
                                key = ((uint64_t)(rid[rr] + P.row_base) << P.key_bits_s) |
                                      (uint64_t)(colid + P.col_base);
                            }
                            if (idx < P.out_cap) P.out[idx] = key;
                        }
                    }
                }
            }
            __syncwarp();
        }
    }
    if (lane == 0 && cand) atomicAdd(P.cand_count, cand);
    if (lane == 0 && exam) atomicAdd(P.exam_count, exam);
    if (LOG) {
        __syncthreads();
        for (int i = threadIdx.x; i < P.n_ops * LOG_FIELDS; i += blockDim.x)
            if (lgs[i]) atomicAdd(&P.log[i], lgs[i]);
    }
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

size_t eval_smem_bytes(int W, int n_eq, int use_lut, int tile) {
    const int R = tile / 32;
    size_t lut = use_lut ? (size_t)8 << n_eq : 0;
    return lut + (size_t)EV_WARPS * 2 * (32 * R) * (W + 1) * 4;
}

template <int R, bool LOG>
static int occupancy(size_t smem) {
    int nb = 0;
    cudaFuncSetAttribute(k_eval<R, LOG>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_eval<R, LOG>, EV_THREADS, smem);
    return nb;
}

int eval_blocks_per_sm(int tile, int logging, size_t smem) {
    if (tile == 64) return logging ? occupancy<2, true>(smem) : occupancy<2, false>(smem);
    return logging ? occupancy<1, true>(smem) : occupancy<1, false>(smem);
}

cudaError_t launch_eval(const EvalParams &p, int grid, size_t smem, int logging, cudaStream_t s) {
    if (p.tile == 64) {
        HB_LAUNCHED(1);
        if (logging) k_eval<2, true><<<grid, EV_THREADS, smem, s>>>(p);
        else k_eval<2, false><<<grid, EV_THREADS, smem, s>>>(p);
    } else {
        HB_LAUNCHED(1);
        if (logging) k_eval<1, true><<<grid, EV_THREADS, smem, s>>>(p);
        else k_eval<1, false><<<grid, EV_THREADS, smem, s>>>(p);
    }
    return cudaGetLastError();
}

void pack_pairs(const uint64_t *keys, int64_t n, int key_bits_s, hb_pair *out, cudaStream_t s) {
    if (n <= 0) return;
    HB_LAUNCHED(1);
    k_pack_pairs<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(keys, n, key_bits_s, out);
}

}  // namespace hb
