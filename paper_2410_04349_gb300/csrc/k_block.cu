// Block builder.  For every MD, tuples that agree on all of its equality keys
// form one block (a pair can satisfy the MD's precondition only inside one).
// Groups are found with an exact open-addressing table over the tuples'
// equality codes; members are laid out per group by a counting sort; every
// group with a pair to compare becomes a block with its tile count.
//
// Small blocks of a self-join (2..SMALL_MAX tuples) are packed: blocks of one
// size n are listed together (their member starts, by size class), and every
// group of floor(T / n) of them becomes one packed tile, whose rows and
// columns are those blocks' members side by side and whose valid pairs stay
// inside each block.
#include <cuda_runtime.h>
#include <stdint.h>

#include "hb_internal.h"

namespace hb {
namespace {

constexpr int BT = 256;
constexpr uint32_t NO_SLOT = 0xFFFFFFFFu;

struct KeyWords {
    int32_t w[MAX_EQ];
    int32_t n;
};

__device__ __forceinline__ uint64_t mixk(uint64_t h, uint32_t v) {
    h ^= (uint64_t)v + 0x9E3779B97F4A7C15ull + (h << 6) + (h >> 2);
    h *= 0xff51afd7ed558ccdull;
    return h ^ (h >> 32);
}

__device__ __forceinline__ bool key_of(const uint32_t *rec, int W, int64_t i, const KeyWords &kw, uint64_t &h) {
    h = 0x243F6A8885A308D3ull;
    for (int e = 0; e < kw.n; e++) {
        uint32_t c = rec[i * W + kw.w[e]];
        if (c >= NOMATCH_CODE) return false;
        h = mixk(h, c);
    }
    return true;
}

__device__ __forceinline__ bool keys_equal(const uint32_t *ra, int64_t i, const uint32_t *rb, int64_t j, int W,
                                           const KeyWords &kw) {
    for (int e = 0; e < kw.n; e++)
        if (ra[i * W + kw.w[e]] != rb[j * W + kw.w[e]]) return false;
    return true;
}

__global__ void k_group_insert(const uint32_t *rec, int W, int64_t n, KeyWords kw, uint64_t *table, uint64_t mask,
                               uint32_t *slot_out) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    if (kw.n == 0) {   // an MD without equality predicates: one group holding every tuple
        slot_out[i] = 0;
        return;
    }
    uint64_t h;
    if (!key_of(rec, W, i, kw, h)) {
        slot_out[i] = NO_SLOT;
        return;
    }
    uint32_t h32 = (uint32_t)(h >> 32);
    uint64_t mine = ((uint64_t)h32 << 32) | (uint64_t)(uint32_t)i;
    uint64_t slot = h & mask;
    for (uint64_t probe = 0; probe <= mask; probe++) {
        uint64_t cur = table[slot];
        if (cur == EMPTY_SLOT) {
            uint64_t prev = atomicCAS(reinterpret_cast<unsigned long long *>(table + slot),
                                      (unsigned long long)EMPTY_SLOT, (unsigned long long)mine);
            if (prev == EMPTY_SLOT) {
                slot_out[i] = (uint32_t)slot;
                return;
            }
            cur = prev;
        }
        if ((uint32_t)(cur >> 32) == h32 && keys_equal(rec, i, rec, (int64_t)(uint32_t)cur, W, kw)) {
            slot_out[i] = (uint32_t)slot;
            return;
        }
        slot = (slot + 1) & mask;
    }
    slot_out[i] = NO_SLOT;
}

__global__ void k_group_probe(const uint32_t *rec, int64_t n, const uint32_t *rec_owner, int W, KeyWords kw,
                              const uint64_t *table, uint64_t mask, uint32_t *slot_out) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    if (kw.n == 0) {
        slot_out[i] = 0;
        return;
    }
    uint64_t h;
    if (!key_of(rec, W, i, kw, h)) {
        slot_out[i] = NO_SLOT;
        return;
    }
    uint32_t h32 = (uint32_t)(h >> 32);
    uint64_t slot = h & mask;
    for (uint64_t probe = 0; probe <= mask; probe++) {
        uint64_t cur = table[slot];
        if (cur == EMPTY_SLOT) break;
        if ((uint32_t)(cur >> 32) == h32 && keys_equal(rec, i, rec_owner, (int64_t)(uint32_t)cur, W, kw)) {
            slot_out[i] = (uint32_t)slot;
            return;
        }
        slot = (slot + 1) & mask;
    }
    slot_out[i] = NO_SLOT;
}

// warp-aggregated increment: lanes with the same slot add once
__global__ void k_count_slots(const uint32_t *slot, int64_t n, uint32_t *count) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    uint32_t s = i < n ? slot[i] : NO_SLOT;
    unsigned peers = __match_any_sync(0xffffffffu, s);
    int lane = threadIdx.x & 31;
    if (s != NO_SLOT && (__ffs(peers) - 1) == lane) atomicAdd(&count[s], (uint32_t)__popc(peers));
}

__global__ void k_scatter_slots(const uint32_t *slot, int64_t n, const uint32_t *start, uint32_t *cursor,
                                uint32_t *members) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    uint32_t s = i < n ? slot[i] : NO_SLOT;
    unsigned peers = __match_any_sync(0xffffffffu, s);
    int lane = threadIdx.x & 31;
    int leader = __ffs(peers) - 1;
    uint32_t base = 0;
    if (s != NO_SLOT && leader == lane) base = atomicAdd(&cursor[s], (uint32_t)__popc(peers));
    base = __shfl_sync(0xffffffffu, base, leader);
    if (s != NO_SLOT) members[HB_IDX(start[s] + base + __popc(peers & ((1u << lane) - 1u)), n, 30)] = (uint32_t)i;
}

// ---- sharding the evaluation over several processes (one GPU each) ----
// A block (one MD's group of tuples that agree on its equality keys) belongs to
// one rank: shard_owner(md, the group's smallest row id), a function of the
// data alone, so every process assigns every block alike however its own
// dictionary and group slots were numbered.  The smallest row of each group:
// the lowest lane among a warp's lanes of one slot holds the smallest row
// (rows increase with the lane), which takes an atomic minimum.
__global__ void k_group_min(const uint32_t *slot, int64_t n, uint32_t *minrow) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const uint32_t s = i < n ? slot[i] : NO_SLOT;
    const unsigned peers = __match_any_sync(0xffffffffu, s);
    if (s != NO_SLOT && (__ffs(peers) - 1) == (int)(threadIdx.x & 31)) atomicMin(&minrow[s], (uint32_t)i);
}

// owner rank: the 32-bit finaliser of MurmurHash3 (Appleby) of the row id
// mixed with the MD index, modulo the number of ranks
__device__ __forceinline__ uint32_t shard_owner(uint32_t md, uint32_t row, uint32_t world) {
    uint32_t h = row ^ (md * 0x9E3779B9u);
    h ^= h >> 16;
    h *= 0x85EBCA6Bu;
    h ^= h >> 13;
    h *= 0xC2B2AE35u;
    h ^= h >> 16;
    return h % world;
}

// groups owned by another rank get no members: their blocks are not emitted
__global__ void k_shard_filter(uint32_t *count_r, uint32_t *count_s, const uint32_t *minrow, uint64_t cap,
                               uint32_t md, uint32_t rank, uint32_t world) {
    const int64_t sl = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (sl >= (int64_t)cap || count_r[sl] == 0) return;
    if (shard_owner(md, minrow[sl], world) != rank) {
        count_r[sl] = 0;
        if (count_s) count_s[sl] = 0;
    }
}

__device__ __forceinline__ uint64_t tiles_of(uint32_t nr, uint32_t ns, int self_join, int tile) {
    uint64_t a = (nr + tile - 1) / tile;
    if (self_join) return a * (a + 1) / 2;
    uint64_t b = (ns + tile - 1) / tile;
    return a * b;
}

__global__ void k_emit_blocks(const uint32_t *count_r, const uint32_t *start_r, const uint32_t *count_s,
                              const uint32_t *start_s, uint64_t cap, uint32_t md, int self_join,
                              uint32_t member_base_r, uint32_t member_base_s, int tile, BlockDesc *blocks,
                              uint64_t *tiles, uint32_t *n_blocks, uint32_t block_cap, unsigned int *overflow,
                              uint32_t small_max) {
    int64_t sl = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    bool keep = false;
    uint32_t nr = 0, ns = 0;
    if (sl < (int64_t)cap) {
        nr = count_r[sl];
        if (self_join) {
            ns = nr;
            keep = nr >= 2 && nr > small_max;   // smaller blocks are packed (k_emit_packed)
        } else {
            ns = count_s[sl];
            keep = nr >= 1 && ns >= 1;
        }
    }
    unsigned bal = __ballot_sync(0xffffffffu, keep);
    int lane = threadIdx.x & 31;
    uint32_t base = 0;
    if (lane == 0 && bal) base = atomicAdd(n_blocks, (uint32_t)__popc(bal));
    base = __shfl_sync(0xffffffffu, base, 0);
    if (keep) {
        uint32_t b = base + __popc(bal & ((1u << lane) - 1u));
        if (b >= block_cap) {
            atomicExch(overflow, 1u);
            return;
        }
        BlockDesc d;
        d.md = md;
        d.n_r = nr;
        d.start_r = member_base_r + start_r[sl];
        d.n_s = ns;
        d.start_s = self_join ? d.start_r : member_base_s + start_s[sl];
        d.packed = 0;
        blocks[b] = d;
        tiles[b] = tiles_of(nr, ns, self_join, tile);
    }
}

// ---- packing of small self-join blocks (metadata words: see SmallMeta)
struct SmallMeta {
    static constexpr int COUNT = 0;     // [n]: blocks of n tuples (this MD)
    static constexpr int OFF = 32;      // [n]: first entry of size class n in the start list
    static constexpr int CURSOR = 64;   // [n]: entries written so far
    static constexpr int TILES = 96;    // [n]: first packed tile of class n; [SMALL_MAX + 1]: this MD's total
};

__global__ void k_small_hist(const uint32_t *count, uint64_t cap, uint32_t *meta) {
    __shared__ uint32_t h[SMALL_MAX + 1];
    for (int t = threadIdx.x; t <= SMALL_MAX; t += blockDim.x) h[t] = 0;
    __syncthreads();
    const int64_t sl = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (sl < (int64_t)cap) {
        const uint32_t n = count[sl];
        if (n >= 2 && n <= (uint32_t)SMALL_MAX) atomicAdd(&h[n], 1u);
    }
    __syncthreads();
    for (int t = threadIdx.x; t <= SMALL_MAX; t += blockDim.x)
        if (h[t]) atomicAdd(&meta[SmallMeta::COUNT + t], h[t]);
}

// one thread: this MD's range of the start list (claimed with an atomic, so
// that MDs built at once get disjoint ranges), its class regions and
// packed-tile ranges
__global__ void k_small_plan(uint32_t *meta, int tile, uint32_t small_cap, unsigned int *overflow,
                             uint32_t *small_total) {
    uint32_t md_total = 0, tp = 0;
    for (int n = 2; n <= SMALL_MAX; n++) md_total += meta[SmallMeta::COUNT + n];
    uint32_t base = atomicAdd(small_total, md_total);
    if ((uint64_t)base + md_total > small_cap) {
        atomicExch(overflow, 1u);
        base = small_cap;   // every tile of this MD then fails the range check of k_emit_packed
    }
    for (int n = 2; n <= SMALL_MAX; n++) {
        const uint32_t cnt = meta[SmallMeta::COUNT + n];
        const uint32_t per = (uint32_t)(tile / n);
        meta[SmallMeta::OFF + n] = base;
        meta[SmallMeta::CURSOR + n] = 0;
        meta[SmallMeta::TILES + n] = tp;
        base += cnt;
        tp += (cnt + per - 1) / per;
    }
    meta[SmallMeta::TILES + SMALL_MAX + 1] = tp;
}

// (lanes of a warp holding blocks of one size take their positions with one
// atomic: the size classes' cursors are only 15 counters)
__global__ void k_small_scatter(const uint32_t *count, const uint32_t *start, uint64_t cap, uint32_t member_base,
                                uint32_t *meta, uint32_t *small, uint32_t small_cap) {
    const int64_t sl = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const uint32_t n = sl < (int64_t)cap ? count[sl] : 0u;
    const bool is_small = n >= 2 && n <= (uint32_t)SMALL_MAX;
    const unsigned peers = __match_any_sync(0xffffffffu, is_small ? n : 0u);
    if (!is_small) return;
    const int lane = threadIdx.x & 31, leader = __ffs(peers) - 1;
    uint32_t b = 0;
    if (lane == leader) b = atomicAdd(&meta[SmallMeta::CURSOR + n], (uint32_t)__popc(peers));
    b = __shfl_sync(peers, b, leader);
    const uint32_t pos = meta[SmallMeta::OFF + n] + b + (uint32_t)__popc(peers & ((1u << lane) - 1u));
    if (pos < small_cap) small[pos] = member_base + start[sl];
}

// one packed tile per work item: floor(T / n) blocks of size class n
__global__ void k_emit_packed(const uint32_t *meta, uint32_t md, int tile, BlockDesc *blocks, uint64_t *tiles,
                              uint32_t *n_blocks, uint32_t *n_packed, uint32_t block_cap, uint32_t small_cap,
                              unsigned int *overflow) {
    const uint32_t total = meta[SmallMeta::TILES + SMALL_MAX + 1];
    for (uint32_t q = blockIdx.x * blockDim.x + threadIdx.x; q < total; q += gridDim.x * blockDim.x) {
        int n = 2;
        while (n < SMALL_MAX && meta[SmallMeta::TILES + n + 1] <= q) n++;
        const uint32_t per = (uint32_t)(tile / n);
        const uint32_t first = (q - meta[SmallMeta::TILES + n]) * per;
        const uint32_t k = min(per, meta[SmallMeta::COUNT + n] - first);
        if ((uint64_t)meta[SmallMeta::OFF + n] + first + k > small_cap) {   // start list overflow: no tile
            atomicExch(overflow, 1u);
            continue;
        }
        const uint32_t b = atomicAdd(n_blocks, 1u);
        atomicAdd(n_packed, 1u);
        if (b >= block_cap) {
            atomicExch(overflow, 1u);
            continue;
        }
        BlockDesc d;
        d.md = md;
        d.n_r = k * (uint32_t)n;
        d.start_r = meta[SmallMeta::OFF + n] + first;
        d.n_s = d.n_r;
        d.start_s = d.start_r;
        d.packed = (uint32_t)n;
        blocks[b] = d;
        tiles[b] = 1;
    }
}

__global__ void k_clamp_blocks(uint32_t *n_blocks, uint32_t block_cap) {
    if (*n_blocks > block_cap) *n_blocks = block_cap;
}

inline unsigned nblk(int64_t n) { return (unsigned)(n > 0 ? (n + BT - 1) / BT : 1); }

}  // namespace

KeyWords make_keywords(const int32_t *eq_words, int n_keys) {
    KeyWords k;
    k.n = n_keys;
    for (int e = 0; e < MAX_EQ; e++) k.w[e] = e < n_keys ? eq_words[e] : 0;
    return k;
}

void group_build(const uint32_t *rec, int W, int64_t n, const int32_t *eq_words, int n_keys, uint64_t *table,
                 uint64_t cap, uint32_t *slot, cudaStream_t s) {
    if (n_keys > 0) cudaMemsetAsync(table, 0xFF, cap * sizeof(uint64_t), s);
    if (n == 0) return;
    HB_LAUNCHED(1);
    k_group_insert<<<nblk(n), BT, 0, s>>>(rec, W, n, make_keywords(eq_words, n_keys), table, cap - 1, slot);
}

void group_probe(const uint32_t *rec_probe, int64_t n, const uint32_t *rec_owner, int W, const int32_t *eq_words,
                 int n_keys, const uint64_t *table, uint64_t cap, uint32_t *slot, cudaStream_t s) {
    if (n == 0) return;
    HB_LAUNCHED(1);
    k_group_probe<<<nblk(n), BT, 0, s>>>(rec_probe, n, rec_owner, W, make_keywords(eq_words, n_keys), table,
                                         cap - 1, slot);
}

void count_slots(const uint32_t *slot, int64_t n, uint32_t *count, cudaStream_t s) {
    if (n == 0) return;
    HB_LAUNCHED(1);
    k_count_slots<<<nblk(n), BT, 0, s>>>(slot, n, count);
}

void scatter_slots(const uint32_t *slot, int64_t n, const uint32_t *start, uint32_t *cursor, uint32_t *members,
                   cudaStream_t s) {
    if (n == 0) return;
    HB_LAUNCHED(1);
    k_scatter_slots<<<nblk(n), BT, 0, s>>>(slot, n, start, cursor, members);
}

void shard_filter(const uint32_t *slot_r, int64_t n_r, uint32_t *count_r, uint32_t *count_s, uint32_t *minrow,
                  uint64_t cap, uint32_t md, uint32_t rank, uint32_t world, cudaStream_t s) {
    cudaMemsetAsync(minrow, 0xFF, sizeof(uint32_t) * (size_t)cap, s);
    HB_LAUNCHED(2);
    if (n_r > 0) k_group_min<<<nblk(n_r), BT, 0, s>>>(slot_r, n_r, minrow);
    k_shard_filter<<<nblk((int64_t)cap), BT, 0, s>>>(count_r, count_s, minrow, cap, md, rank, world);
}

void emit_blocks(const uint32_t *count_r, const uint32_t *start_r, const uint32_t *count_s, const uint32_t *start_s,
                 uint64_t cap, uint32_t md, int self_join, uint32_t member_base_r, uint32_t member_base_s, int tile,
                 BlockDesc *blocks, uint64_t *tiles, uint32_t *n_blocks, uint32_t block_cap, unsigned int *overflow,
                 cudaStream_t s) {
    HB_LAUNCHED(1);
    k_emit_blocks<<<nblk((int64_t)cap), BT, 0, s>>>(count_r, start_r, count_s, start_s, cap, md, self_join,
                                                    member_base_r, member_base_s, tile, blocks, tiles, n_blocks,
                                                    block_cap, overflow, 0u);
}

void emit_blocks_packed(const uint32_t *count_r, const uint32_t *start_r, uint64_t cap, uint32_t md,
                        uint32_t member_base_r, int tile, BlockDesc *blocks, uint64_t *tiles, uint32_t *n_blocks,
                        uint32_t *n_packed, uint32_t block_cap, unsigned int *overflow, uint32_t *small_meta,
                        uint32_t *small, uint32_t small_cap, uint32_t *small_total, int n_sm, cudaStream_t s) {
    cudaMemsetAsync(small_meta + SmallMeta::COUNT, 0, sizeof(uint32_t) * (SMALL_MAX + 1), s);
    HB_LAUNCHED(5);
    k_small_hist<<<nblk((int64_t)cap), BT, 0, s>>>(count_r, cap, small_meta);
    k_small_plan<<<1, 1, 0, s>>>(small_meta, tile, small_cap, overflow, small_total);
    k_small_scatter<<<nblk((int64_t)cap), BT, 0, s>>>(count_r, start_r, cap, member_base_r, small_meta, small,
                                                      small_cap);
    k_emit_blocks<<<nblk((int64_t)cap), BT, 0, s>>>(count_r, start_r, nullptr, nullptr, cap, md, 1, member_base_r, 0,
                                                    tile, blocks, tiles, n_blocks, block_cap, overflow,
                                                    (uint32_t)SMALL_MAX);
    k_emit_packed<<<(unsigned)(2 * n_sm), BT, 0, s>>>(small_meta, md, tile, blocks, tiles, n_blocks, n_packed,
                                                      block_cap, small_cap, overflow);
}

void clamp_blocks(uint32_t *n_blocks, uint32_t block_cap, cudaStream_t s) {
    HB_LAUNCHED(1);
    k_clamp_blocks<<<1, 1, 0, s>>>(n_blocks, block_cap);
}

HB_ERROR_READER(checked_error_block)

}  // namespace hb
