// Device-wide exclusive scan and LSD radix sort (keys only), written for the
// block builder (slot offsets, tile prefixes) and for the final ordering of
// the candidate pairs.  Element counts may live in device memory so that the
// whole blocking sequence runs without a host round trip.
#include <cuda_runtime.h>
#include <stdint.h>

#include "hb_internal.h"

namespace hb {
namespace {

constexpr int SCAN_THREADS = 256;
constexpr int SCAN_ITEMS = 8;
constexpr int SCAN_TILE = SCAN_THREADS * SCAN_ITEMS;

__device__ __forceinline__ int64_t eff_n(int64_t n_max, const uint32_t *n_dev) {
    if (!n_dev) return n_max;
    int64_t v = (int64_t)*n_dev;
    return v < n_max ? v : n_max;
}

template <typename T>
__device__ __forceinline__ T block_exclusive(T v, T *warp_sums, T *total) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    T x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        T y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) warp_sums[wid] = x;
    __syncthreads();
    if (wid == 0) {
        T w = lane < (SCAN_THREADS / 32) ? warp_sums[lane] : T(0);
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            T y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += y;
        }
        if (lane < (SCAN_THREADS / 32)) warp_sums[lane] = w;
    }
    __syncthreads();
    T before = (wid > 0 ? warp_sums[wid - 1] : T(0)) + x - v;
    if (total) *total = warp_sums[SCAN_THREADS / 32 - 1];
    __syncthreads();
    return before;
}

// tile sums; element i >= n counts as zero; covers n_max + 1 elements
template <typename T>
__global__ void k_scan_reduce(const T *in, int64_t n_max, const uint32_t *n_dev, T *partial) {
    __shared__ T ws[SCAN_THREADS / 32];
    const int64_t n = eff_n(n_max, n_dev);
    const int64_t base = (int64_t)blockIdx.x * SCAN_TILE;
    T s = 0;
    for (int i = threadIdx.x; i < SCAN_TILE; i += SCAN_THREADS) {
        int64_t g = base + i;
        if (g < n) s += in[g];
    }
    T tot;
    block_exclusive<T>(s, ws, &tot);
    if (threadIdx.x == 0) partial[blockIdx.x] = tot;
}

// out[i] = sum in[0..i) for i in [0, n_max]; partial[] holds exclusive tile offsets (or null)
template <typename T>
__global__ void k_scan_down(const T *in, T *out, int64_t n_max, const uint32_t *n_dev, const T *partial) {
    __shared__ T tile[SCAN_TILE];
    __shared__ T ws[SCAN_THREADS / 32];
    const int64_t n = eff_n(n_max, n_dev);
    const int64_t base = (int64_t)blockIdx.x * SCAN_TILE;
    for (int i = threadIdx.x; i < SCAN_TILE; i += SCAN_THREADS) {
        int64_t g = base + i;
        tile[i] = (g < n) ? in[g] : T(0);
    }
    __syncthreads();
    T local[SCAN_ITEMS];
    T s = 0;
#pragma unroll
    for (int k = 0; k < SCAN_ITEMS; k++) {
        local[k] = s;
        s += tile[threadIdx.x * SCAN_ITEMS + k];
    }
    T before = block_exclusive<T>(s, ws, nullptr);
    T off = partial ? partial[blockIdx.x] : T(0);
#pragma unroll
    for (int k = 0; k < SCAN_ITEMS; k++) tile[threadIdx.x * SCAN_ITEMS + k] = local[k] + before + off;
    __syncthreads();
    for (int i = threadIdx.x; i < SCAN_TILE; i += SCAN_THREADS) {
        int64_t g = base + i;
        if (g <= n_max) out[g] = tile[i];
    }
}

template <typename T>
size_t scan_tmp_elems(int64_t n) {
    int64_t tiles = (n + 1 + SCAN_TILE - 1) / SCAN_TILE;
    if (tiles <= 1) return 0;
    return (size_t)(tiles + 1) + scan_tmp_elems<T>(tiles);
}

template <typename T>
void scan_impl(const T *in, T *out, int64_t n, const uint32_t *n_dev, T *tmp, cudaStream_t s) {
    int64_t tiles = (n + 1 + SCAN_TILE - 1) / SCAN_TILE;
    if (tiles <= 1) {
        HB_LAUNCHED(1);
        k_scan_down<T><<<1, SCAN_THREADS, 0, s>>>(in, out, n, n_dev, nullptr);
        return;
    }
    T *partial = tmp;
    T *partial_scan = tmp;   // scanned in place (exclusive), size tiles + 1
    HB_LAUNCHED(1);
    k_scan_reduce<T><<<(unsigned)tiles, SCAN_THREADS, 0, s>>>(in, n, n_dev, partial);
    scan_impl<T>(partial, partial_scan, tiles, nullptr, tmp + tiles + 1, s);
    HB_LAUNCHED(1);
    k_scan_down<T><<<(unsigned)tiles, SCAN_THREADS, 0, s>>>(in, out, n, n_dev, partial_scan);
}

// ------------------------------------------------------------------ radix sort
constexpr int RS_THREADS = 256;
constexpr int RS_ITEMS = 8;
constexpr int RS_TILE = RS_THREADS * RS_ITEMS;
constexpr int RS_WARPS = RS_THREADS / 32;

__device__ __forceinline__ int64_t eff_n64(int64_t n_max, const unsigned long long *n_dev) {
    if (!n_dev) return n_max;
    int64_t v = (int64_t)*n_dev;
    return v < n_max ? v : n_max;
}

__global__ void k_radix_hist(const uint64_t *keys, int64_t n_max, const unsigned long long *n_dev, int shift,
                             uint32_t *hist, int64_t ntiles) {
    __shared__ uint32_t h[256];
    const int64_t n = eff_n64(n_max, n_dev);
    h[threadIdx.x] = 0;
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * RS_TILE;
    for (int i = threadIdx.x; i < RS_TILE; i += RS_THREADS) {
        int64_t g = base + i;
        if (g < n) atomicAdd(&h[(keys[g] >> shift) & 255u], 1u);
    }
    __syncthreads();
    hist[(int64_t)threadIdx.x * ntiles + blockIdx.x] = h[threadIdx.x];
}

__global__ void __launch_bounds__(RS_THREADS) k_radix_scatter(const uint64_t *keys, uint64_t *out, int64_t n_max,
                                                               const unsigned long long *n_dev, int shift,
                                                               const uint32_t *offsets, int64_t ntiles) {
    __shared__ uint64_t sk[RS_TILE];
    __shared__ uint64_t sorted[RS_TILE];
    __shared__ uint32_t wc[RS_WARPS][256];
    __shared__ uint32_t pref[256], run[256], goff[256], hcount[256];
    const int64_t n = eff_n64(n_max, n_dev);
    const int64_t base = (int64_t)blockIdx.x * RS_TILE;
    if (base >= n) return;
    const int m = (int)((n - base) < RS_TILE ? (n - base) : RS_TILE);
    const int t = threadIdx.x, lane = t & 31, w = t >> 5;
    hcount[t] = 0;
    run[t] = 0;
    goff[t] = offsets[(int64_t)t * ntiles + blockIdx.x];
    for (int k = 0; k < RS_WARPS; k++) wc[k][t] = 0;
    __syncthreads();
    for (int i = t; i < m; i += RS_THREADS) {
        uint64_t k = keys[base + i];
        sk[i] = k;
        atomicAdd(&hcount[(k >> shift) & 255u], 1u);
    }
    __syncthreads();
    // tile-local exclusive prefix of the digit counts (one thread per digit, warp scan)
    {
        uint32_t v = hcount[t], x = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        __shared__ uint32_t wsum[RS_WARPS];
        if (lane == 31) wsum[w] = x;
        __syncthreads();
        uint32_t add = 0;
        for (int k = 0; k < w; k++) add += wsum[k];
        pref[t] = add + x - v;
    }
    __syncthreads();
    const unsigned lt = (1u << lane) - 1u;
    for (int r = 0; r < RS_ITEMS; r++) {
        const int e = r * RS_THREADS + t;
        const bool valid = e < m;
        uint64_t key = valid ? sk[e] : 0;
        uint32_t d = valid ? (uint32_t)((key >> shift) & 255u) : (256u + (uint32_t)lane);
        unsigned peers = __match_any_sync(0xffffffffu, d);
        uint32_t rank = __popc(peers & lt);
        if (valid && rank == 0) wc[w][d] = __popc(peers);
        __syncthreads();
        {
            uint32_t acc = run[t];
#pragma unroll
            for (int k = 0; k < RS_WARPS; k++) {
                uint32_t c = wc[k][t];
                wc[k][t] = acc;
                acc += c;
            }
            run[t] = acc;
        }
        __syncthreads();
        if (valid) sorted[pref[d] + wc[w][d] + rank] = key;
        __syncthreads();
#pragma unroll
        for (int k = 0; k < RS_WARPS; k++) wc[k][t] = 0;
        __syncthreads();
    }
    for (int i = t; i < m; i += RS_THREADS) {
        uint64_t key = sorted[i];
        uint32_t d = (uint32_t)((key >> shift) & 255u);
        out[goff[d] + (uint32_t)i - pref[d]] = key;
    }
}

}  // namespace

size_t scan_tmp_bytes(int64_t n) { return scan_tmp_elems<uint64_t>(n) * sizeof(uint64_t) + 256; }

void scan_exclusive_u32(const uint32_t *in, uint32_t *out, int64_t n, const uint32_t *n_dev, void *tmp,
                        size_t tmp_bytes, cudaStream_t s) {
    (void)tmp_bytes;
    scan_impl<uint32_t>(in, out, n, n_dev, static_cast<uint32_t *>(tmp), s);
}

void scan_exclusive_u64(const uint64_t *in, uint64_t *out, int64_t n, const uint32_t *n_dev, void *tmp,
                        size_t tmp_bytes, cudaStream_t s) {
    (void)tmp_bytes;
    scan_impl<uint64_t>(in, out, n, n_dev, static_cast<uint64_t *>(tmp), s);
}

size_t radix_tmp_bytes(int64_t n) {
    int64_t ntiles = (n + RS_TILE - 1) / RS_TILE;
    if (ntiles < 1) ntiles = 1;
    int64_t h = 256 * ntiles;
    return (size_t)(2 * (h + 1)) * sizeof(uint32_t) + scan_tmp_bytes(h) + 512;
}

void radix_sort_u64(uint64_t *keys, uint64_t *alt, int64_t n_max, const unsigned long long *n_dev, int bits,
                    void *tmp, size_t tmp_bytes, cudaStream_t s, uint64_t **result) {
    (void)tmp_bytes;
    int64_t ntiles = (n_max + RS_TILE - 1) / RS_TILE;
    if (ntiles < 1) ntiles = 1;
    int64_t h = 256 * ntiles;
    uint32_t *hist = static_cast<uint32_t *>(tmp);
    uint32_t *offs = hist + (h + 1);
    void *stmp = reinterpret_cast<char *>(tmp) + (size_t)(2 * (h + 1)) * sizeof(uint32_t);
    stmp = reinterpret_cast<void *>((reinterpret_cast<uintptr_t>(stmp) + 255) & ~uintptr_t(255));
    uint64_t *src = keys, *dst = alt;
    for (int shift = 0; shift < bits; shift += 8) {
        HB_LAUNCHED(1);
        k_radix_hist<<<(unsigned)ntiles, RS_THREADS, 0, s>>>(src, n_max, n_dev, shift, hist, ntiles);
        scan_impl<uint32_t>(hist, offs, h, nullptr, static_cast<uint32_t *>(stmp), s);
        HB_LAUNCHED(1);
        k_radix_scatter<<<(unsigned)ntiles, RS_THREADS, 0, s>>>(src, dst, n_max, n_dev, shift, offs, ntiles);
        uint64_t *x = src;
        src = dst;
        dst = x;
    }
    *result = src;
}

}  // namespace hb
