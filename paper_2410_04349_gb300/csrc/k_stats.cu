// Planner statistics on a sample of tuples (Section 4.2, "Effectiveness"):
// per predicate, the attribute values of sampled tuples are hashed into k
// buckets with a locality-sensitive hash, so that equal or similar values
// tend to share a bucket; the spread of the bucket counts gives sp(p, D).
//   equality / prefix : the (prefix of the) value itself
//   edit distance     : MinHash over 3-grams
//   q-gram Jaccard    : MinHash over q-grams
//   |a - b| <= delta  : floor(a / delta)
// The same pass records the sampled string lengths and q-gram counts that
// the cost model and the learned model use.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "hb_internal.h"

namespace hb {

namespace {

__device__ __forceinline__ uint64_t smix(uint64_t x) {
    x ^= x >> 31;
    x *= 0x7fb5d329728ea185ull;
    x ^= x >> 27;
    x *= 0x81dadef4bc2dd44dull;
    x ^= x >> 33;
    return x;
}

__device__ __forceinline__ uint64_t shash_bytes(const uint8_t *p, uint32_t n) {
    uint64_t h = 0xcbf29ce484222325ull ^ n;
    for (uint32_t i = 0; i < n; i++) h = (h ^ p[i]) * 0x100000001b3ull;
    return smix(h);
}

// (the number of sampled values present is the sum of a predicate's bucket
// counts: the host adds them up, instead of every sample adding one to a
// single counter)
__global__ void k_lsh_hist(const SampleSpec *specs, int n_preds, int64_t n_rows, int n_samples, int k_buckets,
                           uint32_t *hist, uint32_t *lens, uint32_t *grams, int n_keep) {
    const int p = blockIdx.y;
    const SampleSpec sp = specs[p];
    for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < n_samples; s += gridDim.x * blockDim.x) {
        const int64_t i = (int64_t)((double)s * (double)n_rows / (double)n_samples);
        if (sp.valid && !sp.valid[i]) {
            if (s < n_keep) {
                lens[(int64_t)p * n_keep + s] = NULL_LEN;
                grams[(int64_t)p * n_keep + s] = NULL_LEN;
            }
            continue;
        }
        uint64_t h = 0;
        uint32_t len = 0, ng = 0;
        if (sp.type == HB_COL_STRING) {
            const uint8_t *b = sp.bytes + sp.off[i];
            len = sp.off[i + 1] - sp.off[i];
            if (sp.kind == HB_P_EQ || sp.kind == HB_P_EQ_PREFIX) {
                uint32_t l = (sp.kind == HB_P_EQ_PREFIX && len > (uint32_t)sp.prefix) ? (uint32_t)sp.prefix : len;
                h = shash_bytes(b, l);
            } else {
                const int q = sp.q > 0 ? sp.q : 3;
                if (len < (uint32_t)q) {
                    h = shash_bytes(b, len);
                } else {
                    uint64_t mn = ~0ull;
                    ng = len - q + 1;
                    for (uint32_t j = 0; j + q <= len; j++) {
                        uint32_t g = 0;
                        for (int t = 0; t < q; t++) g = (g << 8) | b[j + t];
                        uint64_t v = smix(0x9E3779B97F4A7C15ull ^ g);
                        mn = v < mn ? v : mn;
                    }
                    h = smix(mn);
                }
            }
        } else if (sp.type == HB_COL_INT32) {
            h = smix((uint64_t)(uint32_t)static_cast<const int32_t *>(sp.vals)[i] + 0x1234567ull);
        } else {
            const float x = static_cast<const float *>(sp.vals)[i];
            if (isnan(x)) continue;
            double cell = sp.delta > 0.f ? floor((double)x / (double)sp.delta) : (double)x;
            h = smix((uint64_t)(int64_t)cell);
        }
        atomicAdd(&hist[(int64_t)p * k_buckets + (h % (uint64_t)k_buckets)], 1u);
        if (s < n_keep) {
            lens[(int64_t)p * n_keep + s] = len;
            grams[(int64_t)p * n_keep + s] = ng;
        }
    }
}

}  // namespace

void lsh_hist(const SampleSpec *specs_dev, int n_preds, int64_t n_rows, int n_samples, int k_buckets,
              uint32_t *hist, uint32_t *lens, uint32_t *grams, int n_keep, cudaStream_t s) {
    if (n_preds == 0 || n_rows == 0) return;
    dim3 grid((unsigned)((n_samples + 255) / 256), (unsigned)n_preds);
    HB_LAUNCHED(1);
    k_lsh_hist<<<grid, 256, 0, s>>>(specs_dev, n_preds, n_rows, n_samples, k_buckets, hist, lens, grams, n_keep);
}

}  // namespace hb
