// Integer issue-rate probe: the measured ceiling the evaluation kernel's
// integer work is compared against.
//
// Every thread runs CHAINS independent dependency chains; each step of a
// chain is a three-input add, a shift and a three-input logic operation
// (x = x + y + i; x ^= (x >> 7) ^ y), i.e. three integer instructions, so the
// schedulers always have independent work and the rate is bound by issue, not
// by latency.  The grid fills every SM with 8 resident 256-thread blocks.
// The result is folded into one word per thread so nothing can be removed.
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "hb_internal.h"

namespace hb {
hb_status fail(hb_status st, const std::string &msg);
namespace {

constexpr int PROBE_THREADS = 256;
constexpr int PROBE_CHAINS = 8;
constexpr int PROBE_OPS_PER_STEP = 3;

__global__ void __launch_bounds__(PROBE_THREADS) k_int_probe(uint32_t seed, int iters, uint32_t *out) {
    const uint32_t tid = blockIdx.x * blockDim.x + threadIdx.x;
    uint32_t x[PROBE_CHAINS], y[PROBE_CHAINS];
#pragma unroll
    for (int c = 0; c < PROBE_CHAINS; c++) {
        x[c] = seed ^ (tid * 0x9E3779B9u + (uint32_t)c);
        y[c] = (seed + (uint32_t)c) * 0x85EBCA6Bu ^ tid;
    }
    for (int i = 0; i < iters; i++) {
#pragma unroll
        for (int c = 0; c < PROBE_CHAINS; c++) {
            x[c] = x[c] + y[c] + (uint32_t)i;
            x[c] = x[c] ^ (x[c] >> 7) ^ y[c];
        }
    }
    uint32_t r = 0;
#pragma unroll
    for (int c = 0; c < PROBE_CHAINS; c++) r ^= x[c];
    out[tid] = r;
}

}  // namespace
}  // namespace hb

extern "C" hb_status hb_probe_int_issue(int32_t iters, double *ops_per_s, double *ms_out, void *stream) {
    using namespace hb;
    if (iters < 1 || !ops_per_s) return fail(HB_ERR_ARG, "hb_probe_int_issue: iters >= 1 and ops_per_s required");
    int dev = 0, n_sm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return fail(HB_ERR_CUDA, std::string("hb_probe_int_issue: ") + cudaGetErrorString(e));
    const unsigned grid = (unsigned)n_sm * 8u;
    const size_t threads = (size_t)grid * PROBE_THREADS;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    uint32_t *out = nullptr;
    cudaEvent_t a = nullptr, b = nullptr;
    e = cudaMallocAsync(&out, threads * sizeof(uint32_t), s);
    if (e == cudaSuccess) e = cudaEventCreate(&a);
    if (e == cudaSuccess) e = cudaEventCreate(&b);
    float ms = 0.f;
    if (e == cudaSuccess) {
        HB_LAUNCHED(2);
        k_int_probe<<<grid, PROBE_THREADS, 0, s>>>(1u, iters / 8 + 1, out);   // warm-up (clocks up)
        cudaEventRecord(a, s);
        k_int_probe<<<grid, PROBE_THREADS, 0, s>>>(2u, iters, out);
        cudaEventRecord(b, s);
        e = cudaEventSynchronize(b);
        if (e == cudaSuccess) e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, a, b);
    }
    if (out) cudaFreeAsync(out, s);
    if (a) cudaEventDestroy(a);
    if (b) cudaEventDestroy(b);
    if (e != cudaSuccess) return fail(HB_ERR_CUDA, std::string("hb_probe_int_issue: ") + cudaGetErrorString(e));
    const double ops = (double)threads * (double)iters * PROBE_CHAINS * PROBE_OPS_PER_STEP;
    *ops_per_s = ops / (ms * 1e-3);
    if (ms_out) *ms_out = ms;
    return HB_OK;
}
