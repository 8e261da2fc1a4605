// Cost-model MLP kernels (Section 4.2, "Shallow NNs"): 32 -> 64 -> 64 -> 1
// with ReLU, trained with mean squared error and Adam (Kingma & Ba).
// Parameters are one fp32 vector: W1[32][64], b1[64], W2[64][64], b2[64],
// W3[64], b3 (row-major, input index first).
//
// The network is tiny (6.3K weights, a few thousand rows), far below the
// size at which tensor cores pay off, so these are plain FMA kernels; the
// bf16 inference path rounds inputs, weights and hidden activations to
// bfloat16 and accumulates in fp32 (a bf16 x bf16 product is exact in fp32).
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>
#include <string>

#include "hb_internal.h"

namespace hb {
hb_status fail(hb_status st, const std::string &msg);
}

namespace hb {
namespace {

constexpr int D0 = 32, D1 = 64, D2 = 64;
constexpr int OFF_W1 = 0, OFF_B1 = OFF_W1 + D0 * D1, OFF_W2 = OFF_B1 + D1, OFF_B2 = OFF_W2 + D1 * D2,
              OFF_W3 = OFF_B2 + D2, OFF_B3 = OFF_W3 + D2, N_PARAMS = OFF_B3 + 1;
static_assert(N_PARAMS == HB_MLP_PARAMS, "parameter layout");
constexpr int ROWS = 32;   // rows per block

__device__ __forceinline__ float rb(float x, bool bf16) {
    return bf16 ? __bfloat162float(__float2bfloat16_rn(x)) : x;
}

// one block: ROWS rows; thread j (0..63) computes hidden unit j for every row.
// z1/z2 (optional) receive the pre-activations for the backward pass.
template <bool BF16>
__global__ void __launch_bounds__(64) k_mlp_fwd(const float *X, int n, const float *P, float *y, float *z1,
                                                float *z2) {
    __shared__ float xs[ROWS][D0];
    __shared__ float h1[ROWS][D1 + 1];
    __shared__ float h2[ROWS][D2 + 1];
    const int r0 = blockIdx.x * ROWS, j = threadIdx.x;
    for (int k = j; k < ROWS * D0; k += 64) {
        int r = k / D0, c = k % D0;
        xs[r][c] = (r0 + r < n) ? rb(X[(int64_t)(r0 + r) * D0 + c], BF16) : 0.f;
    }
    __syncthreads();
    {
        float w[D0];
#pragma unroll
        for (int i = 0; i < D0; i++) w[i] = rb(P[OFF_W1 + i * D1 + j], BF16);
        const float b = P[OFF_B1 + j];
        for (int r = 0; r < ROWS; r++) {
            float acc = b;
#pragma unroll
            for (int i = 0; i < D0; i++) acc = fmaf(xs[r][i], w[i], acc);
            if (z1 && r0 + r < n) z1[(int64_t)(r0 + r) * D1 + j] = acc;
            h1[r][j] = rb(fmaxf(acc, 0.f), BF16);
        }
    }
    __syncthreads();
    {
        const float b = P[OFF_B2 + j];
        for (int r = 0; r < ROWS; r++) {
            float acc = b;
            for (int i = 0; i < D1; i++) acc = fmaf(h1[r][i], rb(P[OFF_W2 + i * D2 + j], BF16), acc);
            if (z2 && r0 + r < n) z2[(int64_t)(r0 + r) * D2 + j] = acc;
            h2[r][j] = rb(fmaxf(acc, 0.f), BF16);
        }
    }
    __syncthreads();
    if (j < ROWS && r0 + j < n) {
        float acc = P[OFF_B3];
        for (int i = 0; i < D2; i++) acc = fmaf(h2[j][i], rb(P[OFF_W3 + i], BF16), acc);
        y[r0 + j] = acc;
    }
}

// per-row backward quantities: dz2[r][j], dz1[r][i] (ReLU masks applied), dy[r]
__global__ void __launch_bounds__(64) k_mlp_bwd_rows(const float *y, const float *t, int n, const float *P,
                                                     const float *z1, float *z2dz2, float *z1dz1, float *dy) {
    __shared__ float d2[ROWS][D2 + 1];
    __shared__ float dys[ROWS];
    const int r0 = blockIdx.x * ROWS, j = threadIdx.x;
    if (j < ROWS) {
        float v = 0.f;
        if (r0 + j < n) v = 2.f * (y[r0 + j] - t[r0 + j]) / (float)n;
        dys[j] = v;
        if (r0 + j < n) dy[r0 + j] = v;
    }
    __syncthreads();
    const float w3 = P[OFF_W3 + j];
    for (int r = 0; r < ROWS; r++) {
        float v = 0.f;
        if (r0 + r < n) {
            const float z = z2dz2[(int64_t)(r0 + r) * D2 + j];
            v = z > 0.f ? dys[r] * w3 : 0.f;
        }
        d2[r][j] = v;
    }
    __syncthreads();
    for (int r = 0; r < ROWS; r++) {
        if (r0 + r >= n) break;
        float acc = 0.f;
        for (int k = 0; k < D2; k++) acc = fmaf(d2[r][k], P[OFF_W2 + j * D2 + k], acc);
        const float z = z1[(int64_t)(r0 + r) * D1 + j];
        z1dz1[(int64_t)(r0 + r) * D1 + j] = z > 0.f ? acc : 0.f;
    }
    __syncthreads();
    for (int r = 0; r < ROWS; r++)
        if (r0 + r < n) z2dz2[(int64_t)(r0 + r) * D2 + j] = d2[r][j];
}

// one thread per parameter, summing over all rows in a fixed order (deterministic)
__global__ void k_mlp_grad(const float *X, int n, const float *z1, const float *z2, const float *dz1,
                           const float *dz2, const float *dy, float *g) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= N_PARAMS) return;
    float acc = 0.f;
    if (p < OFF_B1) {
        const int i = p / D1, j = p % D1;
        for (int r = 0; r < n; r++) acc = fmaf(X[(int64_t)r * D0 + i], dz1[(int64_t)r * D1 + j], acc);
    } else if (p < OFF_W2) {
        const int j = p - OFF_B1;
        for (int r = 0; r < n; r++) acc += dz1[(int64_t)r * D1 + j];
    } else if (p < OFF_B2) {
        const int i = (p - OFF_W2) / D2, j = (p - OFF_W2) % D2;
        for (int r = 0; r < n; r++) acc = fmaf(fmaxf(z1[(int64_t)r * D1 + i], 0.f), dz2[(int64_t)r * D2 + j], acc);
    } else if (p < OFF_W3) {
        const int j = p - OFF_B2;
        for (int r = 0; r < n; r++) acc += dz2[(int64_t)r * D2 + j];
    } else if (p < OFF_B3) {
        const int j = p - OFF_W3;
        for (int r = 0; r < n; r++) acc = fmaf(fmaxf(z2[(int64_t)r * D2 + j], 0.f), dy[r], acc);
    } else {
        for (int r = 0; r < n; r++) acc += dy[r];
    }
    g[p] = acc;
}

__global__ void k_adam(float *p, const float *g, float *m, float *v, int n, float lr, float b1, float b2, float eps,
                       float c1, float c2) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    const float mhat = mi / c1, vhat = vi / c2;
    p[i] -= lr * mhat / (sqrtf(vhat) + eps);
}

}  // namespace

size_t mlp_work_floats(int n) { return (size_t)n * (2 * D1 + 2 * D2 + 2) + 64; }

cudaError_t mlp_forward(const float *X, int n, const float *params, float *y, int bf16, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    const unsigned g = (unsigned)((n + ROWS - 1) / ROWS);
    HB_LAUNCHED(1);
    if (bf16) k_mlp_fwd<true><<<g, 64, 0, s>>>(X, n, params, y, nullptr, nullptr);
    else k_mlp_fwd<false><<<g, 64, 0, s>>>(X, n, params, y, nullptr, nullptr);
    return cudaGetLastError();
}

// work: mlp_work_floats(n) floats
cudaError_t mlp_backward(const float *X, const float *t, int n, const float *params, float *grad, float *work,
                         cudaStream_t s) {
    if (n <= 0) return cudaMemsetAsync(grad, 0, sizeof(float) * N_PARAMS, s);
    float *z1 = work;
    float *z2 = z1 + (size_t)n * D1;
    float *dz1 = z2 + (size_t)n * D2;
    float *y = dz1 + (size_t)n * D1;
    float *dy = y + n;
    const unsigned g = (unsigned)((n + ROWS - 1) / ROWS);
    // z2 is kept; its copy in the backward buffer receives dz2
    float *dz2 = dy + n;   // n * D2
    HB_LAUNCHED(1);
    k_mlp_fwd<false><<<g, 64, 0, s>>>(X, n, params, y, z1, z2);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    e = cudaMemcpyAsync(dz2, z2, sizeof(float) * (size_t)n * D2, cudaMemcpyDeviceToDevice, s);
    if (e != cudaSuccess) return e;
    HB_LAUNCHED(1);
    k_mlp_bwd_rows<<<g, 64, 0, s>>>(y, t, n, params, z1, dz2, dz1, dy);
    HB_LAUNCHED(1);
    k_mlp_grad<<<(N_PARAMS + 127) / 128, 128, 0, s>>>(X, n, z1, z2, dz1, dz2, dy, grad);
    return cudaGetLastError();
}

cudaError_t adam_step(float *params, const float *grad, float *m, float *v, int n, int step, float lr, float b1,
                      float b2, float eps, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    const float c1 = 1.f - powf(b1, (float)step), c2 = 1.f - powf(b2, (float)step);
    HB_LAUNCHED(1);
    k_adam<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(params, grad, m, v, n, lr, b1, b2, eps, c1, c2);
    return cudaGetLastError();
}

}  // namespace hb

// ---------------------------------------------------------------------------
// The paper's per-pair cost model N (Section 4.2 "Shallow NNs"; layer sizes
// 8 -> 2 -> 6 -> 1 with ReLU after the first two, Section 6's defaults):
// parameters W1 [8 x 2], b1 [2], W2 [2 x 6], b2 [6], W3 [6], b3, row-major.
// One thread per row; the backward pass sums each row's gradient into the
// block in shared memory and then into grad with one atomic per parameter.
// ---------------------------------------------------------------------------
namespace hb {
namespace {
constexpr int PF = 8, PH1 = 2, PH2 = 6;
constexpr int PO_W1 = 0, PO_B1 = PO_W1 + PF * PH1, PO_W2 = PO_B1 + PH1, PO_B2 = PO_W2 + PH1 * PH2,
              PO_W3 = PO_B2 + PH2, PO_B3 = PO_W3 + PH2, PN = PO_B3 + 1;
static_assert(PN == HB_PAIR_MODEL_PARAMS, "pair model parameter layout");

__device__ __forceinline__ float pn_forward(const float *x, const float *P, float *z1, float *h1, float *z2,
                                            float *h2) {
#pragma unroll
    for (int j = 0; j < PH1; j++) {
        float acc = P[PO_B1 + j];
#pragma unroll
        for (int i = 0; i < PF; i++) acc = fmaf(x[i], P[PO_W1 + i * PH1 + j], acc);
        z1[j] = acc;
        h1[j] = fmaxf(acc, 0.f);
    }
#pragma unroll
    for (int j = 0; j < PH2; j++) {
        float acc = P[PO_B2 + j];
#pragma unroll
        for (int i = 0; i < PH1; i++) acc = fmaf(h1[i], P[PO_W2 + i * PH2 + j], acc);
        z2[j] = acc;
        h2[j] = fmaxf(acc, 0.f);
    }
    float y = P[PO_B3];
#pragma unroll
    for (int i = 0; i < PH2; i++) y = fmaf(h2[i], P[PO_W3 + i], y);
    return y;
}

__global__ void k_pn_fwd(const float *X, int n, const float *P, float *y) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n) return;
    float x[PF], z1[PH1], h1[PH1], z2[PH2], h2[PH2];
#pragma unroll
    for (int i = 0; i < PF; i++) x[i] = X[(size_t)r * PF + i];
    y[r] = pn_forward(x, P, z1, h1, z2, h2);
}

// gradient of mean((y - t)^2); grad must be zero on entry
__global__ void k_pn_bwd(const float *X, const float *t, int n, const float *P, float *grad) {
    __shared__ float g[PN];
    for (int i = threadIdx.x; i < PN; i += blockDim.x) g[i] = 0.f;
    __syncthreads();
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r < n) {
        float x[PF], z1[PH1], h1[PH1], z2[PH2], h2[PH2];
#pragma unroll
        for (int i = 0; i < PF; i++) x[i] = X[(size_t)r * PF + i];
        const float y = pn_forward(x, P, z1, h1, z2, h2);
        const float dy = 2.f * (y - t[r]) / (float)n;
        atomicAdd(&g[PO_B3], dy);
        float dz2[PH2];
#pragma unroll
        for (int i = 0; i < PH2; i++) {
            atomicAdd(&g[PO_W3 + i], dy * h2[i]);
            dz2[i] = z2[i] > 0.f ? dy * P[PO_W3 + i] : 0.f;
            atomicAdd(&g[PO_B2 + i], dz2[i]);
        }
        float dz1[PH1];
#pragma unroll
        for (int i = 0; i < PH1; i++) {
            float dh = 0.f;
#pragma unroll
            for (int j = 0; j < PH2; j++) {
                atomicAdd(&g[PO_W2 + i * PH2 + j], h1[i] * dz2[j]);
                dh = fmaf(dz2[j], P[PO_W2 + i * PH2 + j], dh);
            }
            dz1[i] = z1[i] > 0.f ? dh : 0.f;
            atomicAdd(&g[PO_B1 + i], dz1[i]);
        }
#pragma unroll
        for (int i = 0; i < PF; i++)
#pragma unroll
            for (int j = 0; j < PH1; j++) atomicAdd(&g[PO_W1 + i * PH1 + j], x[i] * dz1[j]);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < PN; i += blockDim.x)
        if (g[i] != 0.f) atomicAdd(&grad[i], g[i]);
}
}  // namespace

cudaError_t pair_model_forward(const float *X, int n, const float *params, float *y, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    HB_LAUNCHED(1);
    k_pn_fwd<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(X, n, params, y);
    return cudaGetLastError();
}

cudaError_t pair_model_backward(const float *X, const float *t, int n, const float *params, float *grad,
                                cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(grad, 0, sizeof(float) * PN, s);
    if (e != cudaSuccess || n <= 0) return e;
    HB_LAUNCHED(1);
    k_pn_bwd<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(X, t, n, params, grad);
    return cudaGetLastError();
}

}  // namespace hb

// ---------------------------------------------------------------------------
// Allocation-free variant of the backward pass (hb_mlp_backward_noalloc).
//
// Some callers cannot allocate device memory at the moment they need a
// gradient: a process whose device memory is fully pre-partitioned by its own
// pool or by another framework, or a latency-critical loop that must not hit
// cudaMalloc / cudaFree (which can synchronize the device).  For them the
// backward pass keeps its per-row work buffers (pre-activations and their
// gradients) in one fixed file-scope device array instead of memory obtained
// per call.  The array is part of the module: every GPU that loads the
// library holds it (NOALLOC_MAX_ROWS * 258 + 64 floats, about 4.2 MB) until
// the process exits.
//
// Host code cannot use the array's name as a device address, so the address
// is looked up once per device with cudaGetSymbolAddress (with that device
// current) the first time the entry point runs on it; make that first call
// before any stream capture.  The address is kept together with the CUDA
// context it was found in and looked up again when the device's current
// context is another one (after cudaDeviceReset the module is loaded anew);
// a reset that hands out a new context at the very same handle cannot be told
// apart, so do not call the entry point across a device reset.  Every call shares the one array: calls that
// overlap on the GPU (different streams, threads or devices' contexts racing
// on the same device) race on it.  Nothing needs clearing between calls:
// each call writes every scratch word it later reads, for its own rows.
// ---------------------------------------------------------------------------
namespace hb {

constexpr int NOALLOC_MAX_ROWS = 4096;
constexpr size_t NOALLOC_SCRATCH_FLOATS = (size_t)NOALLOC_MAX_ROWS * (2 * D1 + 2 * D2 + 2) + 64;
static __device__ __align__(256) float g_backward_scratch[NOALLOC_SCRATCH_FLOATS];

namespace {
constexpr int NOALLOC_MAX_DEVICES = 64;
std::mutex g_noalloc_mu;
float *g_noalloc_ptr[NOALLOC_MAX_DEVICES] = {};
void *g_noalloc_ctx[NOALLOC_MAX_DEVICES] = {};   // the context each address was looked up in

// the calling thread's current CUDA context (driver cuCtxGetCurrent, reached
// through the runtime so that the library needs no link to libcuda); NULL
// when it cannot be read
void *current_context() {
    using get_fn = int (*)(void **);
    static get_fn fn = []() -> get_fn {
        void *f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) != cudaSuccess ||
            q != cudaDriverEntryPointSuccess)
            return nullptr;
        return reinterpret_cast<get_fn>(f);
    }();
    void *ctx = nullptr;
    if (!fn || fn(&ctx) != 0) return nullptr;
    return ctx;
}
}  // namespace

}  // namespace hb

extern "C" hb_status hb_mlp_backward_noalloc(const float *X, const float *t, int32_t n, const float *params,
                                             float *grad, void *stream) {
    using namespace hb;
    if (n < 0 || !params || !grad || (n > 0 && (!X || !t))) return fail(HB_ERR_ARG, "hb_mlp_backward_noalloc: bad arguments");
    if (n > NOALLOC_MAX_ROWS)
        return fail(HB_ERR_ARG, "hb_mlp_backward_noalloc: n = " + std::to_string(n) + " rows exceeds the fixed scratch "
                                "capacity of " + std::to_string(NOALLOC_MAX_ROWS) + " rows; use hb_mlp_backward");
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return fail(HB_ERR_CUDA, std::string("hb_mlp_backward_noalloc: cudaGetDevice: ") + cudaGetErrorString(e));
    if (dev < 0 || dev >= NOALLOC_MAX_DEVICES) return fail(HB_ERR_ARG, "hb_mlp_backward_noalloc: device ordinal too large");
    float *work = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_noalloc_mu);
        void *ctx = current_context();
        if (!g_noalloc_ptr[dev] || ctx != g_noalloc_ctx[dev]) {
            void *p = nullptr;
            e = cudaGetSymbolAddress(&p, g_backward_scratch);
            if (e != cudaSuccess)
                return fail(HB_ERR_CUDA, std::string("hb_mlp_backward_noalloc: cudaGetSymbolAddress: ") + cudaGetErrorString(e));
            g_noalloc_ptr[dev] = static_cast<float *>(p);
            g_noalloc_ctx[dev] = current_context();   // the lookup made the device's context current
        }
        work = g_noalloc_ptr[dev];
    }
    e = mlp_backward(X, t, n, params, grad, work, static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return fail(HB_ERR_CUDA, std::string("hb_mlp_backward_noalloc: ") + cudaGetErrorString(e));
    return HB_OK;
}
