// Throughput probes of the two ALU pipes the quadrature kernels are bound by:
// the SFU (MUFU: ex2, sin, cos) and the FP32 FMA pipe.  Each thread runs
// independent dependency chains of one instruction kind, enough chains and
// warps per SM that the pipe, not the latency, limits the rate; the kernel
// stores the chain ends so nothing is optimised away.  Host code times the
// launch with CUDA events and reports operations per second.
#include <cuda_runtime.h>

#include "../../include/isrs_gn.h"
#include "quad_common.cuh"

namespace isrs {

constexpr int kProbeChains = 8;

// x <- 2^(-x): one MUFU.EX2 per step, the values stay in [1/2, 1].
__global__ void __launch_bounds__(256) k_probe_mufu(float *out, int iters)
{
    float x[kProbeChains];
#pragma unroll
    for (int k = 0; k < kProbeChains; ++k) x[k] = 0.5f + 1e-3f * k + 1e-7f * threadIdx.x;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < kProbeChains; ++k) x[k] = ex2_approx(-x[k]);
    }
    float s = 0.0f;
#pragma unroll
    for (int k = 0; k < kProbeChains; ++k) s += x[k];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// x <- x a + b: one FFMA per step, converging to b / (1 - a) (no denormals).
__global__ void __launch_bounds__(256) k_probe_ffma(float *out, int iters, float a, float b)
{
    float x[2 * kProbeChains];
#pragma unroll
    for (int k = 0; k < 2 * kProbeChains; ++k) x[k] = 1.0f + 1e-3f * k + 1e-7f * threadIdx.x;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < 2 * kProbeChains; ++k) x[k] = fmaf(x[k], a, b);
    }
    float s = 0.0f;
#pragma unroll
    for (int k = 0; k < 2 * kProbeChains; ++k) s += x[k];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace isrs

using namespace isrs;

extern "C" isrs_status isrs_probe_alu_peaks(int device, int which, double *ops_per_s, float *ms)
{
    if (!ops_per_s || (which != 0 && which != 1)) return ISRS_ERR_INVALID_ARG;
    int n_dev = 0;
    if (cudaGetDeviceCount(&n_dev) != cudaSuccess || device < 0 || device >= n_dev) {
        cudaGetLastError();
        return ISRS_ERR_INVALID_ARG;
    }
    if (cudaSetDevice(device) != cudaSuccess) return ISRS_ERR_CUDA;
    int n_sm = 0;
    if (cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) return ISRS_ERR_CUDA;
    const int block = 256, per_sm = 8;                 // 64 warps per SM: every scheduler has 16
    const int grid = n_sm * per_sm;
    const int iters = which == 0 ? 32768 : 131072;   // ~15 ms per launch on a GB300
    float *out = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaStream_t st = nullptr;
    isrs_status rc = ISRS_OK;
    if (cudaMalloc(&out, sizeof(float) * (size_t)grid * block) != cudaSuccess) return ISRS_ERR_ALLOC;
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess || cudaEventCreate(&e0) != cudaSuccess ||
        cudaEventCreate(&e1) != cudaSuccess) {
        rc = ISRS_ERR_CUDA;
    } else {
        float t = 0.0f;
        for (int rep = 0; rep < 2 && rc == ISRS_OK; ++rep) {   // the first launch warms up
            cudaEventRecord(e0, st);
            if (which == 0) k_probe_mufu<<<grid, block, 0, st>>>(out, iters);
            else k_probe_ffma<<<grid, block, 0, st>>>(out, iters, 0.999f, 1e-3f);
            cudaEventRecord(e1, st);
            if (cudaGetLastError() != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
                cudaEventElapsedTime(&t, e0, e1) != cudaSuccess)
                rc = ISRS_ERR_CUDA;
        }
        if (rc == ISRS_OK) {
            const double chains = which == 0 ? kProbeChains : 2 * kProbeChains;
            *ops_per_s = (double)grid * block * (double)iters * chains / (t * 1e-3);
            if (ms) *ms = t;
        }
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (st) cudaStreamDestroy(st);
    cudaFree(out);
    return rc;
}
