// ohm_util.cu -- small device utilities of the host orchestration (not on the stencil path).
#include <cuda_runtime.h>

#include <algorithm>
#include <cstddef>

#include "ohm.h"
#include "ohm_internal.h"

namespace ohm {

__global__ void __launch_bounds__(256) k_differs(const unsigned long long *__restrict__ a,
                                                  const unsigned long long *__restrict__ b, size_t n, int *flag) {
    bool d = false;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        d |= __ldg(a + i) != __ldg(b + i);
    if (__syncthreads_or(d) && threadIdx.x == 0) *flag = 1;
}

cudaError_t launch_differs(const double *a, const double *b, size_t n, int *flag, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    const unsigned grid = (unsigned)std::min<size_t>((n + 255) / 256, 2048);
    k_differs<<<grid, 256, 0, s>>>(reinterpret_cast<const unsigned long long *>(a),
                                   reinterpret_cast<const unsigned long long *>(b), n, flag);
    return cudaGetLastError();
}

// float64 FMA issue rate: every thread runs 8 independent dependency chains of DFMA (chains
// hide the pipe latency); the result is stored only if it equals a value it never takes, which
// keeps the chains live.
__global__ void __launch_bounds__(256) k_dfma_rate(int iters, double *sink) {
    double a[8];
#pragma unroll
    for (int c = 0; c < 8; c++) a[c] = 1.0 + 1e-3 * (threadIdx.x + c);
    const double m = 0.999999, q = 1e-7;
    for (int i = 0; i < iters; i++) {
#pragma unroll
        for (int c = 0; c < 8; c++) a[c] = fma(a[c], m, q);
    }
    double s = 0.0;
#pragma unroll
    for (int c = 0; c < 8; c++) s += a[c];
    if (s == -1.0 && sink) *sink = s;
}

}  // namespace ohm

using namespace ohm;

extern "C" int ohm_fp64_fma_rate(double *dfma_per_s, void *stream) {
    if (!dfma_per_s) return OHM_ERR_INVALID;
    int dev = 0, nsm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return OHM_ERR_CUDA;
    cudaStream_t s = (cudaStream_t)stream;
    const int blocks = nsm * 8, threads = 256, iters = 4096;
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess) return OHM_ERR_CUDA;
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return OHM_ERR_CUDA;
    }
    float best = 0.f;
    bool ok = true;
    for (int rep = 0; rep < 4 && ok; rep++) {
        ok = cudaEventRecord(e0, s) == cudaSuccess;
        k_dfma_rate<<<blocks, threads, 0, s>>>(iters, nullptr);
        ok = ok && cudaGetLastError() == cudaSuccess && cudaEventRecord(e1, s) == cudaSuccess &&
             cudaEventSynchronize(e1) == cudaSuccess;
        float ms = 0.f;
        ok = ok && cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess;
        if (ok && rep > 0 && (best == 0.f || ms < best)) best = ms;  // the first launch is a warm-up
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (!ok || !(best > 0.f)) return OHM_ERR_CUDA;
    *dfma_per_s = (double)blocks * threads * 8.0 * iters / (best * 1e-3);
    return OHM_OK;
}
