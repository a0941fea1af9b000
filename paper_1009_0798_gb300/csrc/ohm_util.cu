// ohm_util.cu -- small device utilities of the host orchestration (not on the stencil path).
#include <cuda_runtime.h>

#include <algorithm>
#include <cstddef>

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

}  // namespace ohm
