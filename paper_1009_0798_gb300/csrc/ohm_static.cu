// ohm_static.cu -- ohm_residual_static: the residual R = S - L B and its norms on one uniform
// periodic grid, computed without allocating anything.
//
// Why it exists: ohm_create_hierarchy allocates its scratch with cudaMalloc, and some callers
// cannot do that -- hosts that own every device allocation themselves (plugins and embedding
// applications that hand out memory only from their own pool, so a library-side cudaMalloc
// would bypass their accounting or fail under their limits), and real-time loops that must not
// enter the CUDA allocator (its latency is unbounded and it may synchronise the device).  This
// entry point keeps its scratch (block coordinate index, neighbour table, per-block norm
// partials, reduction scratch) in one file-scope device array of fixed size instead.
//
// Scratch rules: the array lives on every device that loads the library until the process
// exits; every call shares it and it keeps the last call's contents (the parts that must
// start at zero are cleared by each call).  Calls whose work overlaps on the GPU (other
// streams, other host threads) race on it.  The first call on a device looks up the array's
// device address and keeps it for the life of the process.  A device reset (cudaDeviceReset)
// invalidates the kept address, so the call must not be used on a device after it has been
// reset.  Every call copies the block list to the
// device, reads the norms back and synchronises its stream before it returns.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <cstring>
#include <mutex>

#include "ohm.h"
#include "ohm_internal.h"

namespace ohm {

constexpr int STATIC_MAX_BLOCKS = 4096;  // 4096 blocks = 2,097,152 cells (e.g. 128^3)

// layout of the scratch array (bytes)
constexpr size_t SO_IJK = 0;                                             // int32 [max][3]
constexpr size_t SO_INDEX = SO_IJK + STATIC_MAX_BLOCKS * 3 * 4;          // int32 [max] coords -> block
constexpr size_t SO_NBR = SO_INDEX + STATIC_MAX_BLOCKS * 4;              // int32 [max][27]
constexpr size_t SO_PART = SO_NBR + (size_t)STATIC_MAX_BLOCKS * 27 * 4;  // double [max][3]
constexpr size_t SO_RED = SO_PART + (size_t)STATIC_MAX_BLOCKS * 3 * 8;   // norm reduction scratch
constexpr size_t SO_NORM = SO_RED + ((NORM_SCRATCH_BYTES + 255) / 256) * 256;  // double [4] + error word
constexpr size_t SO_TOTAL = SO_NORM + 64;

static __device__ __align__(256) unsigned char g_static_scratch[SO_TOTAL];

// coords -> block index; records a duplicate or out-of-range coordinate in the error word
__global__ void k_static_index(const int *__restrict__ ijk, int n, int nbx, int nby, int nbz, int *__restrict__ index,
                               int *__restrict__ err) {
    int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= n) return;
    int i = ijk[3 * b], j = ijk[3 * b + 1], k = ijk[3 * b + 2];
    if (i < 0 || j < 0 || k < 0 || i >= nbx || j >= nby || k >= nbz) {
        atomicOr(err, 1);
        return;
    }
    if (atomicExch(index + (k * nby + j) * nbx + i, b) != -1) atomicOr(err, 2);
}

__global__ void k_static_nbr(const int *__restrict__ ijk, int n, int nbx, int nby, int nbz, const int *__restrict__ index,
                             int *__restrict__ nbr) {
    int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= n * 27) return;
    int b = q / 27, d = q % 27;
    int i = (ijk[3 * b] + d % 3 - 1 + nbx) % nbx;
    int j = (ijk[3 * b + 1] + (d / 3) % 3 - 1 + nby) % nby;
    int k = (ijk[3 * b + 2] + d / 9 - 1 + nbz) % nbz;
    nbr[q] = index[(k * nby + j) * nbx + i];
}

namespace {
constexpr int MAX_DEVICES = 64;
std::mutex g_mu;
unsigned char *g_addr[MAX_DEVICES] = {};

// Device address of the scratch array on the current device (looked up once per device).
cudaError_t scratch_address(unsigned char **out) {
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= MAX_DEVICES) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_addr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_static_scratch);
        if (e != cudaSuccess) return e;
        g_addr[dev] = (unsigned char *)p;
    }
    *out = g_addr[dev];
    return cudaSuccess;
}
}  // namespace

}  // namespace ohm

using namespace ohm;

extern "C" int ohm_residual_static(const int32_t base_cells[3], double dx, double lambda, double dt, int64_t nblocks,
                                   const int32_t *block_ijk, const double *B_dev, const double *S_dev,
                                   const double *eta_dev, double *R_dev, double *norms, void *stream) {
    if (!base_cells || !block_ijk || !B_dev || !S_dev || !eta_dev || !R_dev) return OHM_ERR_INVALID;
    for (int a = 0; a < 3; a++)
        if (base_cells[a] <= 0 || base_cells[a] % BS) return OHM_ERR_INVALID;
    if (!(dx > 0) || !(dt > 0) || !(lambda > 0 && lambda <= 1) || !std::isfinite(dx) || !std::isfinite(dt))
        return OHM_ERR_INVALID;
    const int nbx = base_cells[0] / BS, nby = base_cells[1] / BS, nbz = base_cells[2] / BS;
    const int64_t ncount = (int64_t)nbx * nby * nbz;
    if (nblocks != ncount || ncount > STATIC_MAX_BLOCKS) return OHM_ERR_INVALID;  // whole grid, at most 4096 blocks
    const int n = (int)nblocks;
    // the block list must tile the grid exactly: every coordinate in range, every block once
    // (checked here, on the host, before any work is enqueued)
    {
        uint64_t seen[STATIC_MAX_BLOCKS / 64] = {};
        for (int b = 0; b < n; b++) {
            const int i = block_ijk[3 * b], j = block_ijk[3 * b + 1], k = block_ijk[3 * b + 2];
            if (i < 0 || j < 0 || k < 0 || i >= nbx || j >= nby || k >= nbz) return OHM_ERR_INVALID;
            const int q = (k * nby + j) * nbx + i;
            if (seen[q >> 6] & (1ull << (q & 63))) return OHM_ERR_INVALID;
            seen[q >> 6] |= 1ull << (q & 63);
        }
    }
    cudaStream_t s = (cudaStream_t)stream;
    unsigned char *base = nullptr;
    if (scratch_address(&base) != cudaSuccess) return OHM_ERR_CUDA;
    int *ijk = (int *)(base + SO_IJK), *index = (int *)(base + SO_INDEX), *nbr = (int *)(base + SO_NBR);
    double *part = (double *)(base + SO_PART), *red = (double *)(base + SO_RED), *dnorm = (double *)(base + SO_NORM);
    int *err = (int *)(dnorm + 4);
    // parts that must start cleared: the coordinate index, the reduction ticket, the error word
    if (cudaMemsetAsync(index, 0xff, (size_t)n * 4, s) != cudaSuccess) return OHM_ERR_CUDA;
    if (cudaMemsetAsync(red, 0, NORM_SCRATCH_BYTES, s) != cudaSuccess) return OHM_ERR_CUDA;
    if (cudaMemsetAsync(err, 0, sizeof(int), s) != cudaSuccess) return OHM_ERR_CUDA;
    if (cudaMemcpyAsync(ijk, block_ijk, (size_t)n * 3 * 4, cudaMemcpyHostToDevice, s) != cudaSuccess) return OHM_ERR_CUDA;
    k_static_index<<<(n + 255) / 256, 256, 0, s>>>(ijk, n, nbx, nby, nbz, index, err);
    k_static_nbr<<<(n * 27 + 255) / 256, 256, 0, s>>>(ijk, n, nbx, nby, nbz, index, nbr);
    if (cudaGetLastError() != cudaSuccess) return OHM_ERR_CUDA;
    GridDev g;
    g.nblk = n;
    g.h = dx;
    g.dims[0] = base_cells[0];
    g.dims[1] = base_cells[1];
    g.dims[2] = base_cells[2];
    g.nbr = nbr;
    if (launch_composite<double, double>(g, B_dev, S_dev, eta_dev, nullptr, nullptr, -1.0, -lambda * dt, 1.0, R_dev,
                                         nullptr, nullptr, nullptr, part, dx * dx * dx, s) != cudaSuccess)
        return OHM_ERR_CUDA;
    if (launch_norm_reduce(part, n, red, dnorm, s) != cudaSuccess) return OHM_ERR_CUDA;
    double h[5];
    if (cudaMemcpyAsync(h, dnorm, 5 * sizeof(double), cudaMemcpyDeviceToHost, s) != cudaSuccess) return OHM_ERR_CUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return OHM_ERR_CUDA;
    int e;
    memcpy(&e, &h[4], sizeof(int));
    if (e) return OHM_ERR_INVALID;  // second check of the block list (the host check above passed)
    if (norms) {
        norms[0] = h[1] > 0 ? std::sqrt(h[0] / h[1]) : std::sqrt(h[0]);
        norms[1] = h[2];
        norms[2] = std::sqrt(h[0]);
        norms[3] = std::sqrt(h[1]);
    }
    return OHM_OK;
}
