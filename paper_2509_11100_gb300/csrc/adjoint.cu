// adjoint.cu -- the data movement around one step's adjoint on the device.
//
// The adjoint of a step takes and returns per-particle gradients indexed by
// the particle's id (the label it carries through every re-sort), so that a
// window of steps can chain them without knowing how each push reordered
// the particles. Around the push and deposit adjoints (particles.cu), which
// work in the particles' current order, these kernels gather a species'
// gradients from id order into the current order and scatter (or add) them
// back; a relabelling kernel replaces each carried id j by ids[j] after a
// range check, and a field kernel adds two gradients of B.
//
// All are HBM-bound streams of FP64 (the id-ordered side is a gather or a
// scatter, local as far as the id order still follows the cell order).
#include "launch.cuh"

namespace relsim {
namespace {

constexpr int kThreads = 256;

unsigned grid_for(int64_t n)
{
    int64_t b = (n + kThreads - 1) / kThreads;
    if (b > 152 * 32) b = 152 * 32;
    return (unsigned)(b > 0 ? b : 1);
}

// lu[i] = gu[id[i]] (3 components), lx[i] = gx[id[i]] (2 components)
__global__ void k_gather_grad(const int32_t* __restrict__ id, const double* __restrict__ gu,
                              const double* __restrict__ gx, double* __restrict__ lu, double* __restrict__ lx,
                              int64_t n)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t j = id[i];
        lu[3 * i] = gu[3 * j];
        lu[3 * i + 1] = gu[3 * j + 1];
        lu[3 * i + 2] = gu[3 * j + 2];
        lx[2 * i] = gx[2 * j];
        lx[2 * i + 1] = gx[2 * j + 1];
    }
}

// gu[id[i]] (+)= lu[i], gx[id[i]] (+)= lx[i]
template <bool ADD>
__global__ void k_scatter_grad(const int32_t* __restrict__ id, const double* __restrict__ lu,
                               const double* __restrict__ lx, double* __restrict__ gu, double* __restrict__ gx,
                               int64_t n)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t j = id[i];
        if (ADD) {
            gu[3 * j] += lu[3 * i];
            gu[3 * j + 1] += lu[3 * i + 1];
            gu[3 * j + 2] += lu[3 * i + 2];
            gx[2 * j] += lx[2 * i];
            gx[2 * j + 1] += lx[2 * i + 1];
        } else {
            gu[3 * j] = lu[3 * i];
            gu[3 * j + 1] = lu[3 * i + 1];
            gu[3 * j + 2] = lu[3 * i + 2];
            gx[2 * j] = lx[2 * i];
            gx[2 * j + 1] = lx[2 * i + 1];
        }
    }
}

// gw[id[i]] += lw[i]
__global__ void k_scatter_add_w(const int32_t* __restrict__ id, const double* __restrict__ lw, double* __restrict__ gw,
                                int64_t n)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        gw[id[i]] += lw[i];
}

// bit 0 of *bad if a carried id or a new label is outside [0, n)
__global__ void k_check_ids(const int32_t* __restrict__ id, const int32_t* __restrict__ ids, int64_t n,
                            int* __restrict__ bad)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        if (id[i] < 0 || id[i] >= n || ids[i] < 0 || ids[i] >= n) atomicOr(bad, 1);
}

__global__ void k_relabel_ids(int32_t* __restrict__ id, const int32_t* __restrict__ ids, int64_t n)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        id[i] = ids[id[i]];
}

__global__ void k_add2(const double* __restrict__ a, const double* __restrict__ b, double* __restrict__ out,
                       int64_t n)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = a[i] + b[i];
}

}  // namespace

cudaError_t gather_grad(const int32_t* id, const double* gu, const double* gx, double* lu, double* lx, int64_t n,
                        cudaStream_t st)
{
    if (n <= 0) return cudaSuccess;
    count_launches(1);
    k_gather_grad<<<grid_for(n), kThreads, 0, st>>>(id, gu, gx, lu, lx, n);
    return cudaGetLastError();
}

cudaError_t scatter_grad(const int32_t* id, const double* lu, const double* lx, double* gu, double* gx, int64_t n,
                         bool add, cudaStream_t st)
{
    if (n <= 0) return cudaSuccess;
    count_launches(1);
    if (add)
        k_scatter_grad<true><<<grid_for(n), kThreads, 0, st>>>(id, lu, lx, gu, gx, n);
    else
        k_scatter_grad<false><<<grid_for(n), kThreads, 0, st>>>(id, lu, lx, gu, gx, n);
    return cudaGetLastError();
}

cudaError_t scatter_add_w(const int32_t* id, const double* lw, double* gw, int64_t n, cudaStream_t st)
{
    if (n <= 0) return cudaSuccess;
    count_launches(1);
    k_scatter_add_w<<<grid_for(n), kThreads, 0, st>>>(id, lw, gw, n);
    return cudaGetLastError();
}

cudaError_t check_ids(const int32_t* id, const int32_t* ids, int64_t n, int* bad, cudaStream_t st)
{
    if (n <= 0) return cudaSuccess;
    count_launches(1);
    k_check_ids<<<grid_for(n), kThreads, 0, st>>>(id, ids, n, bad);
    return cudaGetLastError();
}

cudaError_t relabel_ids(int32_t* id, const int32_t* ids, int64_t n, cudaStream_t st)
{
    if (n <= 0) return cudaSuccess;
    count_launches(1);
    k_relabel_ids<<<grid_for(n), kThreads, 0, st>>>(id, ids, n);
    return cudaGetLastError();
}

cudaError_t add_fields(const double* a, const double* b, double* out, int64_t n, cudaStream_t st)
{
    if (n <= 0) return cudaSuccess;
    count_launches(1);
    k_add2<<<grid_for(n), kThreads, 0, st>>>(a, b, out, n);
    return cudaGetLastError();
}

}  // namespace relsim
