// native.cu -- the particles of a species in the library's own form.
//
// The library keeps each species sorted by cell, as the cell start table
// start[ncell + 1] and, per particle, the offsets within its cell (fx, fy and
// in 3D fz, each in [0, 1)), the momenta and the weight, one array per
// component in the context's precision. Reading a species out in this form
// and loading it back is a plain copy (no conversion, no sort) and restores
// the state bit for bit; a load in this form checks on the device what the
// kernels rely on: a start table that begins at 0, ends at n and never
// decreases, offsets in [0, 1), finite momenta and weights, and carried ids
// in [0, n).
#include "launch.cuh"

namespace relsim {
namespace {

constexpr int kThreads = 256;

unsigned grid_for(int64_t n)
{
    int64_t b = (n + kThreads - 1) / kThreads;
    if (b > 152 * 16) b = 152 * 16;
    return (unsigned)(b > 0 ? b : 1);
}

template <typename T>
__device__ __forceinline__ bool offset_ok(T f)
{
    return f >= T(0) && f < T(1);   // false for NaN
}

// bit 0: a non-finite momentum or weight; bit 1: an offset outside [0, 1)
// (or not finite); bit 2: a bad start table; bit 3: an id outside [0, n)
template <typename T>
__global__ void k_check_native(const int32_t* __restrict__ start, int ncell, PArrays<T> p,
                               const T* __restrict__ fz, int64_t n, int* __restrict__ bad)
{
    int flags = 0;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        if (!offset_ok(p.fx[i]) || !offset_ok(p.fy[i]) || (fz && !offset_ok(fz[i]))) flags |= 2;
        if (!isfinite(p.ux[i]) || !isfinite(p.uy[i]) || !isfinite(p.uz[i]) || !isfinite(p.w[i])) flags |= 1;
        if (p.id && (p.id[i] < 0 || p.id[i] >= n)) flags |= 8;
    }
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c <= ncell; c += stride) {
        if (c == 0 && start[0] != 0) flags |= 4;
        if (c == ncell && start[ncell] != n) flags |= 4;
        if (c < ncell && start[c] > start[c + 1]) flags |= 4;
    }
    // one atomic per warp that found something
    const int any = __reduce_or_sync(0xffffffffu, flags);
    if (any && (threadIdx.x & 31) == 0) atomicOr(bad, any);
}

__global__ void k_iota(int32_t* __restrict__ id, int64_t n)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        id[i] = (int32_t)i;
}

}  // namespace

template <typename T>
cudaError_t check_native(const int32_t* start, int ncell, PArrays<T> p, const T* fz, int64_t n, int* bad,
                         cudaStream_t st)
{
    count_launches(1);
    k_check_native<T><<<grid_for(n > ncell ? n : (int64_t)ncell + 1), kThreads, 0, st>>>(start, ncell, p, fz, n,
                                                                                         bad);
    return cudaGetLastError();
}

cudaError_t iota_ids(int32_t* id, int64_t n, cudaStream_t st)
{
    if (n <= 0) return cudaSuccess;
    count_launches(1);
    k_iota<<<grid_for(n), kThreads, 0, st>>>(id, n);
    return cudaGetLastError();
}

template cudaError_t check_native<float>(const int32_t*, int, PArrays<float>, const float*, int64_t, int*,
                                         cudaStream_t);
template cudaError_t check_native<double>(const int32_t*, int, PArrays<double>, const double*, int64_t, int*,
                                          cudaStream_t);

}  // namespace relsim
