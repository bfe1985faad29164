// noalloc.cu -- the one entry point of the library that allocates nothing.
//
// relsim_kinetic_energy_noalloc sums w m (gamma - 1) over caller-owned
// device arrays, like the kinetic-energy reduction behind the energy ledger,
// but it keeps its per-block partial sums in a fixed file-scope device array
// instead of memory from cudaMalloc. It exists for callers that cannot
// allocate device memory at the point where they need the number: a
// diagnostics hook inside a time loop whose device memory is all reserved up
// front by its own pool allocator, or code running where a cudaMalloc /
// cudaFree would synchronise the device or is not allowed at all.
#include <mutex>

#include "launch.cuh"
#include "relsim.h"

namespace relsim {

namespace {

constexpr int kNaThreads = 256;
constexpr int kNaItems = 32;                          // particles per thread
constexpr int64_t kNaChunk = (int64_t)kNaThreads * kNaItems;   // per block
constexpr int kNaMaxBlocks = RELSIM_NOALLOC_MAX_PARTICLES / kNaChunk;
static_assert((int64_t)kNaMaxBlocks * kNaChunk == RELSIM_NOALLOC_MAX_PARTICLES,
              "the particle limit must be whole blocks");

// One FP64 partial sum per block. Every GPU that loads the library keeps
// this 32 KB array until the process exits. Host code must not use its name
// as a device address: the address comes from cudaGetSymbolAddress below.
static __device__ __align__(256) double g_noalloc_partial[kNaMaxBlocks];

// block b sums particles [b*kNaChunk, (b+1)*kNaChunk) of u[3n], w[n]
__global__ void __launch_bounds__(kNaThreads)
k_kinetic_aos_partial(const double* __restrict__ u, const double* __restrict__ w, int64_t n,
                      double m, double* __restrict__ partial)
{
    __shared__ double red[32];
    const int64_t base = (int64_t)blockIdx.x * kNaChunk;
    double acc = 0.0;
    for (int r = 0; r < kNaItems; ++r) {
        const int64_t p = base + (int64_t)r * kNaThreads + threadIdx.x;
        if (p < n) {
            const double ux = u[3 * p], uy = u[3 * p + 1], uz = u[3 * p + 2];
            const double u2 = ux * ux + uy * uy + uz * uz;
            // gamma - 1 = |u|^2 / (gamma + 1), free of cancellation
            acc += w[p] * m * (u2 / (sqrt(1.0 + u2) + 1.0));
        }
    }
    double v[1] = {acc}, out[1];
    block_sum<1>(v, red, out);
    if (threadIdx.x == 0) partial[blockIdx.x] = out[0];
}

// one block: the fixed-order sum of the nb partials
__global__ void k_noalloc_total(const double* __restrict__ partial, int nb, double* out)
{
    __shared__ double red[32];
    double acc = 0.0;
    for (int b = threadIdx.x; b < nb; b += blockDim.x) acc += partial[b];
    double v[1] = {acc}, o[1];
    block_sum<1>(v, red, o);
    if (threadIdx.x == 0) *out = o[0];
}

// device address of the scratch array, looked up once per device
constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
double* g_scratch_ptr[kMaxDevices] = {};

cudaError_t scratch_for_current_device(double** ptr)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch_ptr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_partial);
        if (e != cudaSuccess) return e;
        g_scratch_ptr[dev] = (double*)p;
    }
    *ptr = g_scratch_ptr[dev];
    return cudaSuccess;
}

}  // namespace

}  // namespace relsim

extern "C" int relsim_kinetic_energy_noalloc(const double* u, const double* w, int64_t n, double m,
                                             double* out, void* cuda_stream)
{
    using namespace relsim;
    if (n < 0 || !out || (n > 0 && (!u || !w))) return RELSIM_ERR_INVALID_ARG;
    if (n > RELSIM_NOALLOC_MAX_PARTICLES) return RELSIM_ERR_TOO_LARGE;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    double* scratch = nullptr;
    if (scratch_for_current_device(&scratch) != cudaSuccess) {
        cudaGetLastError();
        return RELSIM_ERR_CUDA;
    }
    const int nb = (int)((n + kNaChunk - 1) / kNaChunk);
    if (nb > 0) {
        count_launches(1);
        k_kinetic_aos_partial<<<nb, kNaThreads, 0, st>>>(u, w, n, m, scratch);
    }
    count_launches(1);
    k_noalloc_total<<<1, kNaThreads, 0, st>>>(scratch, nb, out);
    return cudaGetLastError() == cudaSuccess ? RELSIM_OK : RELSIM_ERR_CUDA;
}
