// common.cuh -- device-side helpers shared by the RelSIM kernels.
//
// Grid conventions (2D, periodic): node (i,j) at (i dx, j dy), cell (i,j)
// spanning [i dx,(i+1) dx) x [j dy,(j+1) dy) with its centre at
// ((i+1/2) dx, (j+1/2) dy); both have linear index j*nx + i. E, Jhat and the
// mass matrix live on nodes, B on cell centres. Field arrays are
// component-major: F[k*ncell + idx].
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace relsim {

// Number of neighbour offsets kept per node in the half-stored mass matrix:
// o_0 = (0,0), o_1 = (1,0), o_2 = (-1,1), o_3 = (0,1), o_4 = (1,1). The other
// four offsets follow from M_{g+o,g} = M_{g,g+o} (alpha is shared by both
// node orderings of a pair).
constexpr int kHalf = 5;
constexpr int kMBlock = kHalf * 9;   // values per node
constexpr int kNDir = 9;             // cell-to-cell moves of one step
constexpr int kMaxSpecies = 4;
constexpr int kMaxRestart = 100;

// 3D: the half-stored mass matrix keeps 14 of the 27 offsets (0,0,0),
// (1,0,0), (di,1,0) for di = -1..1 and (di,dj,1) for di, dj = -1..1; the
// other 13 follow from M_{g+o,g} = M_{g,g+o}.
constexpr int kHalf3 = 14;
constexpr int kMBlock3 = kHalf3 * 9;

// quadratic (TSC) shapes in 2D: 13 of the 25 offsets stored, (0,0), (1,0),
// (2,0), (di,1) and (di,2) for di = -2..2
constexpr int kHalfQ = 13;
constexpr int kMBlockQ = kHalfQ * 9;

// Constants of the grid and step in one precision, derived on the host
// (grid_derive): formed in every thread they would each cost FP64 work (a
// division, a conversion), and this GPU runs every FP64 operation on a pipe
// about 64 times slower than FP32.
template <typename T>
struct GridC {
    T hdx, hdy;          // 1/(2 dx), 1/(2 dy)
    T qdx, qdy, qdz;     // 1/(4 dx), 1/(4 dy), 1/(4 dz)
    T rdx, rdy, rdz;     // 1/dx, 1/dy, 1/dz
    T dt, theta, td;     // dt, theta, theta dt
    T hdV, thdV, dtdV;   // dV/2, (theta - 1/2) dV, dt dV
};

// ncell counts all cells (nx ny nz in 3D); dV is the cell volume (dx dy in
// 2D). nz = 1, dz = 1 and dim = 2 for the 2D form.
struct GridP {
    int nx, ny, ncell;
    double dx, dy, dt, theta, dV;
    int nz = 1, dim = 2;
    double dz = 1.0;
    int shape = 1;   // 1: linear (CIC); 2: quadratic (TSC, 2D)
    int op_y = 0;    // rows of the 2D operator's tiles (0: the form's default)
    int df = 0;      // 1: the GMRES vectors hold double-float pairs (dfloat.cuh)
                     // in their 8-byte slots (FP32 form, 2D, linear shapes)
    GridC<float> cf{};    // derived constants (grid_derive), FP32
    GridC<double> cd{};   // and FP64
};

// x == 1.0 by its bits (an integer compare instead of an FP64 one)
__device__ __forceinline__ bool is_one(double x) { return __double_as_longlong(x) == 0x3FF0000000000000LL; }

template <typename T>
__host__ __device__ __forceinline__ const GridC<T>& gc(const GridP& g);
template <>
__host__ __device__ __forceinline__ const GridC<float>& gc<float>(const GridP& g) { return g.cf; }
template <>
__host__ __device__ __forceinline__ const GridC<double>& gc<double>(const GridP& g) { return g.cd; }

// fill cf and cd from dx, dy, dz, dt, theta and dV (each value formed in FP64
// and rounded once, as a kernel forming it would)
template <typename T>
inline void grid_derive_one(const GridP& g, GridC<T>& c)
{
    c.hdx = (T)(0.5 / g.dx);
    c.hdy = (T)(0.5 / g.dy);
    c.qdx = (T)(0.25 / g.dx);
    c.qdy = (T)(0.25 / g.dy);
    c.qdz = (T)(0.25 / g.dz);
    c.rdx = (T)(1.0 / g.dx);
    c.rdy = (T)(1.0 / g.dy);
    c.rdz = (T)(1.0 / g.dz);
    c.dt = (T)g.dt;
    c.theta = (T)g.theta;
    c.td = (T)(g.theta * g.dt);
    c.hdV = (T)(0.5 * g.dV);
    c.thdV = (T)((g.theta - 0.5) * g.dV);
    c.dtdV = (T)(g.dt * g.dV);
}
inline void grid_derive(GridP& g)
{
    grid_derive_one(g, g.cf);
    grid_derive_one(g, g.cd);
}

__host__ __device__ __forceinline__ int mblock_of(const GridP& g)
{
    return g.dim == 3 ? kMBlock3 : (g.shape == 2 ? kMBlockQ : kMBlock);
}

__host__ __device__ __forceinline__ int wrap1(int i, int n)
{
    // wrap an index known to lie in [-n, 2n)
    return i < 0 ? i + n : (i >= n ? i - n : i);
}

template <typename T>
__device__ __forceinline__ T ld(const T* p) { return __ldg(p); }

__device__ __forceinline__ double warp_sum(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ float warp_sum(float v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ int warp_sum(int v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Block-wide sum of NS doubles; thread 0 of the block gets the totals in
// out[]. Needs blockDim.x a multiple of 32 and <= 1024. smem: 32*NS doubles.
template <int NS>
__device__ __forceinline__ void block_sum(double (&v)[NS], double* smem, double (&out)[NS])
{
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int nw = (blockDim.x + 31) >> 5;
#pragma unroll
    for (int s = 0; s < NS; ++s) {
        double t = warp_sum(v[s]);
        if (lane == 0) smem[wid * NS + s] = t;
    }
    __syncthreads();
    if (wid == 0) {
#pragma unroll
        for (int s = 0; s < NS; ++s) {
            double t = lane < nw ? smem[lane * NS + s] : 0.0;
            t = warp_sum(t);
            out[s] = t;
        }
    }
    __syncthreads();
}

// round-toward-zero conversion keeps an offset in [0,1) below 1 in FP32
template <typename T> __device__ __forceinline__ T from_double_rz(double v);
template <> __device__ __forceinline__ float from_double_rz<float>(double v) { return __double2float_rz(v); }
template <> __device__ __forceinline__ double from_double_rz<double>(double v) { return v; }

template <typename T> struct Consts;
template <> struct Consts<float> {
    static __device__ __forceinline__ float one_below() { return 0.99999994f; }  // 1 - 2^-24
};
template <> struct Consts<double> {
    static __device__ __forceinline__ double one_below() { return 0.99999999999999989; }  // 1 - 2^-53
};

// ---- TMA bulk copies (cp.async.bulk) completing on an mbarrier ----
// A bulk copy needs 16-byte aligned source and destination addresses and a
// size that is a multiple of 16 bytes.

__device__ __forceinline__ unsigned smem_u32(const void* p)
{
    return (unsigned)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t* mb, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(mb)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx_arrive(uint64_t* mb, unsigned bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(mb)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, unsigned bytes, uint64_t* mb)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(mb))
        : "memory");
}

// an asynchronous 4-byte copy from global into shared memory (completes
// at the issuing thread's cp.async.wait_all / wait_group)
__device__ __forceinline__ void cp_async4(void* dst, const void* src)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}

// one arrival (release semantics at CTA scope: the thread's earlier shared
// memory accesses are ordered before a waiter's later ones)
__device__ __forceinline__ void mbar_arrive(uint64_t* mb)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(mb)) : "memory");
}

// bounded wait on the mbarrier phase with the given parity: at most
// max_polls polls; false if it gave up
__device__ __forceinline__ bool mbar_wait(uint64_t* mb, unsigned parity, long long max_polls)
{
    const unsigned a = smem_u32(mb);
    for (long long it = 0; it < max_polls; ++it) {
        unsigned done;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
            " selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(a), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}

// the same, also giving up (false) once *abort is set by another warp
__device__ __forceinline__ bool mbar_wait_or_abort(uint64_t* mb, unsigned parity, long long max_polls,
                                                   const volatile int* abort)
{
    const unsigned a = smem_u32(mb);
    for (long long it = 0; it < max_polls; ++it) {
        unsigned done;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
            " selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(a), "r"(parity)
            : "memory");
        if (done) return true;
        if ((it & 63) == 63 && *abort) return false;
    }
    return false;
}

}  // namespace relsim
