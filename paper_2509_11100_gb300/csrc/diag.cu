// diag.cu -- field diagnostics: the energy in the Fourier modes (along x) of
// one component of B, the linear-tearing diagnostic of Sec. 3.1 (Fig. 1:
// the B_y energy, its low-pass part and single modes m, whose exponential
// growth gives the tearing rate).
//
// Per cell-centre row j and mode m:  F_{m,j} = sum_i B(i, j) e^{-2 pi i m i / nx}
// and the mode energy is  W_m = (1/2) dV (c_m / nx) sum_j |F_{m,j}|^2  with
// c_m = 1 for m = 0 and m = nx/2, else 2 (a mode and its mirror nx - m), so
// that the W_m over m = 0 .. nx/2 add up to (1/2) sum B^2 dV (Parseval).
//
// Kernels: one warp per row accumulates F_{m,j} in the form's precision from
// a cached twiddle table (exact integer phase (m i) mod nx, one FP64 sincospi
// per entry, rounded to T), writes |F|^2 per (m, j) in FP64, and a second
// kernel adds the rows of each mode in a fixed order: no atomics, so the
// result is reproducible bit for bit.
#include "launch.cuh"

namespace relsim {
namespace {

template <typename T>
__global__ void k_twiddles(T* tw, int nx, int nmodes)
{
    const int64_t total = (int64_t)nmodes * nx;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int m = (int)(t / nx), i = (int)(t % nx);
        const int64_t k = ((int64_t)m * i) % nx;
        double s, c;
        sincospi(2.0 * (double)k / (double)nx, &s, &c);
        tw[2 * t] = (T)c;
        tw[2 * t + 1] = (T)s;
    }
}

template <typename T>
__global__ void k_mode_rows(const T* __restrict__ Bc, const T* __restrict__ tw, int nx, int ny, int nmodes,
                            double* __restrict__ rows)
{
    const int warps = blockDim.x >> 5, lane = threadIdx.x & 31;
    for (int j = blockIdx.x * warps + (threadIdx.x >> 5); j < ny; j += gridDim.x * warps) {
        const T* row = Bc + (int64_t)j * nx;
        for (int m = 0; m < nmodes; ++m) {
            const T* t = tw + 2 * (int64_t)m * nx;
            T re = 0, im = 0;
            for (int i = lane; i < nx; i += 32) {
                const T b = row[i];
                re += b * t[2 * i];
                im -= b * t[2 * i + 1];
            }
            double dr = (double)re, di = (double)im;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                dr += __shfl_xor_sync(0xffffffffu, dr, o);
                di += __shfl_xor_sync(0xffffffffu, di, o);
            }
            if (lane == 0) rows[(int64_t)m * ny + j] = dr * dr + di * di;
        }
    }
}

// the energy of mode m from its ny row values |F_{m,j}|^2 (fixed order)
__global__ void k_mode_sum_one(const double* __restrict__ rows, int nx, int ny, int m, double dV,
                               double* __restrict__ out)
{
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int j = 0; j < ny; ++j) s += rows[j];
        const double cm = (m == 0 || 2 * m == nx) ? 1.0 : 2.0;
        *out = 0.5 * dV * cm * s / (double)nx;
    }
}

__global__ void k_mode_sum(const double* __restrict__ rows, int nx, int ny, int nmodes, double dV,
                           double* __restrict__ out)
{
    for (int m = threadIdx.x; m < nmodes; m += blockDim.x) {
        double s = 0.0;
        for (int j = 0; j < ny; ++j) s += rows[(int64_t)m * ny + j];
        const double cm = (m == 0 || 2 * m == nx) ? 1.0 : 2.0;
        out[m] = 0.5 * dV * cm * s / (double)nx;
    }
}

// The gradient of one mode's energy with respect to the component: warp per
// row j forms F_{m,j} as k_mode_rows does, then writes
//   dW_m/dB(i, j) = dV (c_m / nx) (Re F cos(2 pi m i/nx) - Im F sin(2 pi m i/nx))
// (FP64) and |F|^2 for the energy (summed by k_mode_sum).
template <typename T>
__global__ void k_mode_grad(const T* __restrict__ Bc, const T* __restrict__ tw, int nx, int ny, int m,
                            double dV, double* __restrict__ rows, double* __restrict__ g)
{
    const int warps = blockDim.x >> 5, lane = threadIdx.x & 31;
    const double cm = (m == 0 || 2 * m == nx) ? 1.0 : 2.0;
    const double sc = dV * cm / (double)nx;
    const T* t = tw + 2 * (int64_t)m * nx;
    for (int j = blockIdx.x * warps + (threadIdx.x >> 5); j < ny; j += gridDim.x * warps) {
        const T* row = Bc + (int64_t)j * nx;
        T re = 0, im = 0;
        for (int i = lane; i < nx; i += 32) {
            const T b = row[i];
            re += b * t[2 * i];
            im -= b * t[2 * i + 1];
        }
        double dr = (double)re, di = (double)im;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            dr += __shfl_xor_sync(0xffffffffu, dr, o);
            di += __shfl_xor_sync(0xffffffffu, di, o);
        }
        if (lane == 0) rows[j] = dr * dr + di * di;
        double* gr = g + (int64_t)j * nx;
        for (int i = lane; i < nx; i += 32) gr[i] = sc * (dr * (double)t[2 * i] - di * (double)t[2 * i + 1]);
    }
}

}  // namespace

template <typename T>
cudaError_t mode_gradient(const T* Bc, const T* tw, int nx, int ny, int m, double dV, double* rows,
                          double* energy, double* g, cudaStream_t st)
{
    count_launches(2);
    const int warps = 8;
    const int blocks = (ny + warps - 1) / warps;
    k_mode_grad<T><<<blocks, 32 * warps, 0, st>>>(Bc, tw, nx, ny, m, dV, rows, g);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    // one mode: k_mode_sum over a one-mode row table scaled as mode m
    k_mode_sum_one<<<1, 32, 0, st>>>(rows, nx, ny, m, dV, energy);
    return cudaGetLastError();
}

template <typename T>
cudaError_t mode_twiddles(T* tw, int nx, int nmodes, cudaStream_t st)
{
    const int64_t total = (int64_t)nx * nmodes;
    const int blocks = (int)((total + 255) / 256 < 152 * 4 ? (total + 255) / 256 : 152 * 4);
    count_launches(1);
    k_twiddles<T><<<blocks, 256, 0, st>>>(tw, nx, nmodes);
    return cudaGetLastError();
}

template <typename T>
cudaError_t field_modes(const T* Bc, const T* tw, int nx, int ny, int nmodes, double dV, double* rows,
                        double* out, cudaStream_t st)
{
    count_launches(2);
    const int warps = 8;
    const int blocks = (ny + warps - 1) / warps;
    k_mode_rows<T><<<blocks, 32 * warps, 0, st>>>(Bc, tw, nx, ny, nmodes, rows);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_mode_sum<<<1, 256, 0, st>>>(rows, nx, ny, nmodes, dV, out);
    return cudaGetLastError();
}

template cudaError_t mode_twiddles<float>(float*, int, int, cudaStream_t);
template cudaError_t mode_twiddles<double>(double*, int, int, cudaStream_t);
template cudaError_t mode_gradient<float>(const float*, const float*, int, int, int, double, double*, double*,
                                          double*, cudaStream_t);
template cudaError_t mode_gradient<double>(const double*, const double*, int, int, int, double, double*, double*,
                                           double*, cudaStream_t);
template cudaError_t field_modes<float>(const float*, const float*, int, int, int, double, double*, double*,
                                        cudaStream_t);
template cudaError_t field_modes<double>(const double*, const double*, int, int, int, double, double*,
                                         double*, cudaStream_t);

}  // namespace relsim
