// dfloat.cuh -- double-float arithmetic: a value held as the unevaluated sum
// of two FP32 numbers hi + lo with |lo| <= ulp(hi)/2 (about 48 significant
// bits), built from error-free transformations:
//   TwoSum (Knuth, The Art of Computer Programming vol. 2, 4.2.2): s + e = a + b
//     exactly for any a, b, with s = fl(a + b);
//   FastTwoSum (Dekker, "A floating-point technique for extending the
//     available precision", Numer. Math. 18, 1971): the same when |a| >= |b|;
//   TwoProduct with a fused multiply-add: p + e = a b exactly, p = fl(a b),
//     e = fma(a, b, -p).
// The FP32 form's GMRES keeps its Krylov basis, iterate and work vectors in
// this form: on GB300 an FP64 operation issues at about 1/64 of the FP32
// rate, and these few FP32 operations per FP64-equivalent one keep the
// orthogonalisation's precision close to FP64's (relative rounding 2^-44 to
// 2^-46 per operation instead of 2^-53) at FP32 issue cost. The element is
// 8 bytes, the size of a double, so buffers keep their FP64 sizes.
#pragma once

#include <cuda_runtime.h>

namespace relsim {

struct __align__(8) dfl {
    float hi, lo;
};

__device__ __forceinline__ dfl df_make(float hi, float lo) { return dfl{hi, lo}; }
__device__ __forceinline__ dfl df_from_f(float a) { return dfl{a, 0.0f}; }

// |a| >= |b| (or a == 0)
__device__ __forceinline__ dfl df_fast_two_sum(float a, float b)
{
    const float s = __fadd_rn(a, b);
    const float e = __fsub_rn(b, __fsub_rn(s, a));
    return dfl{s, e};
}

__device__ __forceinline__ dfl df_two_sum(float a, float b)
{
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return dfl{s, e};
}

__device__ __forceinline__ dfl df_two_prod(float a, float b)
{
    const float p = __fmul_rn(a, b);
    const float e = __fmaf_rn(a, b, -p);
    return dfl{p, e};
}

// a + b
__device__ __forceinline__ dfl df_add(dfl a, dfl b)
{
    const dfl s = df_two_sum(a.hi, b.hi);
    const dfl t = df_two_sum(a.lo, b.lo);
    const dfl u = df_fast_two_sum(s.hi, __fadd_rn(s.lo, t.hi));
    return df_fast_two_sum(u.hi, __fadd_rn(u.lo, t.lo));
}

__device__ __forceinline__ dfl df_neg(dfl a) { return dfl{-a.hi, -a.lo}; }
__device__ __forceinline__ dfl df_sub(dfl a, dfl b) { return df_add(a, df_neg(b)); }

// a + b, b an FP32 value
__device__ __forceinline__ dfl df_add_f(dfl a, float b)
{
    const dfl s = df_two_sum(a.hi, b);
    return df_fast_two_sum(s.hi, __fadd_rn(s.lo, a.lo));
}

// a b, b an FP32 value
__device__ __forceinline__ dfl df_mul_f(dfl a, float b)
{
    const dfl p = df_two_prod(a.hi, b);
    return df_fast_two_sum(p.hi, __fmaf_rn(a.lo, b, p.lo));
}

// a b
__device__ __forceinline__ dfl df_mul(dfl a, dfl b)
{
    const dfl p = df_two_prod(a.hi, b.hi);
    const float c = __fmaf_rn(a.hi, b.lo, __fmaf_rn(a.lo, b.hi, p.lo));
    return df_fast_two_sum(p.hi, c);
}

// The conversions touch the FP64 pipe: for scalars and per-block sums only.
__host__ __device__ __forceinline__ dfl df_from_double(double x)
{
    const float hi = (float)x;
    const float lo = (float)(x - (double)hi);
    return dfl{hi, lo};
}
__host__ __device__ __forceinline__ double df_to_double(dfl a) { return (double)a.hi + (double)a.lo; }

// the FP32 value nearest hi + lo
__device__ __forceinline__ float df_to_f(dfl a) { return __fadd_rn(a.hi, a.lo); }

__device__ __forceinline__ dfl df_shfl_xor(dfl a, int o)
{
    return dfl{__shfl_xor_sync(0xffffffffu, a.hi, o), __shfl_xor_sync(0xffffffffu, a.lo, o)};
}

__device__ __forceinline__ dfl df_warp_sum(dfl a)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) a = df_add(a, df_shfl_xor(a, o));
    return a;
}

// a block's double-float sums of N values, converted to FP64 once per block
// (every thread of the block calls it; red holds 32 N pairs)
template <int N>
__device__ __forceinline__ void df_block_sum(dfl (&v)[N], dfl* red, double (&out)[N])
{
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int k = 0; k < N; ++k) v[k] = df_warp_sum(v[k]);
    if (lane == 0)
#pragma unroll
        for (int k = 0; k < N; ++k) red[wid * N + k] = v[k];
    __syncthreads();
    if (wid == 0) {
#pragma unroll
        for (int k = 0; k < N; ++k) {
            dfl t = lane < nw ? red[lane * N + k] : dfl{0.f, 0.f};
            t = df_warp_sum(t);
            out[k] = df_to_double(t);
        }
    }
    __syncthreads();
}

}  // namespace relsim
