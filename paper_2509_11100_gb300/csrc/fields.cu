// fields.cu -- grid kernels: right-hand side and matrix-free operator of
// the implicit field equation, the field update with the field terms of the
// energy ledger, the GMRES vector kernels, and format conversions.
//
// GMRES vectors (Krylov basis, iterate, right-hand side, work vectors) have
// 8-byte elements: FP64, or, in the FP32 form of the 2D scheme with linear
// shapes (GridP::df), double-float pairs hi + lo (dfloat.cuh) whose
// arithmetic runs on the FP32 pipe. Kernels take them as double pointers and
// read them through the DF template parameter.
//
// Discrete curls (2D, all three components kept, z ignorable):
//   curl_c (node -> centre (i+1/2, j+1/2)): differences across the cell,
//     averaged over its two edges, e.g. (d_x f) = [(f_{i+1,j} - f_{i,j}) +
//     (f_{i+1,j+1} - f_{i,j+1})]/(2 dx);
//   curl_n (centre -> node (i,j)): the same over the four centres around
//     the node. curl_n is the transpose of curl_c on the periodic grid, which
//     makes the discrete Poynting balance exact.
#include <atomic>

#include "dfloat.cuh"
#include "launch.cuh"

namespace relsim {

namespace {

constexpr int kFieldThreads = 256;
constexpr int kFieldLedger = 6;   // dW_E, dW_B, dissipation, W_E1, W_B1, work_grid

template <typename T>
__global__ void k_from_double(const double* __restrict__ in, T* out, int64_t n, int* bad)
{
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n;
         k += (int64_t)gridDim.x * blockDim.x) {
        double v = in[k];
        if (!isfinite(v)) atomicOr(bad, 1);
        out[k] = (T)v;
    }
}

template <typename T>
__global__ void k_to_double(const T* __restrict__ in, double* out, int64_t n)
{
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n;
         k += (int64_t)gridDim.x * blockDim.x)
        out[k] = (double)in[k];
}

// store v (formed in T) in a GMRES vector slot
template <bool DF, typename T>
__device__ __forceinline__ void vst(double* v, int64_t k, T val)
{
    if constexpr (DF) reinterpret_cast<dfl*>(v)[k] = df_from_f((float)val);
    else v[k] = (double)val;
}

// b = E^n + theta dt curl_n B^n - theta dt Jhat
template <typename T, bool DF>
__global__ void k_rhs(const T* __restrict__ E, const T* __restrict__ B, const T* __restrict__ J,
                      double* __restrict__ b, GridP g)
{
    const int gidx = blockIdx.x * blockDim.x + threadIdx.x;
    if (gidx >= g.ncell) return;
    const int nc = g.ncell, nx = g.nx;
    const int i = gidx % nx, j = gidx / nx;
    const int im = wrap1(i - 1, nx), jm = wrap1(j - 1, g.ny);
    const int c11 = j * nx + i, c01 = j * nx + im, c10 = jm * nx + i, c00 = jm * nx + im;
    const T idx2 = gc<T>(g).hdx, idy2 = gc<T>(g).hdy;
    const T* Bx = B;
    const T* By = B + nc;
    const T* Bz = B + 2 * nc;
    const T dxBy = (By[c11] - By[c01] + By[c10] - By[c00]) * idx2;
    const T dyBx = (Bx[c11] - Bx[c10] + Bx[c01] - Bx[c00]) * idy2;
    const T dxBz = (Bz[c11] - Bz[c01] + Bz[c10] - Bz[c00]) * idx2;
    const T dyBz = (Bz[c11] - Bz[c10] + Bz[c01] - Bz[c00]) * idy2;
    const T td = gc<T>(g).td;
    vst<DF>(b, gidx, E[gidx] + td * dyBz - td * J[gidx]);
    vst<DF>(b, nc + gidx, E[nc + gidx] - td * dxBz - td * J[nc + gidx]);
    vst<DF>(b, 2 * nc + gidx, E[2 * nc + gidx] + td * (dxBy - dyBx) - td * J[2 * nc + gidx]);
}

// a field (T) into a GMRES vector (the initial iterate x = E^n)
template <typename T, bool DF>
__global__ void k_to_vec(const T* __restrict__ in, double* out, int64_t n)
{
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n;
         k += (int64_t)gridDim.x * blockDim.x)
        vst<DF>(out, k, in[k]);
}

// FP64 <-> double-float vectors (the caller-facing operator application)
__global__ void k_df_from_double(const double* __restrict__ in, double* out, int64_t n)
{
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n;
         k += (int64_t)gridDim.x * blockDim.x)
        reinterpret_cast<dfl*>(out)[k] = df_from_double(in[k]);
}
__global__ void k_df_to_double(const double* __restrict__ in, double* out, int64_t n)
{
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n;
         k += (int64_t)gridDim.x * blockDim.x)
        out[k] = df_to_double(reinterpret_cast<const dfl*>(in)[k]);
}

// Node-local loads of a GMRES vector as T
template <typename T, bool DF = false>
__device__ __forceinline__ T vld(const double* v, int64_t k)
{
    if constexpr (DF) {
        const float2 a = __ldg(reinterpret_cast<const float2*>(v) + k);
        return (T)df_to_f(dfl{a.x, a.y});
    } else {
        return (T)__ldg(v + k);
    }
}
__device__ __forceinline__ dfl dld(const double* v, int64_t k)
{
    const float2 a = __ldg(reinterpret_cast<const float2*>(v) + k);
    return dfl{a.x, a.y};
}

// (curl_n curl_c v) and (M v) at a node from its 3x3 stencil of v,
// f[k][a][b] = component k at node (i-1+a, j-1+b), and its mass-matrix
// blocks: Mg = the node's own five blocks M[g][0..4], Mn[o] = the block
// M[g-o][o+1] of the neighbour g - o for the half offsets o = (1,0), (-1,1),
// (0,1), (1,1) (M_{g,g-o} = M_{g-o,g}).
template <typename T, typename P, bool TR>
__device__ __forceinline__ void op_stencil_t(const T (&f)[3][3][3], P Mg, const P (&Mn)[4], T idx2, T idy2,
                                           T cc[3], T mv[3])
{
    // curl_c at the four centres (i-1+ca+1/2, j-1+cb+1/2)
    T C[3][2][2];
#pragma unroll
    for (int ca = 0; ca < 2; ++ca)
#pragma unroll
        for (int cb = 0; cb < 2; ++cb) {
            T dx[3], dy[3];
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                dx[k] = (f[k][ca + 1][cb] - f[k][ca][cb] + f[k][ca + 1][cb + 1] - f[k][ca][cb + 1]) * idx2;
                dy[k] = (f[k][ca][cb + 1] - f[k][ca][cb] + f[k][ca + 1][cb + 1] - f[k][ca + 1][cb]) * idy2;
            }
            C[0][ca][cb] = dy[2];
            C[1][ca][cb] = -dx[2];
            C[2][ca][cb] = dx[1] - dy[0];
        }
    // curl_n at the node from the four centres
    T dx[3], dy[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        dx[k] = (C[k][1][1] - C[k][0][1] + C[k][1][0] - C[k][0][0]) * idx2;
        dy[k] = (C[k][1][1] - C[k][1][0] + C[k][0][1] - C[k][0][0]) * idy2;
    }
    cc[0] = dy[2];
    cc[1] = -dx[2];
    cc[2] = dx[1] - dy[0];
    // M v: own blocks M[g][o] times v(g+o), neighbours' blocks M[g-o][o] times v(g-o);
    // with TR every 3x3 block is applied transposed (M^T v: the stored block
    // of the pair (g, g') serves both orders, M_{g'g} = M_{gg'})
    constexpr int pa[4] = {2, 0, 1, 2}, pb[4] = {1, 2, 2, 2};   // g + o in the stencil
    constexpr int ma[4] = {0, 2, 1, 0}, mb[4] = {1, 0, 0, 0};   // g - o
    T r[3] = {T(0), T(0), T(0)};
#pragma unroll
    for (int rr = 0; rr < 3; ++rr)
#pragma unroll
        for (int s = 0; s < 3; ++s) r[rr] += T(Mg[TR ? s * 3 + rr : rr * 3 + s]) * f[s][1][1];
#pragma unroll
    for (int o = 0; o < 4; ++o) {
        P Mo = Mg + (o + 1) * 9;
#pragma unroll
        for (int rr = 0; rr < 3; ++rr)
#pragma unroll
            for (int s = 0; s < 3; ++s)
                r[rr] += T(Mo[TR ? s * 3 + rr : rr * 3 + s]) * f[s][pa[o]][pb[o]] +
                         T(Mn[o][TR ? s * 3 + rr : rr * 3 + s]) * f[s][ma[o]][mb[o]];
    }
    mv[0] = r[0];
    mv[1] = r[1];
    mv[2] = r[2];
}

template <typename T, typename P>
__device__ __forceinline__ void op_stencil(const T (&f)[3][3][3], P Mg, const P (&Mn)[4], T idx2, T idy2,
                                           T cc[3], T mv[3])
{
    op_stencil_t<T, P, false>(f, Mg, Mn, idx2, idy2, cc, mv);
}

// the same at node (i,j) straight from global memory (v a GMRES vector,
// component-major)
template <typename T, bool DF = false>
__device__ __forceinline__ void op_parts(const T* __restrict__ M, const double* __restrict__ v, int i,
                                         int j, const GridP& g, T cc[3], T mv[3])
{
    const int nx = g.nx, ny = g.ny, nc = g.ncell;
    const int xs[3] = {wrap1(i - 1, nx), i, wrap1(i + 1, nx)};
    const int ys[3] = {wrap1(j - 1, ny) * nx, j * nx, wrap1(j + 1, ny) * nx};
    T f[3][3][3];
#pragma unroll
    for (int k = 0; k < 3; ++k)
#pragma unroll
        for (int a = 0; a < 3; ++a)
#pragma unroll
            for (int b = 0; b < 3; ++b) f[k][a][b] = vld<T, DF>(v, (int64_t)k * nc + ys[b] + xs[a]);
    const T* Mg = M + ((int64_t)ys[1] + xs[1]) * kMBlock;
    const T* Mn[4] = {M + ((int64_t)ys[1] + xs[0]) * kMBlock + 9, M + ((int64_t)ys[0] + xs[2]) * kMBlock + 18,
                      M + ((int64_t)ys[0] + xs[1]) * kMBlock + 27, M + ((int64_t)ys[0] + xs[0]) * kMBlock + 36};
    op_stencil<T, const T*>(f, Mg, Mn, gc<T>(g).hdx, gc<T>(g).hdy, cc, mv);
}

// ---------------------------------------------------------------------------
// The implicit operator A = I + B, B = (theta dt)^2 curl_n curl_c + theta dt M,
// on tiles of X x Y nodes (one thread per node, one warp per tile row). The
// tile's mass-matrix rows j0-1 .. j0+Y-1 (its own blocks and those of the
// row below it that reach into the tile) are staged in shared memory, the
// main columns by TMA bulk copies (one per row) when the rows are 16-byte
// aligned, the two halo columns and the input vector on its 1-node halo by
// plain loads; the input is staged in T, converted once per staged value
// (on GB300 every FP64 operation, conversions included, runs on a pipe about
// 64 times slower than FP32, so the kernels keep their FP64 work to the
// node's own values, the dot products and their reduction). Three modes:
//   kOpA:        out = A in
//   kOpResidual: out = b - A in, per-tile partial of |out|^2
//   kOpArnoldi:  v = s in (written to vj for the tile's nodes when vj is not
//                null), out = B v, per-tile partials of <out, V_q> (q < nv),
//                <out, v> and <out, out> (nv + 2 sums).
// B v is computed in T (the FP32 form's operator precision); the identity,
// the residual and the dot products are formed in FP64.

enum { kOpA = 0, kOpResidual = 1, kOpArnoldi = 2 };
constexpr long long kOpMaxPolls = 1ll << 26;   // bounded mbarrier wait
constexpr int kOpChunk = 8;                    // dot products reduced per shared-memory pass

// The tile height is a compile-time shape with two instances per form (FP32:
// 8 rows, or 4; FP64: 4, or 2); the autotuner picks one per context (YY = 0:
// the default).
template <typename T, int YY = 0>
struct OpTile {
    static constexpr int X = 32;
    static constexpr int Y = YY > 0 ? YY : (sizeof(T) == 4 ? 8 : 4);
    static constexpr int threads = X * Y;
};

template <typename T, int YY = 0>
struct OpShared {
    // rows j0-1 .., columns i0 .. i0+X-1; reused for the dot-product
    // reduction once the operator is applied
    T Mm[OpTile<T, YY>::Y + 1][OpTile<T, YY>::X * kMBlock];
    T Mh[OpTile<T, YY>::Y + 1][2][kMBlock];              // columns i0-1 and i0+tw
    T v[3][OpTile<T, YY>::Y + 2][OpTile<T, YY>::X + 2];  // rows j0-1 .. j0+Y, columns i0-1 .. i0+tw
    uint64_t mbar;
};
template <typename T, int YY>
constexpr bool op_buffer_fits()
{
    return sizeof(T) * (OpTile<T, YY>::Y + 1) * OpTile<T, YY>::X * kMBlock >=
           sizeof(double) * kOpChunk * OpTile<T, YY>::threads;
}
static_assert(op_buffer_fits<float, 0>() && op_buffer_fits<float, 4>() && op_buffer_fits<double, 0>() &&
                  op_buffer_fits<double, 2>(),
              "the reduction buffer fits in the mass-matrix tile");

// Dot2 (Ogita, Rump and Oishi, "Accurate sum and dot product", SIAM J. Sci.
// Comput. 26, 2005) on the FP32 pipe: a running sum s with its error e,
// each term's product split exactly by TwoProduct and added by TwoSum.
struct Dot2 {
    float s = 0.0f, e = 0.0f;
    // += a b, a double-float, b FP32
    __device__ __forceinline__ void add(dfl a, float b)
    {
        const dfl p = df_two_prod(a.hi, b);
        const dfl t = df_two_sum(s, p.hi);
        s = t.hi;
        e = __fadd_rn(e, __fadd_rn(t.lo, __fmaf_rn(a.lo, b, p.lo)));
    }
    // += a b, both double-float
    __device__ __forceinline__ void add(dfl a, dfl b)
    {
        const dfl p = df_two_prod(a.hi, b.hi);
        const float pe = __fmaf_rn(a.hi, b.lo, __fmaf_rn(a.lo, b.hi, p.lo));
        const dfl t = df_two_sum(s, p.hi);
        s = t.hi;
        e = __fadd_rn(e, __fadd_rn(t.lo, pe));
    }
    // -= a b, both double-float
    __device__ __forceinline__ void sub(dfl a, dfl b)
    {
        const dfl p = df_two_prod(a.hi, b.hi);
        const float pe = __fmaf_rn(a.hi, b.lo, __fmaf_rn(a.lo, b.hi, p.lo));
        const dfl t = df_two_sum(s, -p.hi);
        s = t.hi;
        e = __fadd_rn(e, __fsub_rn(t.lo, pe));
    }
    __device__ __forceinline__ dfl value() const { return df_fast_two_sum(s, e); }
};

template <typename T, int MODE, bool TR, int YY = 0, bool DF = false>
__global__ void __launch_bounds__(OpTile<T, YY>::threads, sizeof(T) == 4 ? 3 : 2)
k_op(const T* __restrict__ M, const double* __restrict__ in, double s, const double* __restrict__ b,
     double* __restrict__ out, double* __restrict__ vj, const double* __restrict__ V, int64_t ldv, int nv,
     GridP g, int tma, double* __restrict__ partial, int* __restrict__ err, const GmDyn* __restrict__ dyn)
{
    static_assert(!DF || sizeof(T) == 4, "double-float vectors belong to the FP32 form");
    constexpr int X = OpTile<T, YY>::X, Y = OpTile<T, YY>::Y, NT = OpTile<T, YY>::threads;
    if (MODE == kOpArnoldi && dyn) {
        // arguments of a device-decided Arnoldi iteration
        if (!dyn->live) return;
        in = dyn->in;
        s = dyn->s;
        vj = dyn->vj;
        out = dyn->out;
        nv = dyn->nv;
    }
    extern __shared__ __align__(128) unsigned char op_smem[];
    OpShared<T, YY>& S = *reinterpret_cast<OpShared<T, YY>*>(op_smem);
    const int nx = g.nx, ny = g.ny, nc = g.ncell;
    const int tilesx = (nx + X - 1) / X;
    const int i0 = (blockIdx.x % tilesx) * X, j0 = (blockIdx.x / tilesx) * Y;
    const int tw = min(X, nx - i0), th = min(Y, ny - j0);
    const int tid = threadIdx.x, tx = tid % X, ty = tid / X;
    const bool active = tx < tw && ty < th;
    const int64_t gidx = (int64_t)(j0 + ty) * nx + i0 + tx;

    if (tma) {
        if (tid == 0) {
            mbar_init(&S.mbar, 1);
            asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        }
        __syncthreads();
        if (tid == 0) {
            const unsigned bytes = (unsigned)(tw * kMBlock * sizeof(T));
            mbar_expect_tx_arrive(&S.mbar, bytes * (unsigned)(th + 1));
            for (int r = 0; r <= th; ++r) {
                const int jr = wrap1(j0 - 1 + r, ny);
                bulk_g2s(&S.Mm[r][0], M + ((int64_t)jr * nx + i0) * kMBlock, bytes, &S.mbar);
            }
        }
    } else {
        for (int r = 0; r <= th; ++r) {
            const T* src = M + ((int64_t)wrap1(j0 - 1 + r, ny) * nx + i0) * kMBlock;
            for (int q = tid; q < tw * kMBlock; q += NT) S.Mm[r][q] = ld(src + q);
        }
    }
    // the node's own input value in the vectors' precision (FP64 or
    // double-float; the scale s differs from 1 only for a cycle's first
    // vector)
    double own[3] = {0.0, 0.0, 0.0};
    dfl ownd[3] = {dfl{0.f, 0.f}, dfl{0.f, 0.f}, dfl{0.f, 0.f}};
    if (active)
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            if constexpr (DF) {
                ownd[k] = dld(in, (int64_t)k * nc + gidx);
                if (MODE == kOpArnoldi && !is_one(s)) ownd[k] = df_mul(ownd[k], df_from_double(s));
            } else {
                own[k] = __ldg(in + (int64_t)k * nc + gidx);
                if (MODE == kOpArnoldi && !is_one(s)) own[k] *= s;
            }
        }
    for (int q = tid; q < (th + 1) * 2 * kMBlock; q += NT) {
        const int r = q / (2 * kMBlock), side = (q / kMBlock) % 2, e = q % kMBlock;
        const int ic = side == 0 ? wrap1(i0 - 1, nx) : wrap1(i0 + tw, nx);
        S.Mh[r][side][e] = ld(M + ((int64_t)wrap1(j0 - 1 + r, ny) * nx + ic) * kMBlock + e);
    }
    const int vw = tw + 2, vh = th + 2;
    const T sT = (T)s;
    for (int q = tid; q < 3 * vh * vw; q += NT) {
        const int k = q / (vh * vw), rem = q % (vh * vw), r = rem / vw, cc = rem % vw;
        const int64_t at = (int64_t)k * nc + (int64_t)wrap1(j0 - 1 + r, ny) * nx + wrap1(i0 - 1 + cc, nx);
        T val;
        if constexpr (DF) val = (T)dld(in, at).hi;   // the FP32 operator reads the leading part
        else val = (T)__ldg(in + at);
        if (MODE == kOpArnoldi) val *= sT;
        S.v[k][r][cc] = val;
    }
    bool ok = true;
    if (tma) ok = mbar_wait(&S.mbar, 0, kOpMaxPolls);
    if (__syncthreads_or(!ok)) {   // publishes the plain stores too
        if (tid == 0) {
            atomicOr(err, 2);
            mbar_wait(&S.mbar, 0, kOpMaxPolls);   // let copies in flight land (bounded)
        }
        return;
    }

    double wv[3] = {0.0, 0.0, 0.0};
    dfl wd[3] = {dfl{0.f, 0.f}, dfl{0.f, 0.f}, dfl{0.f, 0.f}};
    float bvf[3] = {0.f, 0.f, 0.f};
    if (active) {
        T f[3][3][3];
#pragma unroll
        for (int k = 0; k < 3; ++k)
#pragma unroll
            for (int a = 0; a < 3; ++a)
#pragma unroll
                for (int bb = 0; bb < 3; ++bb) f[k][a][bb] = S.v[k][ty + bb][tx + a];
        // mass-matrix block row of the node at local column c, local row r
        auto blk = [&](int c, int r) -> const T* {
            return c < 0 ? S.Mh[r + 1][0] : (c >= tw ? S.Mh[r + 1][1] : &S.Mm[r + 1][c * kMBlock]);
        };
        const T* Mn[4] = {blk(tx - 1, ty) + 9, blk(tx + 1, ty - 1) + 18, blk(tx, ty - 1) + 27,
                          blk(tx - 1, ty - 1) + 36};
        T cc[3], mv[3];
        op_stencil_t<T, const T*, TR>(f, blk(tx, ty), Mn, gc<T>(g).hdx, gc<T>(g).hdy, cc, mv);
        const T td = gc<T>(g).td;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const T bvT = td * td * cc[k] + td * mv[k];
            const int64_t at = (int64_t)k * nc + gidx;
            if constexpr (DF) {
                bvf[k] = (float)bvT;
                if (MODE == kOpA) wd[k] = df_add_f(ownd[k], bvf[k]);
                else if (MODE == kOpResidual) wd[k] = df_sub(dld(b, at), df_add_f(ownd[k], bvf[k]));
                else wd[k] = df_from_f(bvf[k]);
                reinterpret_cast<dfl*>(out)[at] = wd[k];
                if (MODE == kOpArnoldi && vj) reinterpret_cast<dfl*>(vj)[at] = ownd[k];
            } else {
                const double bv = (double)bvT;
                if (MODE == kOpA) wv[k] = own[k] + bv;
                else if (MODE == kOpResidual) wv[k] = b[at] - (own[k] + bv);
                else wv[k] = bv;
                out[at] = wv[k];
                if (MODE == kOpArnoldi && vj) vj[at] = own[k];
            }
        }
    }
    if (MODE == kOpA) return;

    // per-tile dot products, kOpChunk at a time: every thread writes its
    // products to shared memory, then each warp sums some of them
    const int nq = MODE == kOpResidual ? 1 : nv + 2;
    const int lane = tid & 31, wid = tid >> 5;
    double* buf = reinterpret_cast<double*>(&S.Mm[0][0]);   // [kOpChunk][NT] (8-byte slots)
    __syncthreads();   // the mass-matrix tile is no longer read
    for (int q0 = 0; q0 < nq; q0 += kOpChunk) {
        const int kc = min(kOpChunk, nq - q0);   // live sums in this pass (warp-uniform)
        if constexpr (DF) {
            dfl* bufd = reinterpret_cast<dfl*>(buf);
            dfl vq[kOpChunk][3];
#pragma unroll
            for (int c = 0; c < kOpChunk; ++c) {
                const int q = q0 + c;
                const bool gl = MODE == kOpArnoldi && active && q < nv;
                const double* Vq = V + (int64_t)(gl ? q : 0) * ldv + gidx;
#pragma unroll
                for (int k = 0; k < 3; ++k) vq[c][k] = gl ? dld(Vq, (int64_t)k * nc) : dfl{0.f, 0.f};
            }
#pragma unroll
            for (int c = 0; c < kOpChunk; ++c) {
                if (c >= kc) break;
                const int q = q0 + c;
                Dot2 d;
                if (active) {
                    if (MODE == kOpResidual) {
#pragma unroll
                        for (int k = 0; k < 3; ++k) d.add(wd[k], wd[k]);
                    } else if (q == nv + 1) {
#pragma unroll
                        for (int k = 0; k < 3; ++k) d.add(df_from_f(bvf[k]), bvf[k]);
                    } else if (q == nv) {
#pragma unroll
                        for (int k = 0; k < 3; ++k) d.add(ownd[k], bvf[k]);
                    } else {
#pragma unroll
                        for (int k = 0; k < 3; ++k) d.add(vq[c][k], bvf[k]);
                    }
                }
                bufd[c * NT + tid] = d.value();
            }
            __syncthreads();
            for (int c = wid; c < kc; c += NT / 32) {
                dfl t = dfl{0.f, 0.f};
#pragma unroll
                for (int m = 0; m < NT / 32; ++m) t = df_add(t, bufd[c * NT + m * 32 + lane]);
                t = df_warp_sum(t);
                if (lane == 0) partial[(int64_t)blockIdx.x * nq + q0 + c] = df_to_double(t);
            }
            __syncthreads();
        } else {
            double vq[kOpChunk][3];
#pragma unroll
            for (int c = 0; c < kOpChunk; ++c) {
                const int q = q0 + c;
                const bool gl = MODE == kOpArnoldi && active && q < nv;
                const double* Vq = V + (int64_t)(gl ? q : 0) * ldv + gidx;
#pragma unroll
                for (int k = 0; k < 3; ++k) vq[c][k] = gl ? __ldg(Vq + (int64_t)k * nc) : 0.0;
            }
            // FP64 work only for the live sums: a branch, not predication (a
            // predicated-off FP64 instruction still takes its slot on the pipe)
#pragma unroll
            for (int c = 0; c < kOpChunk; ++c) {
                if (c >= kc) break;
                const int q = q0 + c;
                double d = 0.0;
                if (active) {
                    if (MODE == kOpResidual || q == nv + 1) d = wv[0] * wv[0] + wv[1] * wv[1] + wv[2] * wv[2];
                    else if (q == nv) d = wv[0] * own[0] + wv[1] * own[1] + wv[2] * own[2];
                    else d = wv[0] * vq[c][0] + wv[1] * vq[c][1] + wv[2] * vq[c][2];
                }
                buf[c * NT + tid] = d;
            }
            __syncthreads();
            for (int c = wid; c < kc; c += NT / 32) {
                double t = 0.0;
#pragma unroll
                for (int m = 0; m < NT / 32; ++m) t += buf[c * NT + m * 32 + lane];
                t = warp_sum(t);
                if (lane == 0) partial[(int64_t)blockIdx.x * nq + q0 + c] = t;
            }
            __syncthreads();
        }
    }
}

// E^{n+theta} from the solve, E^{n+1}, B^{n+1}, and the field ledger terms.
template <typename T, bool DF>
__global__ void __launch_bounds__(kFieldThreads)
k_field_update(const double* __restrict__ x, const T* __restrict__ M, const T* __restrict__ J,
               T* __restrict__ Eth, T* __restrict__ E, const T* __restrict__ B0, T* __restrict__ B1,
               GridP g, double* __restrict__ partial)
{
    __shared__ double red[32 * kFieldLedger];
    const int gidx = blockIdx.x * blockDim.x + threadIdx.x;
    T acc[kFieldLedger] = {T(0), T(0), T(0), T(0), T(0), T(0)};
    if (gidx < g.ncell) {
        const int nc = g.ncell, nx = g.nx, ny = g.ny;
        const int i = gidx % nx, j = gidx / nx;
        const T th = gc<T>(g).theta, hdV = gc<T>(g).hdV;
        T et[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) et[k] = vld<T, DF>(x, (int64_t)k * nc + gidx);
        // E update
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const T e0 = E[(int64_t)k * nc + gidx];
            const T e1 = (et[k] - (T(1) - th) * e0) / th;
            Eth[(int64_t)k * nc + gidx] = et[k];
            E[(int64_t)k * nc + gidx] = e1;
            acc[0] += hdV * (e1 - e0) * (e1 + e0);
            acc[2] += (e1 - e0) * (e1 - e0);
            acc[3] += hdV * e1 * e1;
        }
        // B update of cell (i,j) from E^{n+theta} at its four nodes
        const int i1 = wrap1(i + 1, nx), j1 = wrap1(j + 1, ny);
        const int64_t n00 = (int64_t)j * nx + i, n10 = (int64_t)j * nx + i1;
        const int64_t n01 = (int64_t)j1 * nx + i, n11 = (int64_t)j1 * nx + i1;
        const T idx2 = gc<T>(g).hdx, idy2 = gc<T>(g).hdy;
        T dxE[3], dyE[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const T a = vld<T, DF>(x, k * nc + n00), b = vld<T, DF>(x, k * nc + n10);
            const T c = vld<T, DF>(x, k * nc + n01), d = vld<T, DF>(x, k * nc + n11);
            dxE[k] = (b - a + d - c) * idx2;
            dyE[k] = (c - a + d - b) * idy2;
        }
        const T curl[3] = {dyE[2], -dxE[2], dxE[1] - dyE[0]};
        const T dt = gc<T>(g).dt;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const T b0 = B0[(int64_t)k * nc + gidx];
            const T b1 = b0 - dt * curl[k];
            B1[(int64_t)k * nc + gidx] = b1;
            acc[1] += hdV * (b1 - b0) * (b1 + b0);
            acc[2] += (b1 - b0) * (b1 - b0);
            acc[4] += hdV * b1 * b1;
        }
        acc[2] *= gc<T>(g).thdV;
        // work: dt dV (Jhat + M E^{n+theta}) . E^{n+theta}
        T cc[3], mv[3];
        op_parts<T, DF>(M, x, i, j, g, cc, mv);
        T wk = T(0);
#pragma unroll
        for (int k = 0; k < 3; ++k) wk += (J[(int64_t)k * nc + gidx] + mv[k]) * et[k];
        acc[5] = gc<T>(g).dtdV * wk;
    }
    double out[kFieldLedger];
    if constexpr (sizeof(T) == 4) {
        // the FP32 form: the block's sums as double-float pairs on the FP32
        // pipe (error-free additions), converted to FP64 once per block
        dfl v[kFieldLedger];
#pragma unroll
        for (int s = 0; s < kFieldLedger; ++s) v[s] = dfl{acc[s], 0.f};
        df_block_sum<kFieldLedger>(v, reinterpret_cast<dfl*>(red), out);
    } else {
        double v[kFieldLedger];
#pragma unroll
        for (int s = 0; s < kFieldLedger; ++s) v[s] = (double)acc[s];
        block_sum<kFieldLedger>(v, red, out);
    }
    if (threadIdx.x == 0)
#pragma unroll
        for (int s = 0; s < kFieldLedger; ++s) partial[(int64_t)blockIdx.x * kFieldLedger + s] = out[s];
}

template <typename T>
__global__ void k_field_energy(const T* __restrict__ E, const T* __restrict__ B, GridP g,
                               double* __restrict__ partial)
{
    __shared__ double red[32 * 2];
    T we = T(0), wb = T(0);
    const int64_t n = 3 * (int64_t)g.ncell;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n;
         k += (int64_t)gridDim.x * blockDim.x) {
        we += E[k] * E[k];
        wb += B[k] * B[k];
    }
    double v[2] = {0.5 * g.dV * (double)we, 0.5 * g.dV * (double)wb}, out[2];
    block_sum<2>(v, red, out);
    if (threadIdx.x == 0) {
        partial[blockIdx.x * 2] = out[0];
        partial[blockIdx.x * 2 + 1] = out[1];
    }
}

template <typename T>
__global__ void k_mass_to_double(const T* __restrict__ M, const T* __restrict__ J, double* Md,
                                 double* Jd, GridP g)
{
    const int64_t nm = (int64_t)g.ncell * mblock_of(g), nj = 3 * (int64_t)g.ncell;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < nm;
         k += (int64_t)gridDim.x * blockDim.x) {
        if (Md) Md[k] = (double)M[k];
        if (Jd && k < nj) Jd[k] = (double)J[k];
    }
}

template <typename T>
__global__ void k_mass_from_double(const double* __restrict__ Md, const double* __restrict__ Jd, T* M,
                                   T* J, GridP g, int* bad)
{
    const int64_t nm = (int64_t)g.ncell * mblock_of(g), nj = 3 * (int64_t)g.ncell;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < nm;
         k += (int64_t)gridDim.x * blockDim.x) {
        double a = Md[k];
        if (!isfinite(a)) atomicOr(bad, 1);
        M[k] = (T)a;
        if (k < nj) {
            double b = Jd[k];
            if (!isfinite(b)) atomicOr(bad, 1);
            J[k] = (T)b;
        }
    }
}

// ---------------------------------------------------------------------------
// GMRES vectors: FP64, or double-float (DF) with every sum of products formed
// by Dot2 / Sum2-style compensation on the FP32 pipe

constexpr int kGmThreads = 256;
constexpr int kDotChunk = 8;

template <bool DF>
__global__ void __launch_bounds__(kGmThreads)
k_gm_dots(const double* __restrict__ V, int64_t ldv, int k0, int kc, const double* __restrict__ w,
          int64_t n, double* __restrict__ partial, int stride, bool with_ww)
{
    __shared__ double red[32 * (kDotChunk + 1)];
    double out[kDotChunk + 1];
    if constexpr (DF) {
        Dot2 acc[kDotChunk + 1];
        for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n;
             e += (int64_t)gridDim.x * blockDim.x) {
            const dfl we = dld(w, e);
#pragma unroll
            for (int c = 0; c < kDotChunk; ++c) {
                if (c >= kc) break;
                acc[c].add(dld(V + (int64_t)(k0 + c) * ldv, e), we);
            }
            if (with_ww) acc[kDotChunk].add(we, we);
        }
        dfl v[kDotChunk + 1];
#pragma unroll
        for (int c = 0; c <= kDotChunk; ++c) v[c] = acc[c].value();
        df_block_sum<kDotChunk + 1>(v, reinterpret_cast<dfl*>(red), out);
    } else {
        double acc[kDotChunk + 1];
#pragma unroll
        for (int c = 0; c <= kDotChunk; ++c) acc[c] = 0.0;
        for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n;
             e += (int64_t)gridDim.x * blockDim.x) {
            const double we = w[e];
#pragma unroll
            for (int c = 0; c < kDotChunk; ++c) {
                if (c >= kc) break;   // a branch: no predicated-off FP64 work
                acc[c] += V[(int64_t)(k0 + c) * ldv + e] * we;
            }
            if (with_ww) acc[kDotChunk] += we * we;
        }
        block_sum<kDotChunk + 1>(acc, red, out);
    }
    if (threadIdx.x == 0) {
        for (int c = 0; c < kc; ++c) partial[(int64_t)blockIdx.x * stride + k0 + c] = out[c];
        if (with_ww) partial[(int64_t)blockIdx.x * stride + stride - 1] = out[kDotChunk];
    }
}

constexpr int kGmChunk = 8;   // basis vectors per group of independent loads

// s - sum_c h_c V_c(e) over c < k, double-float (Sum2-style: the running sum
// and its error apart, each product split exactly)
__device__ __forceinline__ dfl df_sub_combination(dfl w, const dfl* hs, const double* __restrict__ V,
                                                  int64_t ldv, int k, int64_t e, float sign)
{
    Dot2 d;
    d.s = w.hi;
    d.e = w.lo;
    for (int c0 = 0; c0 < k; c0 += kGmChunk) {
        const int kc = min(kGmChunk, k - c0);
        dfl vv[kGmChunk];
#pragma unroll
        for (int c = 0; c < kGmChunk; ++c) vv[c] = c < kc ? dld(V + (int64_t)(c0 + c) * ldv, e) : dfl{0.f, 0.f};
#pragma unroll
        for (int c = 0; c < kGmChunk; ++c) {
            if (c >= kc) break;
            const dfl h = hs[c0 + c];
            if (sign < 0.f) d.sub(h, vv[c]);
            else d.add(h, vv[c]);
        }
    }
    return d.value();
}

template <bool DF>
__global__ void __launch_bounds__(kGmThreads)
k_gm_update(double* __restrict__ w, const double* __restrict__ V, int64_t ldv, int k,
            const double* __restrict__ h, int64_t n, double* __restrict__ partial)
{
    __shared__ double hs[kMaxRestart + 1];
    __shared__ double red[32];
    for (int c = threadIdx.x; c < k; c += blockDim.x) {
        if constexpr (DF) reinterpret_cast<dfl*>(hs)[c] = df_from_double(h[c]);
        else hs[c] = h[c];
    }
    __syncthreads();
    double out[1];
    if constexpr (DF) {
        Dot2 acc;
        for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n;
             e += (int64_t)gridDim.x * blockDim.x) {
            const dfl s = df_sub_combination(dld(w, e), reinterpret_cast<const dfl*>(hs), V, ldv, k, e, -1.f);
            reinterpret_cast<dfl*>(w)[e] = s;
            acc.add(s, s);
        }
        dfl v[1] = {acc.value()};
        df_block_sum<1>(v, reinterpret_cast<dfl*>(red), out);
    } else {
        double acc = 0.0;
        for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n;
             e += (int64_t)gridDim.x * blockDim.x) {
            double s = w[e];
            for (int c0 = 0; c0 < k; c0 += kGmChunk) {
                const int kc = min(kGmChunk, k - c0);
                double vv[kGmChunk];
#pragma unroll
                for (int c = 0; c < kGmChunk; ++c) vv[c] = c < kc ? __ldg(V + (int64_t)(c0 + c) * ldv + e) : 0.0;
#pragma unroll
                for (int c = 0; c < kGmChunk; ++c) {
                    if (c >= kc) break;   // a branch: no predicated-off FP64 work
                    s -= hs[c0 + c] * vv[c];
                }
            }
            w[e] = s;
            acc += s * s;
        }
        double v[1] = {acc};
        block_sum<1>(v, red, out);
    }
    if (threadIdx.x == 0) partial[blockIdx.x] = out[0];
}

// Arnoldi update with the normalisation fused: v_{k} = (w - sum_{c<k} h_c V_c)/hn
// with hn^2 = <w,w> - sum h_c^2 (h and <w,w> from the dot-product sums hw =
// [h_0 .. h_{k-1}, <w,w>]; every block forms hn itself).
template <bool DF>
__global__ void __launch_bounds__(kGmThreads)
k_gm_update_scale(const double* __restrict__ w, const double* __restrict__ V, int64_t ldv, int k,
                  const double* __restrict__ hw, double* __restrict__ vout, int64_t n,
                  const GmDyn* __restrict__ dyn)
{
    __shared__ double hs[kMaxRestart + 1];
    __shared__ double inv;
    if (dyn) {
        if (!dyn->live) return;
        w = dyn->out;
        k = dyn->nv + 1;
        hw = dyn->ds;
        vout = const_cast<double*>(V) + (int64_t)k * ldv;
    }
    for (int c = threadIdx.x; c < k; c += blockDim.x) {
        if constexpr (DF) reinterpret_cast<dfl*>(hs)[c] = df_from_double(hw[c]);
        else hs[c] = hw[c];
    }
    if (threadIdx.x == 0) {
        double h2 = hw[k];
        for (int c = 0; c < k; ++c) h2 -= hw[c] * hw[c];
        const double iv = h2 > 0.0 ? 1.0 / sqrt(h2) : 0.0;
        if constexpr (DF) *reinterpret_cast<dfl*>(&inv) = df_from_double(iv);
        else inv = iv;
    }
    __syncthreads();
    if constexpr (DF) {
        const dfl sc = *reinterpret_cast<const dfl*>(&inv);
        for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n;
             e += (int64_t)gridDim.x * blockDim.x) {
            const dfl s = df_sub_combination(dld(w, e), reinterpret_cast<const dfl*>(hs), V, ldv, k, e, -1.f);
            reinterpret_cast<dfl*>(vout)[e] = df_mul(s, sc);
        }
    } else {
        const double sc = inv;
        for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n;
             e += (int64_t)gridDim.x * blockDim.x) {
            double s = w[e];
            for (int c0 = 0; c0 < k; c0 += kGmChunk) {
                const int kc = min(kGmChunk, k - c0);
                double vv[kGmChunk];
#pragma unroll
                for (int c = 0; c < kGmChunk; ++c) vv[c] = c < kc ? __ldg(V + (int64_t)(c0 + c) * ldv + e) : 0.0;
#pragma unroll
                for (int c = 0; c < kGmChunk; ++c) {
                    if (c >= kc) break;   // a branch: no predicated-off FP64 work
                    s -= hs[c0 + c] * vv[c];
                }
            }
            vout[e] = s * sc;
        }
    }
}

template <bool DF>
__global__ void k_gm_scale(double* dst, const double* __restrict__ src, double s, int64_t n)
{
    if constexpr (DF) {
        const dfl sd = df_from_double(s);
        for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n;
             e += (int64_t)gridDim.x * blockDim.x)
            reinterpret_cast<dfl*>(dst)[e] = df_mul(dld(src, e), sd);
    } else {
        for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n;
             e += (int64_t)gridDim.x * blockDim.x)
            dst[e] = src[e] * s;
    }
}

template <bool DF>
__global__ void __launch_bounds__(kGmThreads)
k_gm_sub(double* r, const double* __restrict__ b, const double* __restrict__ Ax, int64_t n,
         double* partial)
{
    __shared__ double red[32];
    double out[1];
    if constexpr (DF) {
        Dot2 acc;
        for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n;
             e += (int64_t)gridDim.x * blockDim.x) {
            const dfl s = df_sub(dld(b, e), dld(Ax, e));
            reinterpret_cast<dfl*>(r)[e] = s;
            acc.add(s, s);
        }
        dfl v[1] = {acc.value()};
        df_block_sum<1>(v, reinterpret_cast<dfl*>(red), out);
    } else {
        double acc = 0.0;
        for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n;
             e += (int64_t)gridDim.x * blockDim.x) {
            double s = b[e] - Ax[e];
            r[e] = s;
            acc += s * s;
        }
        double v[1] = {acc};
        block_sum<1>(v, red, out);
    }
    if (threadIdx.x == 0) partial[blockIdx.x] = out[0];
}

template <bool DF>
__global__ void k_gm_combine(double* x, const double* __restrict__ V, int64_t ldv, int k,
                             const double* __restrict__ y, int64_t n, const int* __restrict__ kdev)
{
    __shared__ double ys[kMaxRestart + 1];
    if (kdev) k = *kdev;   // the dimension decided on the device
    for (int c = threadIdx.x; c < k; c += blockDim.x) {
        if constexpr (DF) reinterpret_cast<dfl*>(ys)[c] = df_from_double(y[c]);
        else ys[c] = y[c];
    }
    __syncthreads();
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n;
         e += (int64_t)gridDim.x * blockDim.x) {
        if constexpr (DF) {
            reinterpret_cast<dfl*>(x)[e] =
                df_sub_combination(dld(x, e), reinterpret_cast<const dfl*>(ys), V, ldv, k, e, 1.f);
        } else {
            double s = x[e];
            for (int c0 = 0; c0 < k; c0 += kGmChunk) {
                const int kc = min(kGmChunk, k - c0);
                double vv[kGmChunk];
#pragma unroll
                for (int c = 0; c < kGmChunk; ++c) vv[c] = c < kc ? __ldg(V + (int64_t)(c0 + c) * ldv + e) : 0.0;
#pragma unroll
                for (int c = 0; c < kGmChunk; ++c) {
                    if (c >= kc) break;   // a branch: no predicated-off FP64 work
                    s += ys[c0 + c] * vv[c];
                }
            }
            x[e] = s;
        }
    }
}

// out[s] = sum_b partial[b*nsums + s], fixed order (deterministic)
__global__ void k_reduce_partials(const double* __restrict__ partial, int nblocks, int nsums,
                                  double* out, const GmDyn* __restrict__ dyn)
{
    __shared__ double red[32];
    const int s = blockIdx.x;
    if (dyn) {
        if (!dyn->live) return;
        nsums = dyn->nv + 2;
        out = dyn->ds;
        if (s >= nsums) return;
    }
    // the loads of a thread's strided partials issued together (U in
    // flight), then added in the order of the plain loop
    constexpr int U = 16;
    const int nt = blockDim.x;
    double acc = 0.0;
    int b = threadIdx.x;
    for (; b + (U - 1) * nt < nblocks; b += U * nt) {
        double t[U];
#pragma unroll
        for (int u = 0; u < U; ++u) t[u] = partial[(int64_t)(b + u * nt) * nsums + s];
#pragma unroll
        for (int u = 0; u < U; ++u) acc += t[u];
    }
    for (; b < nblocks; b += nt) acc += partial[(int64_t)b * nsums + s];
    double v[1] = {acc}, o[1];
    block_sum<1>(v, red, o);
    if (threadIdx.x == 0) out[s] = o[0];
}

int grid_for(int64_t n, int threads, int cap)
{
    int64_t b = (n + threads - 1) / threads;
    if (b < 1) b = 1;
    if (b > cap) b = cap;
    return (int)b;
}

}  // namespace

int field_grid_blocks(GridP g) { return grid_for(g.ncell, kFieldThreads, 1 << 30); }
int op_blocks(GridP g, int precision)
{
    if (g.dim == 3) return op_blocks3(g);
    if (g.shape == 2) return op_blocks_q(g);
    const int X = 32, Y = g.op_y > 0 ? g.op_y : (precision == 32 ? OpTile<float>::Y : OpTile<double>::Y);
    return ((g.nx + X - 1) / X) * ((g.ny + Y - 1) / Y);
}
int gm_blocks(int64_t n) { return grid_for(n, kGmThreads, 152 * 4); }

template <typename T>
cudaError_t fields_from_double(const double* in, T* out, int64_t n, int* bad, cudaStream_t st)
{
    count_launches(1);
    k_from_double<T><<<grid_for(n, 256, 152 * 16), 256, 0, st>>>(in, out, n, bad);
    return cudaGetLastError();
}

template <typename T>
cudaError_t fields_to_double(const T* in, double* out, int64_t n, cudaStream_t st)
{
    count_launches(1);
    k_to_double<T><<<grid_for(n, 256, 152 * 16), 256, 0, st>>>(in, out, n);
    return cudaGetLastError();
}

template <typename T>
cudaError_t rhs(const T* E, const T* B, const T* J, double* b, GridP g, cudaStream_t st)
{
    if (g.dim == 3) return rhs3<T>(E, B, J, b, g, st);
    count_launches(1);
    if constexpr (sizeof(T) == 4) {
        if (g.df) {
            k_rhs<T, true><<<grid_for(g.ncell, 256, 1 << 30), 256, 0, st>>>(E, B, J, b, g);
            return cudaGetLastError();
        }
    }
    k_rhs<T, false><<<grid_for(g.ncell, 256, 1 << 30), 256, 0, st>>>(E, B, J, b, g);
    return cudaGetLastError();
}

template <typename T>
cudaError_t fields_to_vec(const T* in, double* out, int64_t n, int df, cudaStream_t st)
{
    count_launches(1);
    if constexpr (sizeof(T) == 4) {
        if (df) {
            k_to_vec<T, true><<<grid_for(n, 256, 152 * 16), 256, 0, st>>>(in, out, n);
            return cudaGetLastError();
        }
    }
    k_to_vec<T, false><<<grid_for(n, 256, 152 * 16), 256, 0, st>>>(in, out, n);
    return cudaGetLastError();
}

cudaError_t vec_from_double(const double* in, double* out, int64_t n, int df, cudaStream_t st)
{
    if (!df) return in == out ? cudaSuccess : cudaMemcpyAsync(out, in, sizeof(double) * n, cudaMemcpyDeviceToDevice, st);
    count_launches(1);
    k_df_from_double<<<grid_for(n, 256, 152 * 16), 256, 0, st>>>(in, out, n);
    return cudaGetLastError();
}

cudaError_t vec_to_double(const double* in, double* out, int64_t n, int df, cudaStream_t st)
{
    if (!df) return in == out ? cudaSuccess : cudaMemcpyAsync(out, in, sizeof(double) * n, cudaMemcpyDeviceToDevice, st);
    count_launches(1);
    k_df_to_double<<<grid_for(n, 256, 152 * 16), 256, 0, st>>>(in, out, n);
    return cudaGetLastError();
}

template <typename T, int MODE, bool TR, int YY, bool DF>
cudaError_t launch_op_yd(const T* M, const double* in, double sc, const double* b, double* out, double* vj,
                         const double* V, int64_t ldv, int nv, GridP g, double* partial, int* err, cudaStream_t st,
                         const GmDyn* dyn)
{
    // the dynamic shared-memory limit, set once per kernel and device
    static std::atomic<unsigned> attr_set{0};
    const int smem = (int)sizeof(OpShared<T, YY>);
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    const unsigned bit = 1u << (dev & 31);
    if (!(attr_set.load() & bit)) {
        e = cudaFuncSetAttribute(k_op<T, MODE, TR, YY, DF>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e != cudaSuccess) return e;
        attr_set.fetch_or(bit);
    }
    // bulk copies need every staged mass-matrix row to start on 16 bytes
    const int tma = ((int64_t)g.nx * kMBlock * sizeof(T)) % 16 == 0 ? 1 : 0;
    count_launches(1);
    k_op<T, MODE, TR, YY, DF><<<op_blocks(g, sizeof(T) == 4 ? 32 : 64), OpTile<T, YY>::threads, smem, st>>>(
        M, in, sc, b, out, vj, V, ldv, nv, g, tma, partial, err, dyn);
    return cudaGetLastError();
}

template <typename T, int MODE, bool TR, int YY>
cudaError_t launch_op_y(const T* M, const double* in, double sc, const double* b, double* out, double* vj,
                        const double* V, int64_t ldv, int nv, GridP g, double* partial, int* err, cudaStream_t st,
                        const GmDyn* dyn)
{
    if constexpr (sizeof(T) == 4) {
        if (g.df)
            return launch_op_yd<T, MODE, TR, YY, true>(M, in, sc, b, out, vj, V, ldv, nv, g, partial, err, st, dyn);
    }
    return launch_op_yd<T, MODE, TR, YY, false>(M, in, sc, b, out, vj, V, ldv, nv, g, partial, err, st, dyn);
}

template <typename T, int MODE, bool TR = false>
cudaError_t launch_op(const T* M, const double* in, double sc, const double* b, double* out, double* vj,
                      const double* V, int64_t ldv, int nv, GridP g, double* partial, int* err, cudaStream_t st,
                      const GmDyn* dyn = nullptr)
{
    if (g.dim == 3) return launch_op3<T, MODE, TR>(M, in, sc, b, out, vj, V, ldv, nv, g, partial, st, dyn);
    if (g.shape == 2) return launch_op_q<T, MODE, TR>(M, in, sc, b, out, vj, V, ldv, nv, g, partial, st, dyn);
    // the autotuned tile height (g.op_y; 0: the default)
    constexpr int kAlt = sizeof(T) == 4 ? 4 : 2;
    if (g.op_y == kAlt) return launch_op_y<T, MODE, TR, kAlt>(M, in, sc, b, out, vj, V, ldv, nv, g, partial, err, st, dyn);
    return launch_op_y<T, MODE, TR, 0>(M, in, sc, b, out, vj, V, ldv, nv, g, partial, err, st, dyn);
}

template <typename T>
cudaError_t apply_A(const T* M, const double* v, double* out, GridP g, int* err, cudaStream_t st, bool tr)
{
    return tr ? launch_op<T, kOpA, true>(M, v, 1.0, nullptr, out, nullptr, nullptr, 0, 0, g, nullptr, err, st)
              : launch_op<T, kOpA>(M, v, 1.0, nullptr, out, nullptr, nullptr, 0, 0, g, nullptr, err, st);
}

template <typename T>
cudaError_t op_residual(const T* M, const double* x, const double* b, double* r, GridP g, double* partial,
                        int* err, cudaStream_t st, bool tr)
{
    return tr ? launch_op<T, kOpResidual, true>(M, x, 1.0, b, r, nullptr, nullptr, 0, 0, g, partial, err, st)
              : launch_op<T, kOpResidual>(M, x, 1.0, b, r, nullptr, nullptr, 0, 0, g, partial, err, st);
}

template <typename T>
cudaError_t op_arnoldi(const T* M, const double* u, double sc, double* vj, double* w, const double* V,
                       int64_t ldv, int j, GridP g, double* partial, int* err, cudaStream_t st)
{
    return launch_op<T, kOpArnoldi>(M, u, sc, nullptr, w, vj, V, ldv, j, g, partial, err, st);
}

template <typename T>
cudaError_t op_arnoldi_dyn(const T* M, const GmDyn* dyn, const double* V, int64_t ldv, GridP g, double* partial,
                           int* err, cudaStream_t st, bool tr)
{
    return tr ? launch_op<T, kOpArnoldi, true>(M, nullptr, 1.0, nullptr, nullptr, nullptr, V, ldv, 0, g, partial,
                                               err, st, dyn)
              : launch_op<T, kOpArnoldi>(M, nullptr, 1.0, nullptr, nullptr, nullptr, V, ldv, 0, g, partial, err,
                                         st, dyn);
}

template <typename T>
cudaError_t field_update(const double* x, const T* M, const T* J, T* Eth, T* E, const T* B0,
                         T* B1, GridP g, double* partial, int nblocks, cudaStream_t st)
{
    if (g.dim == 3) return field_update3<T>(x, M, J, Eth, E, B0, B1, g, partial, nblocks, st);
    if (g.shape == 2) return field_update_q<T>(x, M, J, Eth, E, B0, B1, g, partial, nblocks, st);
    count_launches(1);
    if constexpr (sizeof(T) == 4) {
        if (g.df) {
            k_field_update<T, true><<<nblocks, kFieldThreads, 0, st>>>(x, M, J, Eth, E, B0, B1, g, partial);
            return cudaGetLastError();
        }
    }
    k_field_update<T, false><<<nblocks, kFieldThreads, 0, st>>>(x, M, J, Eth, E, B0, B1, g, partial);
    return cudaGetLastError();
}

template <typename T>
cudaError_t field_energy(const T* E, const T* B, GridP g, double* partial, int nblocks,
                         cudaStream_t st)
{
    count_launches(1);
    k_field_energy<T><<<nblocks, 256, 0, st>>>(E, B, g, partial);
    return cudaGetLastError();
}

template <typename T>
cudaError_t mass_to_double(const T* M, const T* J, double* Md, double* Jd, GridP g,
                           cudaStream_t st)
{
    count_launches(1);
    k_mass_to_double<T><<<grid_for((int64_t)g.ncell * kMBlock, 256, 152 * 16), 256, 0, st>>>(M, J, Md, Jd, g);
    return cudaGetLastError();
}

template <typename T>
cudaError_t mass_from_double(const double* Md, const double* Jd, T* M, T* J, GridP g, int* bad,
                             cudaStream_t st)
{
    count_launches(1);
    k_mass_from_double<T><<<grid_for((int64_t)g.ncell * kMBlock, 256, 152 * 16), 256, 0, st>>>(Md, Jd, M, J, g, bad);
    return cudaGetLastError();
}

cudaError_t gm_dots(const double* V, int64_t ldv, int k, const double* w, int64_t n,
                    double* partial, int nblocks, cudaStream_t st, int df)
{
    // partial row stride k+1: k dots then w.w
    for (int k0 = 0; k0 < k || k0 == 0; k0 += kDotChunk) {
        int kc = k - k0 < kDotChunk ? k - k0 : kDotChunk;
        if (kc < 0) kc = 0;
        count_launches(1);
        if (df) k_gm_dots<true><<<nblocks, kGmThreads, 0, st>>>(V, ldv, k0, kc, w, n, partial, k + 1, k0 == 0);
        else k_gm_dots<false><<<nblocks, kGmThreads, 0, st>>>(V, ldv, k0, kc, w, n, partial, k + 1, k0 == 0);
        if (k0 + kDotChunk >= k) break;
    }
    return cudaGetLastError();
}

cudaError_t gm_update(double* w, const double* V, int64_t ldv, int k, const double* h, int64_t n,
                      double* partial, int nblocks, cudaStream_t st, int df)
{
    count_launches(1);
    if (df) k_gm_update<true><<<nblocks, kGmThreads, 0, st>>>(w, V, ldv, k, h, n, partial);
    else k_gm_update<false><<<nblocks, kGmThreads, 0, st>>>(w, V, ldv, k, h, n, partial);
    return cudaGetLastError();
}

cudaError_t gm_update_scale(const double* w, const double* V, int64_t ldv, int k, const double* hw,
                            double* vout, int64_t n, cudaStream_t st, int df)
{
    count_launches(1);
    if (df)
        k_gm_update_scale<true><<<grid_for(n, kGmThreads, 152 * 8), kGmThreads, 0, st>>>(w, V, ldv, k, hw, vout, n,
                                                                                        nullptr);
    else
        k_gm_update_scale<false><<<grid_for(n, kGmThreads, 152 * 8), kGmThreads, 0, st>>>(w, V, ldv, k, hw, vout, n,
                                                                                         nullptr);
    return cudaGetLastError();
}

cudaError_t gm_update_scale_dyn(const GmDyn* dyn, const double* V, int64_t ldv, int64_t n, cudaStream_t st, int df)
{
    count_launches(1);
    if (df)
        k_gm_update_scale<true><<<grid_for(n, kGmThreads, 152 * 8), kGmThreads, 0, st>>>(nullptr, V, ldv, 0, nullptr,
                                                                                        nullptr, n, dyn);
    else
        k_gm_update_scale<false><<<grid_for(n, kGmThreads, 152 * 8), kGmThreads, 0, st>>>(nullptr, V, ldv, 0,
                                                                                         nullptr, nullptr, n, dyn);
    return cudaGetLastError();
}

cudaError_t gm_scale(double* dst, const double* src, double s, int64_t n, cudaStream_t st, int df)
{
    count_launches(1);
    if (df) k_gm_scale<true><<<grid_for(n, 256, 152 * 16), 256, 0, st>>>(dst, src, s, n);
    else k_gm_scale<false><<<grid_for(n, 256, 152 * 16), 256, 0, st>>>(dst, src, s, n);
    return cudaGetLastError();
}

cudaError_t gm_sub(double* r, const double* b, const double* Ax, int64_t n, double* partial,
                   int nblocks, cudaStream_t st, int df)
{
    count_launches(1);
    if (df) k_gm_sub<true><<<nblocks, kGmThreads, 0, st>>>(r, b, Ax, n, partial);
    else k_gm_sub<false><<<nblocks, kGmThreads, 0, st>>>(r, b, Ax, n, partial);
    return cudaGetLastError();
}

cudaError_t gm_combine(double* x, const double* V, int64_t ldv, int k, const double* y, int64_t n,
                       cudaStream_t st, int df)
{
    count_launches(1);
    if (df) k_gm_combine<true><<<grid_for(n, 256, 152 * 16), 256, 0, st>>>(x, V, ldv, k, y, n, nullptr);
    else k_gm_combine<false><<<grid_for(n, 256, 152 * 16), 256, 0, st>>>(x, V, ldv, k, y, n, nullptr);
    return cudaGetLastError();
}

cudaError_t gm_combine_dev(double* x, const double* V, int64_t ldv, const int* k, const double* y, int64_t n,
                           cudaStream_t st, int df)
{
    count_launches(1);
    if (df) k_gm_combine<true><<<grid_for(n, 256, 152 * 16), 256, 0, st>>>(x, V, ldv, 0, y, n, k);
    else k_gm_combine<false><<<grid_for(n, 256, 152 * 16), 256, 0, st>>>(x, V, ldv, 0, y, n, k);
    return cudaGetLastError();
}

cudaError_t reduce_partials(const double* partial, int nblocks, int nsums, double* out,
                            cudaStream_t st)
{
    count_launches(1);
    k_reduce_partials<<<nsums, 256, 0, st>>>(partial, nblocks, nsums, out, nullptr);
    return cudaGetLastError();
}

cudaError_t reduce_partials_dyn(const double* partial, int nblocks, const GmDyn* dyn, int maxsums,
                                cudaStream_t st)
{
    count_launches(1);
    k_reduce_partials<<<maxsums, 256, 0, st>>>(partial, nblocks, 0, nullptr, dyn);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Adjoint of the field part of a step (particles held fixed). The forward map
//   b = E0 + theta dt curl_n B0 - theta dt J,   A E_theta = b,
//   E1 = (E_theta - (1 - theta) E0)/theta,     B1 = B0 - dt curl_c E_theta
// is linear in (E0, B0, J); with upstream gradients (gE1, gB1):
//   gE_theta = gE1/theta - dt curl_c^T gB1,    A^T lambda = gE_theta,
//   gE0 = lambda - (1 - theta)/theta gE1,      gB0 = gB1 + theta dt curl_n^T lambda,
//   gJ = -theta dt lambda,  and for the stored block of the node pair (g, g+o)
//   gM = -theta dt (lambda_g E_theta,{g+o}^T + [o != 0] lambda_{g+o} E_theta,g^T).
// On the periodic grid curl_c^T = curl_n exactly, so the transposed curls
// are the curls themselves. FP64 throughout.

// a GMRES vector element in FP64
template <bool DF>
__device__ __forceinline__ double vget(const double* v, int64_t k)
{
    if constexpr (DF) return df_to_double(dld(v, k));
    else return v[k];
}

// curl_c at centre (i, j) = (i+1/2, j+1/2) from the node field v (a GMRES
// vector)
template <bool DF>
__device__ __forceinline__ void curl_c_at(const double* __restrict__ v, int i, int j, const GridP& g, double out[3])
{
    const int nx = g.nx, ny = g.ny, nc = g.ncell;
    const int i1 = wrap1(i + 1, nx), j1 = wrap1(j + 1, ny);
    const int64_t n00 = (int64_t)j * nx + i, n10 = (int64_t)j * nx + i1, n01 = (int64_t)j1 * nx + i,
                  n11 = (int64_t)j1 * nx + i1;
    double dx[3], dy[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const double* f = v + (int64_t)k * nc;
        const double f00 = vget<DF>(f, n00), f10 = vget<DF>(f, n10), f01 = vget<DF>(f, n01), f11 = vget<DF>(f, n11);
        dx[k] = (f10 - f00 + f11 - f01) * g.cd.hdx;
        dy[k] = (f01 - f00 + f11 - f10) * g.cd.hdy;
    }
    out[0] = dy[2];
    out[1] = -dx[2];
    out[2] = dx[1] - dy[0];
}

// curl_n at node (i, j) from the FP64 centre field v (centres i-1, i and j-1, j)
__device__ __forceinline__ void curl_n_at(const double* __restrict__ v, int i, int j, const GridP& g, double out[3])
{
    const int nx = g.nx, ny = g.ny, nc = g.ncell;
    const int im = wrap1(i - 1, nx), jm = wrap1(j - 1, ny);
    const int64_t c11 = (int64_t)j * nx + i, c01 = (int64_t)j * nx + im, c10 = (int64_t)jm * nx + i,
                  c00 = (int64_t)jm * nx + im;
    double dx[3], dy[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const double* f = v + (int64_t)k * nc;
        dx[k] = (f[c11] - f[c01] + f[c10] - f[c00]) * g.cd.hdx;
        dy[k] = (f[c11] - f[c10] + f[c01] - f[c00]) * g.cd.hdy;
    }
    out[0] = dy[2];
    out[1] = -dx[2];
    out[2] = dx[1] - dy[0];
}

template <bool DF>
__global__ void k_adj_pre(const double* __restrict__ gE1, const double* __restrict__ gB1,
                          const double* __restrict__ gEx, double* __restrict__ gEt, GridP g)
{
    for (int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; n < g.ncell; n += (int64_t)gridDim.x * blockDim.x) {
        const int i = (int)(n % g.nx), j = (int)(n / g.nx);
        double cn[3];
        curl_n_at(gB1, i, j, g, cn);
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const double v = gE1[k * g.ncell + n] / g.theta - g.dt * cn[k] + (gEx ? gEx[k * g.ncell + n] : 0.0);
            if constexpr (DF) reinterpret_cast<dfl*>(gEt)[k * g.ncell + n] = df_from_double(v);
            else gEt[k * g.ncell + n] = v;
        }
    }
}

template <bool DF>
__global__ void k_adj_post(const double* __restrict__ gE1, const double* __restrict__ gB1,
                           const double* __restrict__ lam, double* __restrict__ gE0, double* __restrict__ gB0,
                           double* __restrict__ gJ, GridP g)
{
    const double td = g.cd.td, e1 = (1.0 - g.theta) / g.theta;
    for (int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; n < g.ncell; n += (int64_t)gridDim.x * blockDim.x) {
        const int i = (int)(n % g.nx), j = (int)(n / g.nx);
        double cc[3];
        curl_c_at<DF>(lam, i, j, g, cc);
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const int64_t q = k * g.ncell + n;
            const double lq = vget<DF>(lam, q);
            if (gE0) gE0[q] = lq - e1 * gE1[q];
            if (gB0) gB0[q] = gB1[q] + td * cc[k];
            if (gJ) gJ[q] = -td * lq;
        }
    }
}

template <typename T, bool DF>
__global__ void k_adj_mass(const double* __restrict__ lam, const T* __restrict__ Et, double* __restrict__ gM,
                           GridP g)
{
    constexpr int hdi[5] = {0, 1, -1, 0, 1}, hdj[5] = {0, 0, 1, 1, 1};
    const double td = g.cd.td;
    const int nc = g.ncell;
    for (int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; n < nc; n += (int64_t)gridDim.x * blockDim.x) {
        const int i = (int)(n % g.nx), j = (int)(n / g.nx);
        double lg[3], eg[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            lg[k] = vget<DF>(lam, k * nc + n);
            eg[k] = (double)Et[k * nc + n];
        }
#pragma unroll
        for (int o = 0; o < 5; ++o) {
            const int64_t h = (int64_t)wrap1(j + hdj[o], g.ny) * g.nx + wrap1(i + hdi[o], g.nx);
            double lh[3], eh[3];
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                lh[k] = vget<DF>(lam, k * nc + h);
                eh[k] = (double)Et[k * nc + h];
            }
#pragma unroll
            for (int r = 0; r < 3; ++r)
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    double v = lg[r] * eh[c];
                    if (o) v += lh[r] * eg[c];
                    gM[n * kMBlock + o * 9 + r * 3 + c] = -td * v;
                }
        }
    }
}

cudaError_t adjoint_pre(const double* gE1, const double* gB1, const double* gEx, double* gEt, GridP g,
                        cudaStream_t st)
{
    count_launches(1);
    if (g.df) k_adj_pre<true><<<grid_for(g.ncell, 256, 152 * 16), 256, 0, st>>>(gE1, gB1, gEx, gEt, g);
    else k_adj_pre<false><<<grid_for(g.ncell, 256, 152 * 16), 256, 0, st>>>(gE1, gB1, gEx, gEt, g);
    return cudaGetLastError();
}

cudaError_t adjoint_post(const double* gE1, const double* gB1, const double* lam, double* gE0, double* gB0,
                         double* gJ, GridP g, cudaStream_t st)
{
    count_launches(1);
    if (g.df) k_adj_post<true><<<grid_for(g.ncell, 256, 152 * 16), 256, 0, st>>>(gE1, gB1, lam, gE0, gB0, gJ, g);
    else k_adj_post<false><<<grid_for(g.ncell, 256, 152 * 16), 256, 0, st>>>(gE1, gB1, lam, gE0, gB0, gJ, g);
    return cudaGetLastError();
}

template <typename T>
cudaError_t adjoint_mass(const double* lam, const T* Et, double* gM, GridP g, cudaStream_t st)
{
    count_launches(1);
    if (g.df) k_adj_mass<T, true><<<grid_for(g.ncell, 256, 152 * 16), 256, 0, st>>>(lam, Et, gM, g);
    else k_adj_mass<T, false><<<grid_for(g.ncell, 256, 152 * 16), 256, 0, st>>>(lam, Et, gM, g);
    return cudaGetLastError();
}
template cudaError_t adjoint_mass<float>(const double*, const float*, double*, GridP, cudaStream_t);
template cudaError_t adjoint_mass<double>(const double*, const double*, double*, GridP, cudaStream_t);

#define RELSIM_FIELDS_INSTANTIATE(T)                                                               \
    template cudaError_t fields_from_double<T>(const double*, T*, int64_t, int*, cudaStream_t);   \
    template cudaError_t fields_to_double<T>(const T*, double*, int64_t, cudaStream_t);           \
    template cudaError_t fields_to_vec<T>(const T*, double*, int64_t, int, cudaStream_t);          \
    template cudaError_t rhs<T>(const T*, const T*, const T*, double*, GridP, cudaStream_t);      \
    template cudaError_t apply_A<T>(const T*, const double*, double*, GridP, int*, cudaStream_t, bool); \
    template cudaError_t op_residual<T>(const T*, const double*, const double*, double*, GridP,    \
                                        double*, int*, cudaStream_t, bool);                       \
    template cudaError_t op_arnoldi<T>(const T*, const double*, double, double*, double*,         \
                                       const double*, int64_t, int, GridP, double*, int*,          \
                                       cudaStream_t);                                             \
    template cudaError_t op_arnoldi_dyn<T>(const T*, const GmDyn*, const double*, int64_t, GridP, \
                                           double*, int*, cudaStream_t, bool);                    \
    template cudaError_t field_update<T>(const double*, const T*, const T*, T*, T*, const T*, T*, \
                                         GridP, double*, int, cudaStream_t);                      \
    template cudaError_t field_energy<T>(const T*, const T*, GridP, double*, int, cudaStream_t);  \
    template cudaError_t mass_to_double<T>(const T*, const T*, double*, double*, GridP,           \
                                           cudaStream_t);                                         \
    template cudaError_t mass_from_double<T>(const double*, const double*, T*, T*, GridP, int*,   \
                                             cudaStream_t);

RELSIM_FIELDS_INSTANTIATE(float)
RELSIM_FIELDS_INSTANTIATE(double)

}  // namespace relsim
