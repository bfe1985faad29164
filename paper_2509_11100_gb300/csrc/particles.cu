// particles.cu -- particle kernels: load conversion, gather/export, the
// mass-matrix and predicted-current deposit, and the explicit push with the
// cell re-sort.
//
// Particles of a species are stored sorted by cell (SoA, offsets fx, fy in
// [0,1) within the cell, momenta u = gamma v, weight w). Cell c owns the
// index range [start[c], start[c+1]).
#include "dfloat.cuh"
#include "launch.cuh"

namespace relsim {

namespace {

// ---------------------------------------------------------------------------
// load: absolute FP64 positions -> (cell key, offsets), FP64 -> T

// true when v (> 0, finite) is a power of two
__device__ __forceinline__ bool is_pow2(double v)
{
    int e;
    return frexp(v, &e) == 0.5;
}

template <typename T>
__global__ void k_load_convert(const double* __restrict__ x, const double* __restrict__ u,
                               const double* __restrict__ w, int64_t n, GridP g, PArrays<T> out,
                               int32_t* key, int32_t* val, int* bad)
{
    int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    // a power-of-two cell size scales exactly by its reciprocal (FP64
    // division is costly on this GPU); any other size divides
    const double rdx = 1.0 / g.dx, rdy = 1.0 / g.dy;
    const bool exact = is_pow2(g.dx) && is_pow2(g.dy);
    for (; p < n; p += stride) {
        double xs = exact ? x[2 * p] * rdx : x[2 * p] / g.dx;
        double ys = exact ? x[2 * p + 1] * rdy : x[2 * p + 1] / g.dy;
        double ux = u[3 * p], uy = u[3 * p + 1], uz = u[3 * p + 2], ww = w[p];
        if (!isfinite(xs) || !isfinite(ys) || !isfinite(ux) || !isfinite(uy) || !isfinite(uz) ||
            !isfinite(ww)) {
            atomicOr(bad, 1);
            xs = ys = 0.0;
        }
        // periodic wrap into [0, n) (only for positions outside the box),
        // then split into cell + offset
        if (xs < 0.0 || xs >= (double)g.nx) xs -= g.nx * floor(xs / g.nx);
        if (ys < 0.0 || ys >= (double)g.ny) ys -= g.ny * floor(ys / g.ny);
        double fi = floor(xs), fj = floor(ys);
        int i = (int)fi, j = (int)fj;
        if (i >= g.nx) i -= g.nx;
        if (j >= g.ny) j -= g.ny;
        if (i < 0) i = 0;
        if (j < 0) j = 0;
        out.fx[p] = from_double_rz<T>(xs - fi);
        out.fy[p] = from_double_rz<T>(ys - fj);
        out.ux[p] = (T)ux;
        out.uy[p] = (T)uy;
        out.uz[p] = (T)uz;
        out.w[p] = (T)ww;
        key[p] = j * g.nx + i;
        val[p] = (int32_t)p;
    }
}

// sets bit 2 of flag if keys[] is not non-decreasing
__global__ void k_keys_unsorted(const int32_t* __restrict__ keys, int64_t n, int* flag)
{
    bool bad = false;
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p + 1 < n; p += (int64_t)gridDim.x * blockDim.x)
        bad = bad || keys[p] > keys[p + 1];
    if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(flag, 2);
}

template <typename T>
__global__ void k_gather(const int32_t* __restrict__ perm, PArrays<T> src, PArrays<T> dst, int64_t n,
                         bool ids_from_perm)
{
    int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (; p < n; p += stride) {
        int32_t s = perm[p];
        dst.fx[p] = src.fx[s];
        dst.fy[p] = src.fy[s];
        dst.ux[p] = src.ux[s];
        dst.uy[p] = src.uy[s];
        dst.uz[p] = src.uz[s];
        dst.w[p] = src.w[s];
        if (dst.id) dst.id[p] = ids_from_perm ? s : src.id[s];
    }
}

// one warp per cell: absolute positions back to FP64
template <typename T>
__global__ void k_export(PArrays<T> pa, const int32_t* __restrict__ start, GridP g, double* x,
                         double* u, double* w, int32_t* id)
{
    const int lane = threadIdx.x & 31;
    int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    int nwarps = (gridDim.x * blockDim.x) >> 5;
    for (int c = warp; c < g.ncell; c += nwarps) {
        int i = c % g.nx, j = c / g.nx;
        int p1 = start[c + 1];
        for (int p = start[c] + lane; p < p1; p += 32) {
            if (x) {
                x[2 * (int64_t)p] = ((double)i + (double)pa.fx[p]) * g.dx;
                x[2 * (int64_t)p + 1] = ((double)j + (double)pa.fy[p]) * g.dy;
            }
            if (u) {
                u[3 * (int64_t)p] = (double)pa.ux[p];
                u[3 * (int64_t)p + 1] = (double)pa.uy[p];
                u[3 * (int64_t)p + 2] = (double)pa.uz[p];
            }
            if (w) w[p] = (double)pa.w[p];
            if (id && pa.id) id[p] = pa.id[p];
        }
    }
}

// ---------------------------------------------------------------------------
// shared per-particle arithmetic

// Work units of both particle passes: row segments of up to kUnitW
// consecutive cells (same row j, columns i0 .. i0+cn-1), so a unit's
// particles are one contiguous range of the sorted arrays and its fields fit
// a small shared-memory tile.
constexpr int kUnitW = 32;
constexpr int kTB = kUnitW + 2;   // centre columns i0-1 .. i0+cn
constexpr int kTE = kUnitW + 1;   // node columns i0 .. i0+cn
constexpr int kTBD = 43;          // the deposit's padded row strides (tile_B / tile_E)
constexpr int kTED = 43;

struct Unit {
    int j, i0, cn, c0;
};

__device__ __forceinline__ Unit unit_of(int u, int nx)
{
    const int nseg = (nx + kUnitW - 1) / kUnitW;
    Unit r;
    r.j = u / nseg;
    r.i0 = (u - r.j * nseg) * kUnitW;
    r.cn = min(kUnitW, nx - r.i0);
    r.c0 = r.j * nx + r.i0;
    return r;
}

__host__ __device__ __forceinline__ int units_of(int nx, int ny) { return ny * ((nx + kUnitW - 1) / kUnitW); }

// B^n on the centres around a unit: [comp][row j-1, j, j+1][col i0-1 .. i0+cn].
// NTHR threads (tid < NTHR) share the loads; for a warp the loop unrolls so
// its loads issue together.
template <typename T, int NTHR, int RB = kTB>
__device__ __forceinline__ void load_tile_B(T (*sB)[3][RB], const T* __restrict__ B, const Unit& un, int nx,
                                            int ny, int nc, int tid)
{
#pragma unroll(NTHR < 128 ? 16 : 1)
    for (int idx0 = 0; idx0 < 9 * kTB; idx0 += NTHR) {
        const int idx = idx0 + tid;
        const int comp = idx / (3 * kTB), r = (idx / kTB) % 3, col = idx % kTB;
        if (idx < 9 * kTB && col <= un.cn + 1) {
            const int gi = wrap1(un.i0 - 1 + col, nx), gj = wrap1(un.j - 1 + r, ny);
            sB[comp][r][col] = ld(B + comp * nc + gj * nx + gi);
        }
    }
}

// E^{n+theta} on the nodes of a unit: [comp][row j, j+1][col i0 .. i0+cn]
template <typename T, int NTHR, int RE = kTE>
__device__ __forceinline__ void load_tile_E(T (*sE)[2][RE], const T* __restrict__ E, const Unit& un, int nx,
                                            int ny, int nc, int tid)
{
#pragma unroll(NTHR < 128 ? 16 : 1)
    for (int idx0 = 0; idx0 < 6 * kTE; idx0 += NTHR) {
        const int idx = idx0 + tid;
        const int comp = idx / (2 * kTE), r = (idx / kTE) % 2, col = idx % kTE;
        if (idx < 6 * kTE && col <= un.cn) {
            const int gi = wrap1(un.i0 + col, nx), gj = wrap1(un.j + r, ny);
            sE[comp][r][col] = ld(E + comp * nc + gj * nx + gi);
        }
    }
}

// B at a particle of local cell l: the centre lattice coordinate is
// i + fx - 1/2, so the two centres are (i-1, i) when fx < 1/2, else (i, i+1)
template <typename T, int RB = kTB>
__device__ __forceinline__ void tile_B(const T (*sB)[3][RB], int l, T fx, T fy, T& Bx, T& By, T& Bz)
{
    const bool lx = fx < T(0.5), ly = fy < T(0.5);
    const T tx = lx ? fx + T(0.5) : fx - T(0.5);
    const T ty = ly ? fy + T(0.5) : fy - T(0.5);
    const int c0 = lx ? l : l + 1;
    const int r0 = ly ? 0 : 1;
    const T w00 = (T(1) - tx) * (T(1) - ty), w10 = tx * (T(1) - ty);
    const T w01 = (T(1) - tx) * ty, w11 = tx * ty;
    Bx = w00 * sB[0][r0][c0] + w10 * sB[0][r0][c0 + 1] + w01 * sB[0][r0 + 1][c0] + w11 * sB[0][r0 + 1][c0 + 1];
    By = w00 * sB[1][r0][c0] + w10 * sB[1][r0][c0 + 1] + w01 * sB[1][r0 + 1][c0] + w11 * sB[1][r0 + 1][c0 + 1];
    Bz = w00 * sB[2][r0][c0] + w10 * sB[2][r0][c0 + 1] + w01 * sB[2][r0 + 1][c0] + w11 * sB[2][r0 + 1][c0 + 1];
}

// E at a particle of local cell l from the four nodes of the cell
template <typename T>
__device__ __forceinline__ void tile_E(const T (*sE)[2][kTE], int l, T W0, T W1, T W2, T W3, T& Ex, T& Ey,
                                       T& Ez)
{
    Ex = W0 * sE[0][0][l] + W1 * sE[0][0][l + 1] + W2 * sE[0][1][l] + W3 * sE[0][1][l + 1];
    Ey = W0 * sE[1][0][l] + W1 * sE[1][0][l + 1] + W2 * sE[1][1][l] + W3 * sE[1][1][l + 1];
    Ez = W0 * sE[2][0][l] + W1 * sE[2][0][l + 1] + W2 * sE[2][1][l] + W3 * sE[2][1][l + 1];
}

// E^n on a unit's nodes, held only by the predicted-gamma variant (gbar =
// gamma(u^n + beta E^n(x))); empty otherwise
template <typename T, bool PRED, int RE = kTE>
struct PredTile {
    __device__ const T (*en() const)[2][RE] { return nullptr; }
};
template <typename T, int RE>
struct PredTile<T, true, RE> {
    T En[3][2][RE];
    __device__ const T (*en() const)[2][RE] { return En; }
};

// |u|^2 of the momentum whose Lorentz factor enters alpha: u^n, or with
// PRED the predicted u^n + beta E^n(x) (node weights W0..W3 of cell l)
template <typename T, bool PRED, int RE = kTE>
__device__ __forceinline__ T gbar_u2(T ux, T uy, T uz, T beta, const T (*sEn)[2][RE], int l, T W0, T W1, T W2,
                                     T W3, T& sx, T& sy, T& sz)
{
    if (!PRED) {
        sx = ux;
        sy = uy;
        sz = uz;
        return ux * ux + uy * uy + uz * uz;
    }
    // one component at a time (compiler barriers between them): the twelve
    // tile loads in flight together would push the deposit past its 128
    // registers
    sx = ux + beta * (W0 * sEn[0][0][l] + W1 * sEn[0][0][l + 1] + W2 * sEn[0][1][l] + W3 * sEn[0][1][l + 1]);
    asm volatile("" ::: "memory");
    sy = uy + beta * (W0 * sEn[1][0][l] + W1 * sEn[1][0][l + 1] + W2 * sEn[1][1][l] + W3 * sEn[1][1][l + 1]);
    asm volatile("" ::: "memory");
    sz = uz + beta * (W0 * sEn[2][0][l] + W1 * sEn[2][0][l + 1] + W2 * sEn[2][1][l] + W3 * sEn[2][1][l + 1]);
    asm volatile("" ::: "memory");
    return sx * sx + sy * sy + sz * sz;
}

// reciprocal square root and reciprocal: the hardware approximations in the
// FP32 form (a few ulp), exact operations in the FP64 form
__device__ __forceinline__ float rsqrt_t(float x) { return rsqrtf(x); }
__device__ __forceinline__ double rsqrt_t(double x) { return 1.0 / sqrt(x); }
__device__ __forceinline__ float rcp_t(float x) { return __fdividef(1.0f, x); }
__device__ __forceinline__ double rcp_t(double x) { return 1.0 / x; }

// The rotation of one particle, shared by the deposit and the push so both
// see the same alpha: 1/gbar, a = beta B/gbar and 1/(1 + |a|^2).
template <typename T>
struct Rot {
    T ig, ax, ay, az, sa;
};

template <typename T>
__device__ __forceinline__ Rot<T> rotation(T u2, T Bx, T By, T Bz, T beta)
{
    Rot<T> r;
    r.ig = rsqrt_t(T(1) + u2);
    const T bg = beta * r.ig;
    r.ax = bg * Bx;
    r.ay = bg * By;
    r.az = bg * Bz;
    r.sa = rcp_t(T(1) + r.ax * r.ax + r.ay * r.ay + r.az * r.az);
    return r;
}

// ---------------------------------------------------------------------------
// deposit: G lanes per cell accumulate 81 mass-matrix moments and 12 current
// values in registers, reduce across the group, then flush with atomics.
//
// Moments: S[k][e] = sum_p c_p XX_xx YY_yy alpha'_e with k = xx*3 + yy,
// XX = ((1-fx)^2, (1-fx) fx, fx^2), YY likewise in y, alpha' = alpha (1+|a|^2)
// and c_p = w q beta /(gbar dV (1+|a|^2)). The ten node pairs of a cell take
// nine distinct weight products; (n00,n11) and (n10,n01) share k = 4.
//
// A CTA handles units (row segments of up to 32 cells, one contiguous
// particle range per species). Each (unit, species) stage is copied into
// shared memory by TMA bulk copies (cp.async.bulk, completion on an
// mbarrier), two stages in flight, so two CTAs fit on an SM; the groups read
// their cell's particles and the unit's B tile from shared memory. A stage
// larger than the buffer is read from global memory instead.

constexpr int kDepThreads = 256;
constexpr int kDepG = 8;                               // lanes per cell
constexpr int kDepCells = kDepThreads / kDepG;         // = kUnitW cells per unit
constexpr int kDepCap = 2176;                          // particles per staged array
constexpr int kDepBuf = 2;                             // stages in flight
constexpr long long kDepMaxPolls = 1ll << 26;          // bounded mbarrier wait
constexpr long long kDepWarpPolls = 1ll << 22;         // bounded wait on the other warps (tiles, refills)
static_assert(kDepCells == kUnitW, "one group of lanes per cell of a unit");

// Register accumulators of one lane: 81 moments S[k][e] and 12 currents.
// The FP32 form packs pairs of alpha' entries so the moment update is 45
// paired FMAs (__ffma2_rn) instead of 81.
template <typename T>
struct Moments {
    T S[81];
    T Jm[12];
    __device__ __forceinline__ void zero()
    {
#pragma unroll
        for (int q = 0; q < 81; ++q) S[q] = T(0);
#pragma unroll
        for (int q = 0; q < 12; ++q) Jm[q] = T(0);
    }
    __device__ __forceinline__ void add(const T (&t)[9], const T (&e)[9])
    {
#pragma unroll
        for (int k = 0; k < 9; ++k)
#pragma unroll
            for (int q = 0; q < 9; ++q) S[k * 9 + q] += t[k] * e[q];
    }
    __device__ __forceinline__ T get(int k, int q) const { return S[k * 9 + q]; }
    template <int G>
    __device__ __forceinline__ void group_reduce()
    {
#pragma unroll
        for (int o = G / 2; o >= 1; o >>= 1) {
#pragma unroll
            for (int q = 0; q < 81; ++q) S[q] += __shfl_xor_sync(0xffffffffu, S[q], o);
#pragma unroll
            for (int q = 0; q < 12; ++q) Jm[q] += __shfl_xor_sync(0xffffffffu, Jm[q], o);
        }
    }
};

template <>
struct Moments<float> {
    // the 81 moments S[k][q] in 81 registers: P[k*4 + h] = (S[k][2h],
    // S[k][2h+1]) for q < 8, Q[m] = (S[2m][8], S[2m+1][8]), R = S[8][8]; all
    // but R accumulate with paired FMAs (FFMA2)
    float2 P[36];
    float2 Q[4];
    float R;
    float Jm[12];
    __device__ __forceinline__ void zero()
    {
#pragma unroll
        for (int q = 0; q < 36; ++q) P[q] = make_float2(0.f, 0.f);
#pragma unroll
        for (int m = 0; m < 4; ++m) Q[m] = make_float2(0.f, 0.f);
        R = 0.f;
#pragma unroll
        for (int q = 0; q < 12; ++q) Jm[q] = 0.f;
    }
    __device__ __forceinline__ void add(const float (&t)[9], const float (&e)[9])
    {
        const float2 e2[4] = {make_float2(e[0], e[1]), make_float2(e[2], e[3]), make_float2(e[4], e[5]),
                              make_float2(e[6], e[7])};
#pragma unroll
        for (int k = 0; k < 9; ++k) {
            const float2 tk = make_float2(t[k], t[k]);
#pragma unroll
            for (int h = 0; h < 4; ++h) P[k * 4 + h] = __ffma2_rn(tk, e2[h], P[k * 4 + h]);
        }
        const float2 e8 = make_float2(e[8], e[8]);
#pragma unroll
        for (int m = 0; m < 4; ++m) Q[m] = __ffma2_rn(make_float2(t[2 * m], t[2 * m + 1]), e8, Q[m]);
        R = fmaf(t[8], e[8], R);
    }
    __device__ __forceinline__ float get(int k, int q) const
    {
        if (q < 8) return (q & 1) ? P[k * 4 + q / 2].y : P[k * 4 + q / 2].x;
        if (k < 8) return (k & 1) ? Q[k / 2].y : Q[k / 2].x;
        return R;
    }
    template <int G>
    __device__ __forceinline__ void group_reduce()
    {
#pragma unroll
        for (int o = G / 2; o >= 1; o >>= 1) {
#pragma unroll
            for (int q = 0; q < 36; ++q) {
                P[q].x += __shfl_xor_sync(0xffffffffu, P[q].x, o);
                P[q].y += __shfl_xor_sync(0xffffffffu, P[q].y, o);
            }
#pragma unroll
            for (int m = 0; m < 4; ++m) {
                Q[m].x += __shfl_xor_sync(0xffffffffu, Q[m].x, o);
                Q[m].y += __shfl_xor_sync(0xffffffffu, Q[m].y, o);
            }
            R += __shfl_xor_sync(0xffffffffu, R, o);
#pragma unroll
            for (int q = 0; q < 12; ++q) Jm[q] += __shfl_xor_sync(0xffffffffu, Jm[q], o);
        }
    }
    // Reduce-scatter over the 8 lanes of a group (recursive halving, partner
    // distances 4, 2, 1): afterwards lane gl holds the group sums of the 12
    // flat values 12 gl .. 12 gl + 11, where lane L's block is S[L][0..8]
    // followed by S[8][3L..3L+2] (L < 3), Jm[3(L-3)..3(L-3)+2] (3 <= L < 7)
    // or zeros (L = 7). Each sum pairs the lanes' values in the order the
    // butterfly of group_reduce does, so the results are the same.
    __device__ __forceinline__ void reduce_scatter8(int gl, float (&r)[12]) const
    {
        float v[96];
#pragma unroll
        for (int L = 0; L < 8; ++L) {
#pragma unroll
            for (int q = 0; q < 9; ++q) v[12 * L + q] = get(L, q);
#pragma unroll
            for (int e = 0; e < 3; ++e)
                v[12 * L + 9 + e] = L < 3 ? get(8, 3 * L + e) : L < 7 ? Jm[3 * (L - 3) + e] : 0.f;
        }
        float h[48];
        const bool b2 = (gl & 4) != 0, b1 = (gl & 2) != 0, b0 = (gl & 1) != 0;
#pragma unroll
        for (int i = 0; i < 48; ++i) {
            const float keep = b2 ? v[48 + i] : v[i], send = b2 ? v[i] : v[48 + i];
            h[i] = keep + __shfl_xor_sync(0xffffffffu, send, 4);
        }
        float g[24];
#pragma unroll
        for (int i = 0; i < 24; ++i) {
            const float keep = b1 ? h[24 + i] : h[i], send = b1 ? h[i] : h[24 + i];
            g[i] = keep + __shfl_xor_sync(0xffffffffu, send, 2);
        }
#pragma unroll
        for (int i = 0; i < 12; ++i) {
            const float keep = b0 ? g[12 + i] : g[i], send = b0 ? g[i] : g[12 + i];
            r[i] = keep + __shfl_xor_sync(0xffffffffu, send, 1);
        }
    }
};

// The node and half offset where the moments S[k][*] of a cell go (k = xx*3
// + yy): nodes 0..3 = n00, n10, n01, n11; S[4][*] goes to (n00, 4) and also
// to (n10, 2). Packed 2 and 3 bits per k for a lane-indexed lookup.
constexpr int kMomNode[9] = {0, 0, 2, 0, 0, 2, 1, 1, 3};
constexpr int kMomOff[9] = {0, 3, 0, 1, 4, 1, 0, 3, 0};
constexpr unsigned pack_bits(const int (&a)[9], int w)
{
    unsigned v = 0;
    for (int k = 0; k < 9; ++k) v |= (unsigned)a[k] << (w * k);
    return v;
}
constexpr unsigned kMomNodeBits = pack_bits(kMomNode, 2);
constexpr unsigned kMomOffBits = pack_bits(kMomOff, 3);

// The deposit's field tiles of a unit: B^n on the centres and, for the
// predicted gamma, E^n on the nodes. The rows are padded to 43 (11 mod 32
// banks): the two rows a warp's B gathers touch, over the six columns of its
// four cells, fall in distinct banks (34 would put row r + 1 column c on
// row r column c + 2).
template <typename T, bool PRED>
struct DepTiles {
    T B[3][3][kTBD];
    PredTile<T, PRED, kTED> En;
    __device__ __forceinline__ void load(const T* __restrict__ Bg, const T* __restrict__ Eg, const Unit& un, int nx,
                                         int ny, int nc, int tid)
    {
        load_tile_B<T, kDepThreads, kTBD>(B, Bg, un, nx, ny, nc, tid);
        if constexpr (PRED) load_tile_E<T, kDepThreads, kTED>(En.En, Eg, un, nx, ny, nc, tid);
    }
    __device__ __forceinline__ void gather_B(int l, T fx, T fy, T& Bx, T& By, T& Bz) const
    {
        tile_B<T, kTBD>(B, l, fx, fy, Bx, By, Bz);
    }
    __device__ __forceinline__ T u2(T ux, T uy, T uz, T beta, int l, T W0, T W1, T W2, T W3, T& sx, T& sy,
                                    T& sz) const
    {
        return gbar_u2<T, PRED, kTED>(ux, uy, uz, beta, En.en(), l, W0, W1, W2, W3, sx, sy, sz);
    }
};

// FP32: every entry holds a value and its right neighbour, so the two
// columns of a gather come in one 64-bit load (six loads for B, six for E^n
// instead of twelve each). Rows of 38 pairs (6 mod 16 bank pairs) keep the
// two rows of a warp's B gathers apart as above.
constexpr int kTBP = 38;
template <bool PRED>
struct DepTiles<float, PRED> {
    float2 B[3][3][kTBP];   // [comp][row j-1, j, j+1][col]: (B(i0-1+col), B(i0+col)), col = 0..cn
    float2 En[PRED ? 3 : 1][2][PRED ? kUnitW : 1];   // [comp][row j, j+1][l]: (E(i0+l), E(i0+l+1))
    __device__ __forceinline__ void load(const float* __restrict__ Bg, const float* __restrict__ Eg, const Unit& un,
                                         int nx, int ny, int nc, int tid)
    {
        for (int idx = tid; idx < 9 * (kUnitW + 1); idx += kDepThreads) {
            const int comp = idx / (3 * (kUnitW + 1)), r = (idx / (kUnitW + 1)) % 3, col = idx % (kUnitW + 1);
            if (col <= un.cn) {
                const int gj = wrap1(un.j - 1 + r, ny);
                const float* row = Bg + comp * nc + gj * nx;
                B[comp][r][col] = make_float2(ld(row + wrap1(un.i0 - 1 + col, nx)), ld(row + wrap1(un.i0 + col, nx)));
            }
        }
        if constexpr (PRED) {
            for (int idx = tid; idx < 6 * kUnitW; idx += kDepThreads) {
                const int comp = idx / (2 * kUnitW), r = (idx / kUnitW) % 2, l = idx % kUnitW;
                if (l < un.cn) {
                    const int gj = wrap1(un.j + r, ny);
                    const float* row = Eg + comp * nc + gj * nx;
                    En[comp][r][l] = make_float2(ld(row + wrap1(un.i0 + l, nx)), ld(row + wrap1(un.i0 + l + 1, nx)));
                }
            }
        }
    }
    __device__ __forceinline__ void gather_B(int l, float fx, float fy, float& Bx, float& By, float& Bz) const
    {
        const bool lx = fx < 0.5f, ly = fy < 0.5f;
        const float tx = lx ? fx + 0.5f : fx - 0.5f;
        const float ty = ly ? fy + 0.5f : fy - 0.5f;
        const int c0 = lx ? l : l + 1;
        const int r0 = ly ? 0 : 1;
        const float w00 = (1.f - tx) * (1.f - ty), w10 = tx * (1.f - ty);
        const float w01 = (1.f - tx) * ty, w11 = tx * ty;
        const float2 x0 = B[0][r0][c0], x1 = B[0][r0 + 1][c0];
        Bx = w00 * x0.x + w10 * x0.y + w01 * x1.x + w11 * x1.y;
        const float2 y0 = B[1][r0][c0], y1 = B[1][r0 + 1][c0];
        By = w00 * y0.x + w10 * y0.y + w01 * y1.x + w11 * y1.y;
        const float2 z0 = B[2][r0][c0], z1 = B[2][r0 + 1][c0];
        Bz = w00 * z0.x + w10 * z0.y + w01 * z1.x + w11 * z1.y;
    }
    __device__ __forceinline__ float u2(float ux, float uy, float uz, float beta, int l, float W0, float W1,
                                        float W2, float W3, float& sx, float& sy, float& sz) const
    {
        if constexpr (!PRED) {
            sx = ux;
            sy = uy;
            sz = uz;
            return ux * ux + uy * uy + uz * uz;
        } else {
            // one component at a time, as in gbar_u2
            const float2 a0 = En[0][0][l], a1 = En[0][1][l];
            sx = ux + beta * (W0 * a0.x + W1 * a0.y + W2 * a1.x + W3 * a1.y);
            asm volatile("" ::: "memory");
            const float2 b0 = En[1][0][l], b1 = En[1][1][l];
            sy = uy + beta * (W0 * b0.x + W1 * b0.y + W2 * b1.x + W3 * b1.y);
            asm volatile("" ::: "memory");
            const float2 c0 = En[2][0][l], c1 = En[2][1][l];
            sz = uz + beta * (W0 * c0.x + W1 * c0.y + W2 * c1.x + W3 * c1.y);
            asm volatile("" ::: "memory");
            return sx * sx + sy * sy + sz * sz;
        }
    }
};

template <typename T, bool PRED>
__device__ __forceinline__ void deposit_particle(const T fx, const T fy, const T ux, const T uy, const T uz,
                                                 const T w, const DepTiles<T, PRED>& tl, int l, T beta, T cJ,
                                                 T cM, Moments<T>& acc)
{
    T Bx, By, Bz;
    tl.gather_B(l, fx, fy, Bx, By, Bz);
    T sx, sy, sz;
    const T u2 = tl.u2(ux, uy, uz, beta, l, (T(1) - fx) * (T(1) - fy), fx * (T(1) - fy), (T(1) - fx) * fy,
                       fx * fy, sx, sy, sz);
    const Rot<T> r = rotation<T>(u2, Bx, By, Bz, beta);
    const T ax = r.ax, ay = r.ay, az = r.az;
    T e[9];
    e[0] = T(1) + ax * ax; e[1] = ax * ay + az;   e[2] = ax * az - ay;
    e[3] = ax * ay - az;   e[4] = T(1) + ay * ay; e[5] = ay * az + ax;
    e[6] = ax * az + ay;   e[7] = ay * az - ax;   e[8] = T(1) + az * az;
    // predicted current: w q alpha u / gbar / dV at the 4 nodes
    const T cj = w * cJ * r.sa * r.ig;
    const T vx = cj * (e[0] * ux + e[1] * uy + e[2] * uz);
    const T vy = cj * (e[3] * ux + e[4] * uy + e[5] * uz);
    const T vz = cj * (e[6] * ux + e[7] * uy + e[8] * uz);
    const T X0 = T(1) - fx, X1 = fx, Y0 = T(1) - fy, Y1 = fy;
    const T W[4] = {X0 * Y0, X1 * Y0, X0 * Y1, X1 * Y1};
#pragma unroll
    for (int a = 0; a < 4; ++a) {
        acc.Jm[a * 3 + 0] += W[a] * vx;
        acc.Jm[a * 3 + 1] += W[a] * vy;
        acc.Jm[a * 3 + 2] += W[a] * vz;
    }
    const T cm = w * cM * r.sa * r.ig;
    const T xx[3] = {cm * X0 * X0, cm * X0 * X1, cm * X1 * X1};
    const T yy[3] = {Y0 * Y0, Y0 * Y1, Y1 * Y1};
    T t[9];
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b) t[a * 3 + b] = xx[a] * yy[b];
    acc.add(t, e);
}

// the instance of a shared launch that owns global unit u: the last whose
// first unit is <= u (the descriptors ascend in unit0)
template <typename D>
__device__ __forceinline__ int find_inst(const D* __restrict__ d, int n, int u)
{
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (d[mid].unit0 <= u) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// Where the deposit's units come from: one instance (the kernel's own
// arguments) or the instances of a shared launch (units numbered across them;
// the stage of a unit takes its instance's particles, fields and grid).
template <typename T>
struct DepSingle {
    const DepositSpecies<T>* sp;   // the kernel's own (grid-constant) argument
    const T* B;
    const T* En;
    T* M;
    T* J;
    GridP g;
    __device__ __forceinline__ int nsp() const { return sp->nsp; }
    __device__ __forceinline__ int nunits() const { return units_of(g.nx, g.ny); }
    __device__ __forceinline__ int inst(int) const { return 0; }
    __device__ __forceinline__ int unit(int, int gu) const { return gu; }
    __device__ __forceinline__ GridP grid(int) const { return g; }
    __device__ __forceinline__ const int32_t* start(int, int s) const { return sp->start[s]; }
    __device__ __forceinline__ const T* arr(int, int a, int s) const
    {
        return a == 0 ? sp->fx[s] : a == 1 ? sp->fy[s] : a == 2 ? sp->ux[s] : a == 3 ? sp->uy[s]
               : a == 4 ? sp->uz[s] : sp->w[s];
    }
    __device__ __forceinline__ T beta(int, int s) const { return sp->beta[s]; }
    __device__ __forceinline__ T cJ(int, int s) const { return sp->cJ[s]; }
    __device__ __forceinline__ T cM(int, int s) const { return sp->cM[s]; }
    __device__ __forceinline__ const T* Bf(int) const { return B; }
    __device__ __forceinline__ const T* Enf(int) const { return En; }
    __device__ __forceinline__ T* Mf(int) const { return M; }
    __device__ __forceinline__ T* Jf(int) const { return J; }
};

template <typename T>
struct DepBatch {
    const DepDesc<T>* __restrict__ d;
    int n, total;
    __device__ __forceinline__ int nsp() const { return d[0].ds.nsp; }
    __device__ __forceinline__ int nunits() const { return total; }
    __device__ __forceinline__ int inst(int gu) const { return find_inst(d, n, gu); }
    __device__ __forceinline__ int unit(int i, int gu) const { return gu - d[i].unit0; }
    __device__ __forceinline__ GridP grid(int i) const { return d[i].g; }
    __device__ __forceinline__ const int32_t* start(int i, int s) const { return d[i].ds.start[s]; }
    __device__ __forceinline__ const T* arr(int i, int a, int s) const
    {
        const DepositSpecies<T>& sp = d[i].ds;
        return a == 0 ? sp.fx[s] : a == 1 ? sp.fy[s] : a == 2 ? sp.ux[s] : a == 3 ? sp.uy[s] : a == 4 ? sp.uz[s] : sp.w[s];
    }
    __device__ __forceinline__ T beta(int i, int s) const { return d[i].ds.beta[s]; }
    __device__ __forceinline__ T cJ(int i, int s) const { return d[i].ds.cJ[s]; }
    __device__ __forceinline__ T cM(int i, int s) const { return d[i].ds.cM[s]; }
    __device__ __forceinline__ const T* Bf(int i) const { return d[i].B; }
    __device__ __forceinline__ const T* Enf(int i) const { return d[i].En; }
    __device__ __forceinline__ T* Mf(int i) const { return d[i].M; }
    __device__ __forceinline__ T* Jf(int i) const { return d[i].J; }
};

// The deposit body. The block's warps share no barrier inside the stage
// loop: each (unit, species) stage sits in one of two staging buffers,
// filled by TMA bulk copies (an mbarrier per buffer counts the bytes), and
// the warp that finishes a stage last refills its buffer with the stage two
// ahead (its particle range brought into shared memory by an asynchronous
// copy one stage earlier); a unit's
// field tiles alternate between two copies, which every thread fills one
// unit ahead, with an mbarrier that counts the threads' stores (full) and
// one that counts the warps done with the unit (free). So the warps drift
// apart by up to a unit instead of meeting at every stage, and a stage's
// uneven cells no longer hold the block back. Every wait is bounded; a warp
// that gives up raises the block's abort flag, the others leave at their
// next wait, and the copies in flight land before the block exits.
template <typename T, bool PRED, class Src>
__device__ __forceinline__ void deposit_core(const Src& src, int* __restrict__ err)
{
    constexpr int G = kDepG;
    constexpr int NB = kDepBuf;
    constexpr int NW = kDepThreads / 32;
    constexpr int A = 16 / sizeof(T);   // elements per 16 bytes (TMA granule)
    extern __shared__ __align__(128) unsigned char dsmem[];
    __shared__ uint64_t mbar[NB];    // staged particles landed
    __shared__ uint64_t tfull[2];    // a tile copy stored (kDepThreads arrivals)
    __shared__ uint64_t tfree[2];    // every warp done with that copy's unit (NW arrivals)
    __shared__ int sp0a[NB];         // aligned first particle of the staged range
    __shared__ int sstaged[NB];      // 1 if staged in shared memory, 0 if read from global
    __shared__ int sdone[NB];        // warps done with the stage in the buffer
    __shared__ int slast[NB];        // the last stage issued into the buffer
    __shared__ volatile int sabort;
    __shared__ int srng[NW][2];      // each warp's copy of the range two stages ahead
    __shared__ DepTiles<T, PRED> stl[2];
    T* buf = reinterpret_cast<T*>(dsmem);
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const int gl = tid % G, grp = tid / G;
    const int nsp = src.nsp();
    const int nunits = src.nunits();
    const int myunits = blockIdx.x < nunits ? (nunits - 1 - blockIdx.x) / gridDim.x + 1 : 0;
    const int nstages = myunits * nsp;
    if (nstages == 0) return;

    // the range of stage k's particles (lane-local loads of the start table)
    auto range_of = [&](int k, int& p0, int& p1) {
        const int gu = blockIdx.x + (k / nsp) * gridDim.x;
        const int ii = src.inst(gu);
        const Unit un = unit_of(src.unit(ii, gu), src.grid(ii).nx);
        const int32_t* st0 = src.start(ii, k % nsp);
        p0 = st0[un.c0];
        p1 = st0[un.c0 + un.cn];
    };
    // one lane: start the copies of stage k (particles p0 .. p1) into buffer k % NB
    auto issue = [&](int k, int p0, int p1) {
        const int b = k % NB;
        const int gu = blockIdx.x + (k / nsp) * gridDim.x;
        const int ii = src.inst(gu);
        const int s = k % nsp;
        const int p0a = p0 & ~(A - 1);
        const int p1a = (p1 + A - 1) & ~(A - 1);
        const int cnt = p1a - p0a;
        sp0a[b] = p0a;
        slast[b] = k;
        if (p1 > p0 && cnt <= kDepCap) {
            sstaged[b] = 1;
            const unsigned bytes = (unsigned)(cnt * sizeof(T));
            mbar_expect_tx_arrive(&mbar[b], 6 * bytes);
            T* dst = buf + (size_t)b * 6 * kDepCap;
#pragma unroll
            for (int a2 = 0; a2 < 6; ++a2) bulk_g2s(dst + a2 * kDepCap, src.arr(ii, a2, s) + p0a, bytes, &mbar[b]);
        } else {
            sstaged[b] = 0;
            mbar_expect_tx_arrive(&mbar[b], 0);
        }
    };
    // every thread: its share of unit u's tiles into copy u % 2, then one arrival
    auto load_tiles = [&](int u) {
        const int gu = blockIdx.x + u * gridDim.x;
        const int ii = src.inst(gu);
        const GridP gg = src.grid(ii);
        const Unit un = unit_of(src.unit(ii, gu), gg.nx);
        stl[u & 1].load(src.Bf(ii), src.Enf(ii), un, gg.nx, gg.ny, gg.ncell, tid);
        mbar_arrive(&tfull[u & 1]);
    };

    if (tid == 0) {
        for (int b = 0; b < NB; ++b) {
            mbar_init(&mbar[b], 1);
            sdone[b] = 0;
            slast[b] = -1;
        }
        for (int x = 0; x < 2; ++x) {
            mbar_init(&tfull[x], kDepThreads);
            mbar_init(&tfree[x], NW);
        }
        sabort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    if (tid == 0)
        for (int k = 0; k < NB && k < nstages; ++k) {
            int p0, p1;
            range_of(k, p0, p1);
            issue(k, p0, p1);
        }
    load_tiles(0);

    Moments<T> acc;
    bool ok = true;
    for (int k = 0; k < nstages; ++k) {
        const int b = k % NB;
        const int u = k / nsp, s = k % nsp;
        const int gu = blockIdx.x + u * gridDim.x;
        const int ii = src.inst(gu);
        const GridP gg = src.grid(ii);
        const int nx = gg.nx, ny = gg.ny, nc = gg.ncell;
        const Unit un = unit_of(src.unit(ii, gu), nx);
        if (s == 0) {
            acc.zero();
            if (u + 1 < myunits) {
                // copy (u+1) % 2 last held unit u - 1: wait until every warp is done with it
                if (u >= 1) ok = mbar_wait_or_abort(&tfree[(u + 1) & 1], (unsigned)(((u - 1) >> 1) & 1),
                                                    kDepWarpPolls, &sabort);
                ok = __all_sync(0xffffffffu, ok);   // the warp leaves as one
                if (!ok) break;
                load_tiles(u + 1);
            }
            ok = mbar_wait_or_abort(&tfull[u & 1], (unsigned)((u >> 1) & 1), kDepWarpPolls, &sabort);
            ok = __all_sync(0xffffffffu, ok);
            if (!ok) break;
        }
        // the range of the stage this buffer takes next: copied into the
        // warp's slot by an asynchronous copy while this stage runs (no
        // registers held across the stage)
        if (lane == 0 && k + NB < nstages) {
            const int kn = k + NB;
            const int gun = blockIdx.x + (kn / nsp) * gridDim.x;
            const int iin = src.inst(gun);
            const Unit unn = unit_of(src.unit(iin, gun), src.grid(iin).nx);
            const int32_t* stn = src.start(iin, kn % nsp);
            // the slot's previous copy (a stage old, long landed) completes
            // first: two copies in flight to one address land in no fixed order
            asm volatile("cp.async.wait_all;" ::: "memory");
            cp_async4(&srng[wid][0], stn + unn.c0);
            cp_async4(&srng[wid][1], stn + unn.c0 + unn.cn);
            asm volatile("cp.async.commit_group;" ::: "memory");
        }
        ok = mbar_wait_or_abort(&mbar[b], (unsigned)((k / NB) & 1), kDepWarpPolls, &sabort);
        ok = __all_sync(0xffffffffu, ok);
        if (!ok) break;
        const DepTiles<T, PRED>& tl = stl[u & 1];
        const bool valid = grp < un.cn;
        const int c = un.c0 + grp;
        if (valid) {
            const int32_t* st0 = src.start(ii, s);
            const int p0 = st0[c], p1 = st0[c + 1];
            const T beta = src.beta(ii, s), cJ = src.cJ(ii, s), cM = src.cM(ii, s);
            if (sstaged[b]) {
                const T* sb = buf + (size_t)b * 6 * kDepCap - sp0a[b];
                for (int p = p0 + gl; p < p1; p += G)
                    deposit_particle<T, PRED>(sb[p], sb[kDepCap + p], sb[2 * kDepCap + p], sb[3 * kDepCap + p],
                                              sb[4 * kDepCap + p], sb[5 * kDepCap + p], tl, grp, beta, cJ, cM,
                                              acc);
            } else {
                const T *gfx = src.arr(ii, 0, s), *gfy = src.arr(ii, 1, s), *gux = src.arr(ii, 2, s),
                        *guy = src.arr(ii, 3, s), *guz = src.arr(ii, 4, s), *gw = src.arr(ii, 5, s);
                for (int p = p0 + gl; p < p1; p += G)
                    deposit_particle<T, PRED>(ld(gfx + p), ld(gfy + p), ld(gux + p), ld(guy + p), ld(guz + p),
                                              ld(gw + p), tl, grp, beta, cJ, cM, acc);
            }
        }
        if (s == nsp - 1) {
            T* const M = src.Mf(ii);
            T* const J = src.Jf(ii);
            if constexpr (std::is_same<T, float>::value) {
                static_assert(G == 8, "the FP32 flush scatters over 8 lanes");
                float r[12];
                acc.reduce_scatter8(gl, r);
                if (valid) {
                    const int i = un.i0 + grp, j = un.j;
                    const int i1 = wrap1(i + 1, nx), j1 = wrap1(j + 1, ny);
                    const int n00 = j * nx + i, n10 = j * nx + i1, n01 = j1 * nx + i, n11 = j1 * nx + i1;
                    // lane gl: S[gl][0..8] to its node and offset (S[4] twice)
                    const int nd = (kMomNodeBits >> (2 * gl)) & 3, of = (kMomOffBits >> (3 * gl)) & 7;
                    const int nn = nd == 0 ? n00 : nd == 1 ? n10 : nd == 2 ? n01 : n11;
                    float* const mk = M + (int64_t)nn * kMBlock + of * 9;
#pragma unroll
                    for (int q = 0; q < 9; ++q) atomicAdd(mk + q, r[q]);
                    if (gl == 4) {
                        float* const m4 = M + (int64_t)n10 * kMBlock + 2 * 9;
#pragma unroll
                        for (int q = 0; q < 9; ++q) atomicAdd(m4 + q, r[q]);
                    }
                    // the extras: S[8][3gl..3gl+2] (node n11, offset 0) or the
                    // currents of node gl - 3, components 0..2
                    if (gl < 3) {
                        float* const m8 = M + (int64_t)n11 * kMBlock + 3 * gl;
#pragma unroll
                        for (int e = 0; e < 3; ++e) atomicAdd(m8 + e, r[9 + e]);
                    } else if (gl < 7) {
                        const int a = gl - 3;
                        const int jn = a == 0 ? n00 : a == 1 ? n10 : a == 2 ? n01 : n11;
#pragma unroll
                        for (int e = 0; e < 3; ++e) atomicAdd(J + (int64_t)e * nc + jn, r[9 + e]);
                    }
                }
            } else {
                acc.template group_reduce<G>();
                if (valid) {
                    const int i = un.i0 + grp, j = un.j;
                    const int i1 = wrap1(i + 1, nx), j1 = wrap1(j + 1, ny);
                    const int n00 = j * nx + i, n10 = j * nx + i1, n01 = j1 * nx + i, n11 = j1 * nx + i1;
                    // (destination node, half offset, moment k) of the ten node pairs
                    const int pn[10] = {n00, n00, n00, n00, n10, n10, n10, n01, n01, n11};
                    constexpr int po[10] = {0, 1, 3, 4, 0, 2, 3, 0, 1, 0};
                    constexpr int pk[10] = {0, 3, 1, 4, 6, 4, 7, 2, 5, 8};
#pragma unroll
                    for (int it = 0; it < 90; ++it) {
                        if (it % G == gl) {
                            const int pr = it / 9, q = it % 9;
                            atomicAdd(M + (int64_t)pn[pr] * kMBlock + po[pr] * 9 + q, acc.get(pk[pr], q));
                        }
                    }
                    const int jn[4] = {n00, n10, n01, n11};
#pragma unroll
                    for (int it = 0; it < 12; ++it)
                        if ((90 + it) % G == gl) atomicAdd(J + (int64_t)(it % 3) * nc + jn[it / 3], acc.Jm[it]);
                }
            }
        }
        // the warp is done with buffer b (and, after its unit's last stage,
        // with the tile copy); the last warp out refills the buffer
        __syncwarp();
        if (lane == 0) {
            if (atomicAdd(&sdone[b], 1) == NW - 1) {
                sdone[b] = 0;
                if (k + NB < nstages) {
                    asm volatile("cp.async.wait_all;" ::: "memory");
                    issue(k + NB, srng[wid][0], srng[wid][1]);
                }
            }
            if (s == nsp - 1) mbar_arrive(&tfree[u & 1]);
        }
    }
    if (!ok) {
        sabort = 1;
        if (lane == 0) atomicOr(err, 2);
    }
    // every warp out of the loop, its range copies landed; then the bulk
    // copies still in flight land (bounded)
    asm volatile("cp.async.wait_all;" ::: "memory");
    __syncthreads();
    if (sabort && tid == 0)
        for (int b = 0; b < NB; ++b)
            if (slast[b] >= 0) mbar_wait(&mbar[b], (unsigned)((slast[b] / NB) & 1), kDepMaxPolls);
}

template <typename T, bool PRED>
__global__ void __launch_bounds__(kDepThreads, sizeof(T) == 4 ? 2 : 1)
k_deposit(const __grid_constant__ DepositSpecies<T> sp, const T* __restrict__ B, const T* __restrict__ En,
          T* __restrict__ M, T* __restrict__ J, GridP g, int* __restrict__ err)
{
    const DepSingle<T> src{&sp, B, En, M, J, g};
    deposit_core<T, PRED>(src, err);
}

// the deposit over the units of several instances in one launch
template <typename T, bool PRED>
__global__ void __launch_bounds__(kDepThreads, sizeof(T) == 4 ? 2 : 1)
k_deposit_batch(const DepDesc<T>* __restrict__ descs, int ninst, int total_units, int* __restrict__ err)
{
    const DepBatch<T> src{descs, ninst, total_units};
    deposit_core<T, PRED>(src, err);
}

// ---------------------------------------------------------------------------
// push. A warp owns a unit (a row segment of up to 32 cells), whose particles
// are one contiguous range of the sorted arrays, and gathers E^{n+theta} and
// B^n from the unit's shared field tile.
//
// The re-sort by the new cell takes two kernels. k_push_sort pushes each
// cell's particles once (batches of 32 lanes), ranks them per move
// direction d = (sy+1)*3 + (sx+1) with ballots (in particle order), keeps the
// pushed records in shared memory and writes the cell back over its own
// index range grouped by direction (coalesced stores). Runs (old cell c,
// direction d) are then contiguous: n9[c][d] particles starting at
// off9[c][d]. k_permute builds the new order: the particles of new cell k
// are the nine runs that end in k, in ascending order of their old cell
// (the stable counting sort), copied with coalesced stores. A particle moves
// at most one cell per step when c dt <= min(dx, dy); otherwise the library
// takes the general path (k_push_general + radix sort).

template <typename T> struct PushCfg {
    static constexpr int warps = 4;                        // static shared memory < 48 KB
    static constexpr int threads = 32 * warps;
    static constexpr int min_blocks = sizeof(T) == 4 ? 5 : 2;
    static constexpr int cap = sizeof(T) == 4 ? 256 : 128;   // particles of a cell group staged per warp
    // with the E^n tile of the predicted gamma (3 KB more per block in
    // FP32) a smaller group keeps five blocks on an SM
    static constexpr int cap_pred = sizeof(T) == 4 ? 224 : 128;
};
constexpr int kGroupMax = 8;    // cells staged together at most
constexpr int kLedger = 4;      // dK, work, mismatch, K1 (K0 is the previous K1)

template <typename T>
struct Pushed {
    T fxn, fyn, u1x, u1y, u1z, w;
    int sx, sy, dir;
};

// the explicit push of one particle: E^{n+theta}, B^n gathered at x^{n+1/2},
// ubar = alpha (u + beta E), u1 = 2 ubar - u, x += dt u1/gamma1; ledger sums
template <typename T, bool PRED>
__device__ __forceinline__ void push_particle(const T fx, const T fy, const T ux, const T uy, const T uz,
                                              const T w, int l, const T (*sE)[2][kTE],
                                              const T (*sB)[3][kTB], const T (*sEn)[2][kTE], T beta, T dt_dx,
                                              T dt_dy, T qdt, T m, bool clamp, bool ledger, T (&acc)[kLedger],
                                              Pushed<T>& o)
{
    T Bx, By, Bz, Ex, Ey, Ez;
    tile_B(sB, l, fx, fy, Bx, By, Bz);
    const T X0 = T(1) - fx, Y0 = T(1) - fy;
    tile_E(sE, l, X0 * Y0, fx * Y0, X0 * fy, fx * fy, Ex, Ey, Ez);
    const T u02 = ux * ux + uy * uy + uz * uz;
    T psx, psy, psz;   // the momentum whose Lorentz factor is gbar
    const T us2 = gbar_u2<T, PRED>(ux, uy, uz, beta, sEn, l, X0 * Y0, fx * Y0, X0 * fy, fx * fy, psx, psy, psz);
    const Rot<T> r = rotation<T>(us2, Bx, By, Bz, beta);
    const T ax = r.ax, ay = r.ay, az = r.az, sa = r.sa;
    // ubar = alpha w = (w + w x a + (w.a) a)/(1 + |a|^2), w = u + beta E
    const T wx = ux + beta * Ex, wy = uy + beta * Ey, wz = uz + beta * Ez;
    const T wa = wx * ax + wy * ay + wz * az;
    const T ubx = sa * (wx + (wy * az - wz * ay) + wa * ax);
    const T uby = sa * (wy + (wz * ax - wx * az) + wa * ay);
    const T ubz = sa * (wz + (wx * ay - wy * ax) + wa * az);
    o.u1x = T(2) * ubx - ux;
    o.u1y = T(2) * uby - uy;
    o.u1z = T(2) * ubz - uz;
    o.w = w;
    const T u12 = o.u1x * o.u1x + o.u1y * o.u1y + o.u1z * o.u1z;
    const T ig1 = rsqrt_t(T(1) + u12);
    // x^{n+3/2} = x^{n+1/2} + dt u^{n+1}/gamma^{n+1}, as cell shift + offset
    const T tx = fx + dt_dx * (o.u1x * ig1);
    const T ty = fy + dt_dy * (o.u1y * ig1);
    const T flx = floor(tx), fly = floor(ty);
    int sx = (int)flx, sy = (int)fly;
    T fxn = tx - flx, fyn = ty - fly;
    if (fxn >= T(1)) { fxn -= T(1); sx += 1; }
    if (fyn >= T(1)) { fyn -= T(1); sy += 1; }
    if (clamp) {
        // with c dt <= dx a move of more than one cell can only come from
        // rounding at |v| = c; keep the particle on the last representable
        // point of the neighbour cell
        if (sx > 1) { sx = 1; fxn = Consts<T>::one_below(); }
        if (sx < -1) { sx = -1; fxn = T(0); }
        if (sy > 1) { sy = 1; fyn = Consts<T>::one_below(); }
        if (sy < -1) { sy = -1; fyn = T(0); }
    }
    o.fxn = fxn;
    o.fyn = fyn;
    o.sx = sx;
    o.sy = sy;
    o.dir = (sy + 1) * 3 + (sx + 1);
    if (ledger) {
        const T g1 = (T(1) + u12) * ig1;
        const T ue = ubx * Ex + uby * Ey + ubz * Ez;
        // g0 - g1 = (u0 - u1).(u0 + u1)/(g0 + g1)
        const T du = (ux - o.u1x) * (ux + o.u1x) + (uy - o.u1y) * (uy + o.u1y) +
                     (uz - o.u1z) * (uz + o.u1z);
        if (!PRED) {
            const T g0 = (T(1) + u02) * r.ig;   // gbar = g0
            const T igs = rcp_t(g0 + g1);
            acc[0] -= w * m * du * igs;                          // dK
            acc[1] += qdt * w * ue * r.ig;                       // work
            acc[2] += qdt * w * ue * du * igs * igs * r.ig;      // mismatch
        } else {
            // 2/(g0+g1) - 1/gbar = ((gbar-g0) + (gbar-g1))/(gbar (g0+g1)),
            // gbar^2 - g^2 = |u*|^2 - |u|^2
            const T g0 = (T(1) + u02) * rsqrt_t(T(1) + u02);
            const T gb = (T(1) + us2) * r.ig;
            const T igs = rcp_t(g0 + g1);
            const T d0 = (psx - ux) * (psx + ux) + (psy - uy) * (psy + uy) + (psz - uz) * (psz + uz);
            const T d1 = (psx - o.u1x) * (psx + o.u1x) + (psy - o.u1y) * (psy + o.u1y) +
                         (psz - o.u1z) * (psz + o.u1z);
            const T dif = d0 * rcp_t(gb + g0) + d1 * rcp_t(gb + g1);
            acc[0] -= w * m * du * igs;                          // dK
            acc[1] += qdt * w * ue * r.ig;                       // work
            acc[2] += qdt * w * ue * dif * igs * r.ig;           // mismatch
        }
        acc[3] += w * m * u12 * rcp_t(g1 + T(1));            // K1
    }
}

template <typename T>
struct PushTile {
    T B[3][3][kTB];
    T E[3][2][kTE];
};

// a cell's pushed particles, staged for the write back in direction order
// a group of cells' pushed particles, staged for the write back in cell and
// direction order
template <typename T, int C>
struct PushStage {
    T fx[C], fy[C], ux[C], uy[C], uz[C], w[C];
    int32_t id[C];
    uint8_t dir[C], rank[C], inv[C], cell[C];
    int doff[kGroupMax * (kNDir + 1)];
    int run[kGroupMax * kNDir];
};
static_assert(PushCfg<float>::cap <= 256 && PushCfg<double>::cap <= 256 && PushCfg<float>::cap_pred <= 256 &&
                  PushCfg<double>::cap_pred <= 256,
              "uint8 staging indices");

template <typename T>
__device__ __forceinline__ void block_ledger(const T (&acc)[kLedger], double* red, double* __restrict__ lsum)
{
    double out[kLedger];
    if constexpr (sizeof(T) == 4) {
        // FP32 sums as double-float pairs (error-free additions on the FP32
        // pipe), one conversion to FP64 per block
        dfl v[kLedger];
#pragma unroll
        for (int s = 0; s < kLedger; ++s) v[s] = dfl{acc[s], 0.f};
        df_block_sum<kLedger>(v, reinterpret_cast<dfl*>(red), out);
    } else {
        double v[kLedger];
#pragma unroll
        for (int s = 0; s < kLedger; ++s) v[s] = (double)acc[s];
        block_sum<kLedger>(v, red, out);
    }
    if (threadIdx.x == 0)
#pragma unroll
        for (int s = 0; s < kLedger; ++s) lsum[(int64_t)blockIdx.x * kLedger + s] = out[s];
}

// load a unit's cell starts (ss[0..cn]) and field tiles
template <typename T>
__device__ __forceinline__ void unit_setup(const Unit& un, const int32_t* __restrict__ start, int* ss,
                                           PushTile<T>& tl, const T* __restrict__ Eth, const T* __restrict__ B,
                                           int nx, int ny, int nc, int lane)
{
#pragma unroll
    for (int k0 = 0; k0 <= kUnitW; k0 += 32)
        if (k0 + lane <= un.cn) ss[k0 + lane] = start[un.c0 + k0 + lane];
    load_tile_B<T, 32>(tl.B, B, un, nx, ny, nc, lane);
    load_tile_E<T, 32>(tl.E, Eth, un, nx, ny, nc, lane);
    __syncwarp();
}

// lanes 0..9 store the exclusive prefix of the per-direction counts run[]:
// doff[d] = run[0] + .. + run[d-1], doff[9] = the total
__device__ __forceinline__ void store_doff(const int* run, int* doff, int lane)
{
    int v = 0;
#pragma unroll
    for (int d = 0; d < kNDir; ++d) v += d < lane ? run[d] : 0;
    if (lane <= kNDir) doff[lane] = v;
}

// the warp's ledger sums of one unit added to an instance's slots (FP64)
template <typename T>
__device__ __forceinline__ void ledger_to_instance(T (&acc)[kLedger], double* led, int lane)
{
#pragma unroll
    for (int s = 0; s < kLedger; ++s) {
        double v;
        if constexpr (sizeof(T) == 4) v = df_to_double(df_warp_sum(dfl{acc[s], 0.f}));   // FP32 pipe
        else v = warp_sum((double)acc[s]);
        if (lane == 0) atomicAdd(led + s, v);
        acc[s] = T(0);
    }
}

// The push body, shared by the single-instance kernel and the shared launch
// over several instances (BATCH: units numbered across the instances of
// descs; each unit takes its instance's arrays, fields, grid and constants,
// and its ledger sums go to that instance's slots).
template <typename T, bool PRED, bool BATCH>
__device__ __forceinline__ void push_sort_core(PArrays<T> src, PArrays<T> dst, const int32_t* __restrict__ start,
                                               int32_t* __restrict__ n9, int32_t* __restrict__ off9,
                                               const T* __restrict__ Eth, const T* __restrict__ B,
                                               const T* __restrict__ En, GridP g, T beta, T dt_dx, T dt_dy, T qdt,
                                               T m, double* __restrict__ lsum, const PushDesc<T>* __restrict__ descs,
                                               int ninst, int total_units)
{
    constexpr int W = PushCfg<T>::warps;
    __shared__ int sstart[W][kUnitW + 1];
    __shared__ PushTile<T> stile[W];
    __shared__ PredTile<T, PRED> sen[W];
    constexpr int CAP = PRED ? PushCfg<T>::cap_pred : PushCfg<T>::cap;
    __shared__ PushStage<T, CAP> sstage[W];
    __shared__ double red[32 * kLedger];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nwarps = (gridDim.x * blockDim.x) >> 5;
    int nx = g.nx, ny = g.ny, nc = g.ncell;
    const int nunits = BATCH ? total_units : units_of(nx, ny);
    const unsigned lt = (1u << lane) - 1u;
    int* ss = sstart[wib];
    PushTile<T>& tl = stile[wib];
    PushStage<T, CAP>& st = sstage[wib];
    bool ids = dst.id != nullptr;
    T acc[kLedger] = {T(0), T(0), T(0), T(0)};

    for (int ug = warp; ug < nunits; ug += nwarps) {
        int u = ug;
        double* led = nullptr;
        if constexpr (BATCH) {
            const PushDesc<T>& d = descs[find_inst(descs, ninst, ug)];
            src = d.src;
            dst = d.dst;
            start = d.start;
            n9 = d.n9;
            off9 = d.off9;
            Eth = d.Eth;
            B = d.B;
            if constexpr (PRED) En = d.En;
            nx = d.g.nx;
            ny = d.g.ny;
            nc = d.g.ncell;
            beta = d.beta;
            dt_dx = d.dt_dx;
            dt_dy = d.dt_dy;
            qdt = d.qdt;
            m = d.m;
            led = d.led;
            ids = dst.id != nullptr;
            u = ug - d.unit0;
        }
        const Unit un = unit_of(u, nx);
        unit_setup<T>(un, start, ss, tl, Eth, B, nx, ny, nc, lane);
        if constexpr (PRED) {
            load_tile_E<T, 32>(sen[wib].En, En, un, nx, ny, nc, lane);
            __syncwarp();
        }
        const int P1 = ss[un.cn];
        int pf_pos = -1;   // the first particle of the prefetched batch
        T pfx = T(0), pfy = T(0), pux = T(0), puy = T(0), puz = T(0), pw = T(0);
        for (int l = 0; l < un.cn;) {
            const int s0 = ss[l];
            if (ss[l + 1] - s0 > CAP) {
                // a big cell alone: a counting pass (no ledger, nothing
                // written), then every particle written to its slot directly
                const int s1 = ss[l + 1];
                int* run = st.run;
                if (lane < kNDir) run[lane] = 0;
                __syncwarp();
                for (int b0 = s0; b0 < s1; b0 += 32) {
                    const int p = b0 + lane;
                    const bool act = p < s1;
                    const int q = act ? p : s0;
                    Pushed<T> o;
                    push_particle<T, PRED>(ld(src.fx + q), ld(src.fy + q), ld(src.ux + q), ld(src.uy + q),
                                           ld(src.uz + q), ld(src.w + q), l, tl.E, tl.B, sen[wib].en(), beta,
                                           dt_dx, dt_dy, qdt, m, true, false, acc, o);
                    const unsigned peers = __match_any_sync(0xffffffffu, act ? o.dir : 1024 + lane);
                    if (act && (peers & lt) == 0) run[o.dir] += __popc(peers);
                    __syncwarp();
                }
                store_doff(run, st.doff, lane);
                __syncwarp();
                if (lane < kNDir) run[lane] = 0;
                __syncwarp();
                for (int b0 = s0; b0 < s1; b0 += 32) {
                    const int p = b0 + lane;
                    const bool act = p < s1;
                    const int q = act ? p : s0;
                    T fx, fy, ux, uy, uz, w;
                    if (pf_pos == b0) {
                        fx = pfx; fy = pfy; ux = pux; uy = puy; uz = puz; w = pw;
                    } else {
                        fx = ld(src.fx + q); fy = ld(src.fy + q); ux = ld(src.ux + q);
                        uy = ld(src.uy + q); uz = ld(src.uz + q); w = ld(src.w + q);
                    }
                    pf_pos = -1;
                    Pushed<T> o;
                    push_particle<T, PRED>(fx, fy, ux, uy, uz, act ? w : T(0), l, tl.E, tl.B, sen[wib].en(), beta,
                                           dt_dx, dt_dy, qdt, m, true, true, acc, o);
                    const unsigned peers = __match_any_sync(0xffffffffu, act ? o.dir : 1024 + lane);
                    const int rank = (act ? run[o.dir] : 0) + __popc(peers & lt);
                    __syncwarp();
                    if (act && (peers & lt) == 0) run[o.dir] += __popc(peers);
                    __syncwarp();
                    if (act) {
                        const int pos = s0 + st.doff[o.dir] + rank;
                        dst.fx[pos] = o.fxn;
                        dst.fy[pos] = o.fyn;
                        dst.ux[pos] = o.u1x;
                        dst.uy[pos] = o.u1y;
                        dst.uz[pos] = o.u1z;
                        dst.w[pos] = o.w;
                        if (ids) dst.id[pos] = src.id[p];
                    }
                }
                const int c = un.c0 + l;
                if (lane < kNDir) {
                    n9[(int64_t)c * kNDir + lane] = st.doff[lane + 1] - st.doff[lane];
                    off9[(int64_t)c * kNDir + lane] = s0 + st.doff[lane];
                }
                __syncwarp();
                ++l;
                continue;
            }
            // a group of consecutive cells staged together: the warp's lanes
            // run over the group's particles in batches of 32 whatever cell
            // they belong to, so short cells do not leave lanes idle
            int gsz = 1, tot = ss[l + 1] - s0;
            while (gsz < kGroupMax && l + gsz < un.cn) {
                const int nn = ss[l + gsz + 1] - ss[l + gsz];
                if (tot + nn > CAP) break;
                tot += nn;
                ++gsz;
            }
            const int s1 = s0 + tot;
            for (int i = lane; i < gsz * kNDir; i += 32) st.run[i] = 0;
            __syncwarp();
            int ci = 0;   // this lane's cell within the group
            // the next batch of the unit (this group's or the next cell's) is
            // loaded while this one is pushed
            for (int b0 = s0; b0 < s1; b0 += 32) {
                const int p = b0 + lane;
                const bool act = p < s1;
                const int q = act ? p : s0;
                while (ci + 1 < gsz && ss[l + ci + 1] <= p) ++ci;
                T fx, fy, ux, uy, uz, w;
                if (pf_pos == b0) {
                    fx = pfx; fy = pfy; ux = pux; uy = puy; uz = puz; w = pw;
                } else {
                    fx = ld(src.fx + q); fy = ld(src.fy + q); ux = ld(src.ux + q);
                    uy = ld(src.uy + q); uz = ld(src.uz + q); w = ld(src.w + q);
                }
                pf_pos = b0 + 32 < s1 ? b0 + 32 : s1;
                if (pf_pos < P1) {
                    const int pq = pf_pos + lane < P1 ? pf_pos + lane : P1 - 1;
                    pfx = ld(src.fx + pq);
                    pfy = ld(src.fy + pq);
                    pux = ld(src.ux + pq);
                    puy = ld(src.uy + pq);
                    puz = ld(src.uz + pq);
                    pw = ld(src.w + pq);
                }
                Pushed<T> o;
                // idle lanes carry weight 0: no ledger contribution (and nothing is stored)
                push_particle<T, PRED>(fx, fy, ux, uy, uz, act ? w : T(0), l + ci, tl.E, tl.B, sen[wib].en(),
                                       beta, dt_dx, dt_dy, qdt, m, true, true, acc, o);
                // rank among the group's particles of the same cell and direction, in order
                const unsigned peers = __match_any_sync(0xffffffffu, act ? ci * 16 + o.dir : 1024 + lane);
                const int ridx = ci * kNDir + o.dir;
                const int rank = (act ? st.run[ridx] : 0) + __popc(peers & lt);
                __syncwarp();
                if (act && (peers & lt) == 0) st.run[ridx] += __popc(peers);
                __syncwarp();
                if (act) {
                    const int e = p - s0;
                    st.fx[e] = o.fxn;
                    st.fy[e] = o.fyn;
                    st.ux[e] = o.u1x;
                    st.uy[e] = o.u1y;
                    st.uz[e] = o.u1z;
                    st.w[e] = o.w;
                    if (ids) st.id[e] = src.id[p];
                    st.dir[e] = (uint8_t)o.dir;
                    st.rank[e] = (uint8_t)rank;
                    st.cell[e] = (uint8_t)ci;
                }
            }
            // offsets per (cell, direction) within the group, the inverse
            // permutation, then one coalesced write of the group in cell and
            // direction order
            for (int i = lane; i < gsz; i += 32) {
                int v = ss[l + i] - s0;
#pragma unroll
                for (int d = 0; d < kNDir; ++d) {
                    st.doff[i * (kNDir + 1) + d] = v;
                    v += st.run[i * kNDir + d];
                }
                st.doff[i * (kNDir + 1) + kNDir] = v;
            }
            __syncwarp();
            for (int e = lane; e < tot; e += 32)
                st.inv[st.doff[st.cell[e] * (kNDir + 1) + st.dir[e]] + st.rank[e]] = (uint8_t)e;
            __syncwarp();
            for (int qq = lane; qq < tot; qq += 32) {
                const int e = st.inv[qq];
                dst.fx[s0 + qq] = st.fx[e];
                dst.fy[s0 + qq] = st.fy[e];
                dst.ux[s0 + qq] = st.ux[e];
                dst.uy[s0 + qq] = st.uy[e];
                dst.uz[s0 + qq] = st.uz[e];
                dst.w[s0 + qq] = st.w[e];
                if (ids) dst.id[s0 + qq] = st.id[e];
            }
            // the runs of the group's cells: counts and starts per direction
            for (int i = lane; i < gsz * kNDir; i += 32) {
                const int gi = i / kNDir, d = i - gi * kNDir;
                const int64_t c = un.c0 + l + gi;
                n9[c * kNDir + d] = st.run[i];
                off9[c * kNDir + d] = s0 + st.doff[gi * (kNDir + 1) + d];
            }
            __syncwarp();
            l += gsz;
        }
        if constexpr (BATCH) ledger_to_instance<T>(acc, led, lane);
    }
    if constexpr (!BATCH) block_ledger<T>(acc, red, lsum);
}

template <typename T, bool PRED>
__global__ void __launch_bounds__(PushCfg<T>::threads, PushCfg<T>::min_blocks)
k_push_sort(PArrays<T> src, PArrays<T> dst, const int32_t* __restrict__ start, int32_t* __restrict__ n9,
            int32_t* __restrict__ off9, const T* __restrict__ Eth, const T* __restrict__ B,
            const T* __restrict__ En, GridP g, T beta, T dt_dx, T dt_dy, T qdt, T m, double* __restrict__ lsum)
{
    push_sort_core<T, PRED, false>(src, dst, start, n9, off9, Eth, B, En, g, beta, dt_dx, dt_dy, qdt, m, lsum,
                                   nullptr, 0, 0);
}

// the push of one species over the units of several instances in one launch
template <typename T, bool PRED>
__global__ void __launch_bounds__(PushCfg<T>::threads, PushCfg<T>::min_blocks)
k_push_sort_batch(const PushDesc<T>* __restrict__ descs, int ninst, int total_units)
{
    PArrays<T> none;
    memset(&none, 0, sizeof(none));
    push_sort_core<T, PRED, true>(none, none, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, GridP{}, T(0),
                                  T(0), T(0), T(0), T(0), nullptr, descs, ninst, total_units);
}

// General path (moves of more than one cell): push in place order, write the
// pushed particle to the same index of dst and its new cell to key.
template <typename T, bool PRED>
__global__ void __launch_bounds__(PushCfg<T>::threads, PushCfg<T>::min_blocks)
k_push_general(PArrays<T> src, PArrays<T> dst, const int32_t* __restrict__ start, int32_t* __restrict__ key,
               const T* __restrict__ Eth, const T* __restrict__ B, const T* __restrict__ En, GridP g, T beta,
               T dt_dx, T dt_dy, T qdt, T m, double* __restrict__ lsum)
{
    constexpr int W = PushCfg<T>::warps;
    __shared__ int sstart[W][kUnitW + 1];
    __shared__ PushTile<T> stile[W];
    __shared__ PredTile<T, PRED> sen[W];
    __shared__ double red[32 * kLedger];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nwarps = (gridDim.x * blockDim.x) >> 5;
    const int nx = g.nx, ny = g.ny, nc = g.ncell;
    const int nunits = units_of(nx, ny);
    int* ss = sstart[wib];
    PushTile<T>& tl = stile[wib];
    T acc[kLedger] = {T(0), T(0), T(0), T(0)};
    for (int u = warp; u < nunits; u += nwarps) {
        const Unit un = unit_of(u, nx);
        unit_setup<T>(un, start, ss, tl, Eth, B, nx, ny, nc, lane);
        if constexpr (PRED) {
            load_tile_E<T, 32>(sen[wib].En, En, un, nx, ny, nc, lane);
            __syncwarp();
        }
        const int P0 = ss[0], P1 = ss[un.cn];
        int cl = 0;   // the lane's current local cell (particles ascend)
        for (int p = P0 + lane; p < P1; p += 32) {
            while (ss[cl + 1] <= p) ++cl;
            Pushed<T> o;
            push_particle<T, PRED>(ld(src.fx + p), ld(src.fy + p), ld(src.ux + p), ld(src.uy + p),
                                   ld(src.uz + p), ld(src.w + p), cl, tl.E, tl.B, sen[wib].en(), beta, dt_dx, dt_dy,
                                   qdt, m, false, true, acc, o);
            int ni = (un.i0 + cl + o.sx) % nx, nj = (un.j + o.sy) % ny;
            if (ni < 0) ni += nx;
            if (nj < 0) nj += ny;
            dst.fx[p] = o.fxn;
            dst.fy[p] = o.fyn;
            dst.ux[p] = o.u1x;
            dst.uy[p] = o.u1y;
            dst.uz[p] = o.u1z;
            dst.w[p] = o.w;
            if (dst.id) dst.id[p] = src.id[p];
            key[p] = nj * nx + ni;
        }
        __syncwarp();
    }
    block_ledger<T>(acc, red, lsum);
}

// The new cell order: warp per unit of new cells. New cell k (its particles at
// [start_new[k], start_new[k+1])) is the concatenation of the nine runs
// (old cell k - o_d, direction d) in ascending order of the old cell index.
// Lane l sets up the runs of the unit's cell l (sorted, with prefix sums);
// then the lanes walk the unit's whole new range, 32 consecutive particles at
// a time, each finding its cell and run. A cell whose runs do not add up to
// its new count flags err.
template <typename T, bool BATCH>
__device__ __forceinline__ void permute_core(PArrays<T> src, PArrays<T> dst, const int32_t* __restrict__ start_new,
                                             const int32_t* __restrict__ n9, const int32_t* __restrict__ off9,
                                             GridP g, int* __restrict__ err, const PushDesc<T>* __restrict__ descs,
                                             int ninst, int total_units)
{
    __shared__ int scs[8][kUnitW + 1];          // new cell starts of the unit
    __shared__ int srs[8][kUnitW][kNDir];       // run start in src, in run order
    __shared__ int srp[8][kUnitW][kNDir + 1];   // run prefix within the cell
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nwarps = (gridDim.x * blockDim.x) >> 5;
    int nx = g.nx, ny = g.ny;
    const int nunits = BATCH ? total_units : units_of(nx, ny);
    bool ids = dst.id != nullptr;
    int* cs = scs[wib];
    for (int ug = warp; ug < nunits; ug += nwarps) {
        int u = ug;
        if constexpr (BATCH) {
            // the re-sort reads the push's output (dst of the push) and
            // writes the new order back into the push's input
            const PushDesc<T>& d = descs[find_inst(descs, ninst, ug)];
            src = d.dst;
            dst = d.src;
            start_new = d.start_new;
            n9 = d.n9;
            off9 = d.off9;
            err = d.err;
            nx = d.g.nx;
            ny = d.g.ny;
            ids = dst.id != nullptr;
            u = ug - d.unit0;
        }
        const Unit un = unit_of(u, nx);
        const int cn = un.cn;
#pragma unroll
        for (int k0 = 0; k0 <= kUnitW; k0 += 32)
            if (k0 + lane <= cn) cs[k0 + lane] = start_new[un.c0 + k0 + lane];
        if (lane < cn) {
            const int i = un.i0 + lane, j = un.j;
            int sc[kNDir], cnt[kNDir], st0[kNDir];
#pragma unroll
            for (int d = 0; d < kNDir; ++d) {
                const int sx = d % 3 - 1, sy = d / 3 - 1;
                sc[d] = wrap1(j - sy, ny) * nx + wrap1(i - sx, nx);
                cnt[d] = n9[(int64_t)sc[d] * kNDir + d];
                st0[d] = off9[(int64_t)sc[d] * kNDir + d];
            }
            int* rp = srp[wib][lane];
            int tot = 0;
#pragma unroll
            for (int d = 0; d < kNDir; ++d) {
                int r = 0;   // rank of the run among the nine (old cells are distinct)
#pragma unroll
                for (int e = 0; e < kNDir; ++e) r += sc[e] < sc[d] ? 1 : 0;
                srs[wib][lane][r] = st0[d];
                rp[r + 1] = cnt[d];
                tot += cnt[d];
            }
            rp[0] = 0;
#pragma unroll
            for (int r = 0; r < kNDir; ++r) rp[r + 1] += rp[r];
            if (tot != start_new[un.c0 + lane + 1] - start_new[un.c0 + lane]) atomicOr(err, 1);
        }
        __syncwarp();
        const int q0 = cs[0], q1 = cs[cn];
        constexpr int U = 4;   // positions per lane in flight
        int l = 0;             // the lane's current cell (positions ascend)
        for (int qb = q0 + lane; qb < q1; qb += 32 * U) {
            int sp[U], qd[U];
#pragma unroll
            for (int v = 0; v < U; ++v) {
                const int q = qb + 32 * v;
                qd[v] = -1;
                sp[v] = 0;
                if (q < q1) {
                    while (l + 1 < cn && cs[l + 1] <= q) ++l;
                    const int e = q - cs[l];
                    const int* rp = srp[wib][l];
                    int r = 0;
#pragma unroll
                    for (int t = 1; t < kNDir; ++t) r += rp[t] <= e ? 1 : 0;
                    if (e < rp[kNDir]) {   // else inconsistent counts (flagged above)
                        sp[v] = srs[wib][l][r] + (e - rp[r]);
                        qd[v] = q;
                    }
                }
            }
            T a[U][6];
            int32_t idv[U];
#pragma unroll
            for (int v = 0; v < U; ++v) {
                const int p = sp[v];
                a[v][0] = ld(src.fx + p);
                a[v][1] = ld(src.fy + p);
                a[v][2] = ld(src.ux + p);
                a[v][3] = ld(src.uy + p);
                a[v][4] = ld(src.uz + p);
                a[v][5] = ld(src.w + p);
                idv[v] = ids ? src.id[p] : 0;
            }
#pragma unroll
            for (int v = 0; v < U; ++v) {
                const int q = qd[v];
                if (q < 0) continue;
                dst.fx[q] = a[v][0];
                dst.fy[q] = a[v][1];
                dst.ux[q] = a[v][2];
                dst.uy[q] = a[v][3];
                dst.uz[q] = a[v][4];
                dst.w[q] = a[v][5];
                if (ids) dst.id[q] = idv[v];
            }
        }
        __syncwarp();
    }
}

template <typename T>
__global__ void __launch_bounds__(256)
k_permute(PArrays<T> src, PArrays<T> dst, const int32_t* __restrict__ start_new, const int32_t* __restrict__ n9,
          const int32_t* __restrict__ off9, GridP g, int* __restrict__ err)
{
    permute_core<T, false>(src, dst, start_new, n9, off9, g, err, nullptr, 0, 0);
}

// the re-sort of one species over the units of several instances
template <typename T>
__global__ void __launch_bounds__(256)
k_permute_batch(const PushDesc<T>* __restrict__ descs, int ninst, int total_units)
{
    PArrays<T> none;
    memset(&none, 0, sizeof(none));
    permute_core<T, true>(none, none, nullptr, nullptr, nullptr, GridP{}, nullptr, descs, ninst, total_units);
}

template <typename T>
__global__ void k_kinetic(PArrays<T> pa, int64_t n, T m, double* partial)
{
    __shared__ double red[32];
    T acc = T(0);
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n;
         p += (int64_t)gridDim.x * blockDim.x) {
        const T ux = pa.ux[p], uy = pa.uy[p], uz = pa.uz[p];
        const T u2 = ux * ux + uy * uy + uz * uz;
        acc += pa.w[p] * m * (u2 / (sqrt(T(1) + u2) + T(1)));
    }
    double v[1] = {(double)acc}, out[1];
    block_sum<1>(v, red, out);
    if (threadIdx.x == 0) partial[blockIdx.x] = out[0];
}

// The particle spectrum: every particle adds its weight (and 1 to the count)
// to the bin of x = gamma - 1 (variable 0) or x = |u| (variable 1) among the
// ascending edges e_0 < .. < e_nbins: bin 0 below e_0, bin b for
// e_{b-1} <= x < e_b, bin nbins+1 at or above e_nbins. x is formed with
// round-to-nearest operations and no contraction, in T; the edges arrive
// rounded up to T, so the comparisons equal those against the FP64 edges.
// Per block the bins live in shared memory; one atomic flush per bin.
__device__ __forceinline__ float mul_rn(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double mul_rn(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float add_rn(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ double add_rn(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ float div_rn(float a, float b) { return __fdiv_rn(a, b); }
__device__ __forceinline__ double div_rn(double a, double b) { return __ddiv_rn(a, b); }
__device__ __forceinline__ float sqrt_rn(float a) { return __fsqrt_rn(a); }
__device__ __forceinline__ double sqrt_rn(double a) { return __dsqrt_rn(a); }

template <typename T>
__global__ void __launch_bounds__(256)
k_spectrum(PArrays<T> pa, int64_t n, int variable, const T* __restrict__ edges, int nbins,
           double* __restrict__ wsum, unsigned long long* __restrict__ cnt)
{
    extern __shared__ __align__(16) unsigned char ssm[];
    const int nb = nbins + 2;
    double* sw = reinterpret_cast<double*>(ssm);
    unsigned* sc = reinterpret_cast<unsigned*>(sw + nb);
    T* se = reinterpret_cast<T*>(sw + 2 * nb);   // past both bin arrays, 8-byte aligned
    for (int b = threadIdx.x; b < nb; b += blockDim.x) {
        sw[b] = 0.0;
        sc[b] = 0u;
    }
    for (int b = threadIdx.x; b <= nbins; b += blockDim.x) se[b] = edges[b];
    __syncthreads();
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x) {
        const T ux = pa.ux[p], uy = pa.uy[p], uz = pa.uz[p];
        const T u2 = add_rn(add_rn(mul_rn(ux, ux), mul_rn(uy, uy)), mul_rn(uz, uz));
        const T x = variable == 0 ? div_rn(u2, add_rn(sqrt_rn(add_rn(T(1), u2)), T(1))) : sqrt_rn(u2);
        int a = 0, b = nbins + 1;   // the number of edges <= x
        while (a < b) {
            const int mid = (a + b) >> 1;
            if (se[mid] <= x) a = mid + 1;
            else b = mid;
        }
        atomicAdd(&sw[a], (double)pa.w[p]);
        atomicAdd(&sc[a], 1u);
    }
    __syncthreads();
    for (int b = threadIdx.x; b < nb; b += blockDim.x)
        if (sc[b]) {
            atomicAdd(&wsum[b], sw[b]);
            atomicAdd(&cnt[b], (unsigned long long)sc[b]);
        }
}

int blocks_for(int64_t n, int threads, int cap)
{
    int64_t b = (n + threads - 1) / threads;
    if (b < 1) b = 1;
    if (b > cap) b = cap;
    return (int)b;
}

}  // namespace

// ---------------------------------------------------------------------------
// the adjoints of the push and the deposit (they reuse the unit tiles above)
namespace {

// Segmented sums across a warp for the adjoints' scatters. In one pass of a
// unit the lanes hold consecutive particles, so their cells ascend and the
// lanes of one cell are consecutive: a suffix sum over those runs (five
// shuffle steps) leaves each run's total in its first lane, which alone
// issues the FP64 atomics. This replaces one global atomic per lane and
// target by one per cell and target.
struct Runs {
    unsigned same;   // bit s: lane + 2^s < 32 holds the same key
    bool head;       // first lane of its run
};

__device__ __forceinline__ Runs runs_of(int key, int lane)
{
    Runs r;
    r.same = 0u;
#pragma unroll
    for (int s = 0; s < 5; ++s) {
        const int d = 1 << s;
        const int ko = __shfl_down_sync(0xffffffffu, key, d);
        if (lane + d < 32 && ko == key) r.same |= 1u << s;
    }
    const int kp = __shfl_up_sync(0xffffffffu, key, 1);
    r.head = lane == 0 || kp != key;
    return r;
}

template <typename A>
__device__ __forceinline__ A run_sum(A v, const Runs& r)
{
#pragma unroll
    for (int s = 0; s < 5; ++s) {
        const A o = __shfl_down_sync(0xffffffffu, v, 1 << s);
        if ((r.same >> s) & 1u) v += o;
    }
    return v;
}

// The 3x3 cell centres around cell (i, j) (tile rows j-1..j+1, columns
// i-1..i+1): a particle's four centre weights Wc as separable factors
// Ry[r] Cx[c], zero outside its 2x2 (rows 0-1 when fy < 1/2, else 1-2;
// likewise the columns).
template <typename A>
__device__ __forceinline__ void centre_factors(bool lx, bool ly, A tx, A ty, A (&Cx)[3], A (&Ry)[3])
{
    Cx[0] = lx ? A(1) - tx : A(0);
    Cx[1] = lx ? tx : A(1) - tx;
    Cx[2] = lx ? A(0) : tx;
    Ry[0] = ly ? A(1) - ty : A(0);
    Ry[1] = ly ? ty : A(1) - ty;
    Ry[2] = ly ? A(0) : ty;
}

// the run totals of a 3x3 centre scatter (3 components) added to gB
template <typename A>
__device__ __forceinline__ void flush_centres(const A (&gc)[3][3][3], const Runs& rn, bool act, double* gB, int i,
                                              int j, int nx, int ny, int nc)
{
#pragma unroll
    for (int r = 0; r < 3; ++r) {
        const int gj = wrap1(j - 1 + r, ny);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const int64_t cell = (int64_t)gj * nx + wrap1(i - 1 + c, nx);
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                const A s = run_sum(gc[k][r][c], rn);
                if (rn.head && act) atomicAdd(gB + (int64_t)k * nc + cell, (double)s);
            }
        }
    }
}

// Adjoint of the push with the fields held fixed (base scheme, gbar =
// gamma(u^n)): per particle, the push is replayed from the stored values in
// the form's precision (FP32 for the FP32 form: GB300's FP64 rate is a
// small fraction of its FP32 rate) and the chain rule run in reverse. The
// gathers' transposes are scatters with the same weights into gE on the
// nodes and gB on the centres, summed per cell across the warp and added
// with FP64 atomics; alpha's transpose is applied to the gradient of ubar,
// and d alpha = -alpha d[a]x alpha gives the gradient of a = beta B/gbar.
// gu1, gx1 are dL/du^{n+1}, dL/dx^{n+3/2} (FP64, interleaved, in the
// particles' current order); gu0, gx0 receive dL/du^n, dL/dx^{n+1/2}.
template <typename T, bool PRED>
__global__ void __launch_bounds__(PushCfg<T>::threads, sizeof(T) == 4 ? 4 : 1)
k_push_adjoint(PArrays<T> src, const int32_t* __restrict__ start, const double* __restrict__ gu1,
               const double* __restrict__ gx1, double* __restrict__ gu0, double* __restrict__ gx0,
               double* __restrict__ gE, double* __restrict__ gB, const T* __restrict__ Eth,
               const T* __restrict__ B, GridP g, double beta_d, const T* __restrict__ Eold,
               double* __restrict__ gEold)
{
    using A = T;
    constexpr int W = PushCfg<T>::warps;
    __shared__ int sstart[W][kUnitW + 1];
    __shared__ PushTile<T> stile[W];
    __shared__ PredTile<T, PRED> sen[W];   // E^n of the predicted gbar
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nwarps = (gridDim.x * blockDim.x) >> 5;
    const int nx = g.nx, ny = g.ny, nc = g.ncell;
    const int nunits = units_of(nx, ny);
    int* ss = sstart[wib];
    PushTile<T>& tl = stile[wib];
    const A rdx = A(1.0 / g.dx), rdy = A(1.0 / g.dy), dt = A(g.dt), beta = A(beta_d);
    for (int u = warp; u < nunits; u += nwarps) {
        const Unit un = unit_of(u, nx);
        unit_setup<T>(un, start, ss, tl, Eth, B, nx, ny, nc, lane);
        if constexpr (PRED) {
            load_tile_E<T, 32>(sen[wib].En, Eold, un, nx, ny, nc, lane);
            __syncwarp();
        }
        const int P0 = ss[0], P1 = ss[un.cn];
        int cl = 0;
        for (int p0 = P0; p0 < P1; p0 += 32) {
            const int p = p0 + lane;
            const bool act = p < P1;
            if (act)
                while (ss[cl + 1] <= p) ++cl;
            A gn[4][3], gc[3][3][3];   // this lane's node and centre scatters
            A go[PRED ? 4 : 1][3];     // and, predicted gbar, its E^n node scatter
#pragma unroll
            for (int q = 0; q < (PRED ? 4 : 1); ++q)
#pragma unroll
                for (int k = 0; k < 3; ++k) go[q][k] = A(0);
#pragma unroll
            for (int q = 0; q < 4; ++q)
#pragma unroll
                for (int k = 0; k < 3; ++k) gn[q][k] = A(0);
#pragma unroll
            for (int k = 0; k < 3; ++k)
#pragma unroll
                for (int r = 0; r < 3; ++r)
#pragma unroll
                    for (int c = 0; c < 3; ++c) gc[k][r][c] = A(0);
            if (act) {
                const A fx = ld(src.fx + p), fy = ld(src.fy + p);
                const A u0[3] = {ld(src.ux + p), ld(src.uy + p), ld(src.uz + p)};
                // node weights and their derivatives in x, y
                const A X0 = A(1) - fx, Y0 = A(1) - fy;
                const A Wn[4] = {X0 * Y0, fx * Y0, X0 * fy, fx * fy};
                const A Wnx[4] = {-Y0 * rdx, Y0 * rdx, -fy * rdx, fy * rdx};
                const A Wny[4] = {-X0 * rdy, -fx * rdy, X0 * rdy, fx * rdy};
                A En[4][3];
#pragma unroll
                for (int k = 0; k < 3; ++k) {
                    En[0][k] = tl.E[k][0][cl];
                    En[1][k] = tl.E[k][0][cl + 1];
                    En[2][k] = tl.E[k][1][cl];
                    En[3][k] = tl.E[k][1][cl + 1];
                }
                // centre weights (the two centres below or above the offset)
                const bool lx = fx < A(0.5), ly = fy < A(0.5);
                const A tx = lx ? fx + A(0.5) : fx - A(0.5), ty = ly ? fy + A(0.5) : fy - A(0.5);
                const int c0 = lx ? cl : cl + 1, r0 = ly ? 0 : 1;
                const A Wc[4] = {(A(1) - tx) * (A(1) - ty), tx * (A(1) - ty), (A(1) - tx) * ty, tx * ty};
                const A Wcx[4] = {-(A(1) - ty) * rdx, (A(1) - ty) * rdx, -ty * rdx, ty * rdx};
                const A Wcy[4] = {-(A(1) - tx) * rdy, -tx * rdy, (A(1) - tx) * rdy, tx * rdy};
                A Bc[4][3];
#pragma unroll
                for (int k = 0; k < 3; ++k) {
                    Bc[0][k] = tl.B[k][r0][c0];
                    Bc[1][k] = tl.B[k][r0][c0 + 1];
                    Bc[2][k] = tl.B[k][r0 + 1][c0];
                    Bc[3][k] = tl.B[k][r0 + 1][c0 + 1];
                }
                A Ep[3], Bp[3];
#pragma unroll
                for (int k = 0; k < 3; ++k) {
                    Ep[k] = Wn[0] * En[0][k] + Wn[1] * En[1][k] + Wn[2] * En[2][k] + Wn[3] * En[3][k];
                    Bp[k] = Wc[0] * Bc[0][k] + Wc[1] * Bc[1][k] + Wc[2] * Bc[2][k] + Wc[3] * Bc[3][k];
                }
                // forward replay; gbar = gamma(s), s = u^n or, predicted,
                // u^n + beta E^n(x)
                A sv[3] = {u0[0], u0[1], u0[2]};
                A Eo[PRED ? 4 : 1][3];
                if constexpr (PRED) {
                    const T (*te)[2][kTE] = sen[wib].en();
#pragma unroll
                    for (int k = 0; k < 3; ++k) {
                        Eo[0][k] = te[k][0][cl];
                        Eo[1][k] = te[k][0][cl + 1];
                        Eo[2][k] = te[k][1][cl];
                        Eo[3][k] = te[k][1][cl + 1];
                        sv[k] += beta * (Wn[0] * Eo[0][k] + Wn[1] * Eo[1][k] + Wn[2] * Eo[2][k] + Wn[3] * Eo[3][k]);
                    }
                }
                const A gb = sqrt(A(1) + sv[0] * sv[0] + sv[1] * sv[1] + sv[2] * sv[2]);
                const A a[3] = {beta * Bp[0] / gb, beta * Bp[1] / gb, beta * Bp[2] / gb};
                const A ia = A(1) / (A(1) + a[0] * a[0] + a[1] * a[1] + a[2] * a[2]);
                // alpha = (I - [a]x + a a^T)/(1 + |a|^2) = (I + [a]x)^{-1}
                A al[3][3];
                al[0][0] = (A(1) + a[0] * a[0]) * ia; al[0][1] = (a[0] * a[1] + a[2]) * ia; al[0][2] = (a[0] * a[2] - a[1]) * ia;
                al[1][0] = (a[0] * a[1] - a[2]) * ia; al[1][1] = (A(1) + a[1] * a[1]) * ia; al[1][2] = (a[1] * a[2] + a[0]) * ia;
                al[2][0] = (a[0] * a[2] + a[1]) * ia; al[2][1] = (a[1] * a[2] - a[0]) * ia; al[2][2] = (A(1) + a[2] * a[2]) * ia;
                A w[3], ub[3], u1[3];
#pragma unroll
                for (int k = 0; k < 3; ++k) w[k] = u0[k] + beta * Ep[k];
#pragma unroll
                for (int r = 0; r < 3; ++r) ub[r] = al[r][0] * w[0] + al[r][1] * w[1] + al[r][2] * w[2];
#pragma unroll
                for (int k = 0; k < 3; ++k) u1[k] = A(2) * ub[k] - u0[k];
                const A g1 = sqrt(A(1) + u1[0] * u1[0] + u1[1] * u1[1] + u1[2] * u1[2]);
                // backward: x1 = x + dt u1/g1
                const A gp[3] = {(A)gx1[2 * (int64_t)p], (A)gx1[2 * (int64_t)p + 1], A(0)};
                const A up = u1[0] * gp[0] + u1[1] * gp[1];
                A gt[3], gub[3], gu[3], gw[3];
#pragma unroll
                for (int k = 0; k < 3; ++k) {
                    gt[k] = (A)gu1[3 * (int64_t)p + k] + dt * (gp[k] / g1 - u1[k] * up / (g1 * g1 * g1));
                    gub[k] = A(2) * gt[k];
                    gu[k] = -gt[k];
                }
#pragma unroll
                for (int k = 0; k < 3; ++k) gw[k] = al[0][k] * gub[0] + al[1][k] * gub[1] + al[2][k] * gub[2];
#pragma unroll
                for (int k = 0; k < 3; ++k) gu[k] += gw[k];
                // G = -alpha^T (gub w^T) alpha^T = -(alpha^T gub)(alpha w)^T = -gw ub^T
                // (the outer product factorises); ga from <G, [da]x>
                const A ga[3] = {-(gw[2] * ub[1] - gw[1] * ub[2]), -(gw[0] * ub[2] - gw[2] * ub[0]),
                                 -(gw[1] * ub[0] - gw[0] * ub[1])};
                const A gBp[3] = {beta * ga[0] / gb, beta * ga[1] / gb, beta * ga[2] / gb};
                const A ggb = -beta * (ga[0] * Bp[0] + ga[1] * Bp[1] + ga[2] * Bp[2]) / (gb * gb);
                // dL/dgbar through gbar = gamma(s): to u^n and, predicted,
                // to E^n at the particle (beta dL/ds)
                A gs[3];
#pragma unroll
                for (int k = 0; k < 3; ++k) {
                    gs[k] = ggb * sv[k] / gb;
                    gu[k] += gs[k];
                }
                const A gEp[3] = {beta * gw[0], beta * gw[1], beta * gw[2]};
                A gxp = gp[0], gyp = gp[1];
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    A eg = A(0), bg = A(0);
#pragma unroll
                    for (int k = 0; k < 3; ++k) {
                        gn[q][k] = Wn[q] * gEp[k];
                        eg += En[q][k] * gEp[k];
                        bg += Bc[q][k] * gBp[k];
                    }
                    if constexpr (PRED) {
#pragma unroll
                        for (int k = 0; k < 3; ++k) {
                            go[q][k] = Wn[q] * beta * gs[k];
                            eg += Eo[q][k] * beta * gs[k];
                        }
                    }
                    gxp += Wnx[q] * eg + Wcx[q] * bg;
                    gyp += Wny[q] * eg + Wcy[q] * bg;
                }
                A Cx[3], Ry[3];
                centre_factors(lx, ly, tx, ty, Cx, Ry);
#pragma unroll
                for (int k = 0; k < 3; ++k)
#pragma unroll
                    for (int r = 0; r < 3; ++r)
#pragma unroll
                        for (int c = 0; c < 3; ++c) gc[k][r][c] = Ry[r] * Cx[c] * gBp[k];
#pragma unroll
                for (int k = 0; k < 3; ++k) gu0[3 * (int64_t)p + k] = (double)gu[k];
                gx0[2 * (int64_t)p] = (double)gxp;
                gx0[2 * (int64_t)p + 1] = (double)gyp;
            }
            // the cell runs' totals: nodes (i, j), (i+1, j), (i, j+1), (i+1, j+1)
            const Runs rn = runs_of(act ? cl : -1, lane);
            const int i = un.i0 + cl, j = un.j;
            const int i1 = wrap1(i + 1, nx), j1 = wrap1(j + 1, ny);
            const int64_t nodes[4] = {(int64_t)j * nx + i, (int64_t)j * nx + i1, (int64_t)j1 * nx + i,
                                      (int64_t)j1 * nx + i1};
#pragma unroll
            for (int q = 0; q < 4; ++q)
#pragma unroll
                for (int k = 0; k < 3; ++k) {
                    const A s = run_sum(gn[q][k], rn);
                    if (rn.head && act) atomicAdd(gE + (int64_t)k * nc + nodes[q], (double)s);
                }
            if constexpr (PRED) {
#pragma unroll
                for (int q = 0; q < 4; ++q)
#pragma unroll
                    for (int k = 0; k < 3; ++k) {
                        const A s = run_sum(go[q][k], rn);
                        if (rn.head && act) atomicAdd(gEold + (int64_t)k * nc + nodes[q], (double)s);
                    }
            }
            flush_centres(gc, rn, act, gB, i, j, nx, ny, nc);
        }
        __syncwarp();
    }
}

// Adjoint of the deposit (base scheme): per particle, alpha, gbar and the
// shape weights are rebuilt from the stored values in the form's precision;
// the gradient of alpha collects the predicted current's (gJ at the cell's
// 4 nodes) and the 10 node pairs' stored mass-matrix block gradients (gM,
// ncell x 45), then flows through a = beta B/gbar to B (summed per cell
// across the warp, FP64 atomics on the centres) and gbar; the weights'
// derivatives give dL/dx. Outputs per particle dL/du^n (gu0, interleaved)
// and dL/dx^{n+1/2} (gx0), FP64.
template <typename T, bool PRED>
__global__ void __launch_bounds__(PushCfg<T>::threads, sizeof(T) == 4 ? 4 : 1)
k_deposit_adjoint(PArrays<T> src, const int32_t* __restrict__ start, const double* __restrict__ gJ,
                  const double* __restrict__ gM, double* __restrict__ gu0, double* __restrict__ gx0,
                  double* __restrict__ gw0, double* __restrict__ gB, const T* __restrict__ B, GridP g, double beta_d,
                  double cq, const T* __restrict__ Eold, double* __restrict__ gEold)
{
    using A = T;
    constexpr int W = PushCfg<T>::warps;
    __shared__ int sstart[W][kUnitW + 1];
    __shared__ PushTile<T> stile[W];
    __shared__ PredTile<T, PRED> sen[W];   // E^n of the predicted gbar
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nwarps = (gridDim.x * blockDim.x) >> 5;
    const int nx = g.nx, ny = g.ny, nc = g.ncell;
    const int nunits = units_of(nx, ny);
    int* ss = sstart[wib];
    PushTile<T>& tl = stile[wib];
    const A rdx = A(1.0 / g.dx), rdy = A(1.0 / g.dy), beta = A(beta_d);
    const A cJ0 = A(cq / g.dV), cM0 = A(cq * beta_d / g.dV);
    // the cell's node pairs: (node a, node b, storing node, half offset)
    constexpr int pa[10] = {0, 0, 0, 0, 1, 1, 1, 2, 2, 3};
    constexpr int pb[10] = {0, 1, 2, 3, 1, 2, 3, 2, 3, 3};
    constexpr int ps[10] = {0, 0, 0, 0, 1, 1, 1, 2, 2, 3};
    constexpr int po[10] = {0, 1, 3, 4, 0, 2, 3, 0, 1, 0};
    for (int u = warp; u < nunits; u += nwarps) {
        const Unit un = unit_of(u, nx);
        unit_setup<T>(un, start, ss, tl, B, B, nx, ny, nc, lane);
        if constexpr (PRED) {
            load_tile_E<T, 32>(sen[wib].En, Eold, un, nx, ny, nc, lane);
            __syncwarp();
        }
        const int P0 = ss[0], P1 = ss[un.cn];
        int cl = 0;
        for (int p0 = P0; p0 < P1; p0 += 32) {
            const int p = p0 + lane;
            const bool act = p < P1;
            if (act)
                while (ss[cl + 1] <= p) ++cl;
            const int i = un.i0 + cl, j = un.j;
            A go[PRED ? 4 : 1][3];   // predicted gbar: this lane's E^n node scatter
#pragma unroll
            for (int q = 0; q < (PRED ? 4 : 1); ++q)
#pragma unroll
                for (int k = 0; k < 3; ++k) go[q][k] = A(0);
            A gc[3][3][3];
#pragma unroll
            for (int k = 0; k < 3; ++k)
#pragma unroll
                for (int r = 0; r < 3; ++r)
#pragma unroll
                    for (int c = 0; c < 3; ++c) gc[k][r][c] = A(0);
            if (act) {
                const A fx = ld(src.fx + p), fy = ld(src.fy + p);
                const A u0[3] = {ld(src.ux + p), ld(src.uy + p), ld(src.uz + p)};
                const A wt = ld(src.w + p);
                const A X0 = A(1) - fx, Y0 = A(1) - fy;
                const A Wn[4] = {X0 * Y0, fx * Y0, X0 * fy, fx * fy};
                const A Wnx[4] = {-Y0 * rdx, Y0 * rdx, -fy * rdx, fy * rdx};
                const A Wny[4] = {-X0 * rdy, -fx * rdy, X0 * rdy, fx * rdy};
                const bool lx = fx < A(0.5), ly = fy < A(0.5);
                const A tx = lx ? fx + A(0.5) : fx - A(0.5), ty = ly ? fy + A(0.5) : fy - A(0.5);
                const int c0 = lx ? cl : cl + 1, r0 = ly ? 0 : 1;
                const A Wc[4] = {(A(1) - tx) * (A(1) - ty), tx * (A(1) - ty), (A(1) - tx) * ty, tx * ty};
                const A Wcx[4] = {-(A(1) - ty) * rdx, (A(1) - ty) * rdx, -ty * rdx, ty * rdx};
                const A Wcy[4] = {-(A(1) - tx) * rdy, -tx * rdy, (A(1) - tx) * rdy, tx * rdy};
                A Bc[4][3];
#pragma unroll
                for (int k = 0; k < 3; ++k) {
                    Bc[0][k] = tl.B[k][r0][c0];
                    Bc[1][k] = tl.B[k][r0][c0 + 1];
                    Bc[2][k] = tl.B[k][r0 + 1][c0];
                    Bc[3][k] = tl.B[k][r0 + 1][c0 + 1];
                }
                A Bp[3];
#pragma unroll
                for (int k = 0; k < 3; ++k)
                    Bp[k] = Wc[0] * Bc[0][k] + Wc[1] * Bc[1][k] + Wc[2] * Bc[2][k] + Wc[3] * Bc[3][k];
                // gbar = gamma(s), s = u^n or, predicted, u^n + beta E^n(x)
                A sv[3] = {u0[0], u0[1], u0[2]};
                A Eo[PRED ? 4 : 1][3];
                if constexpr (PRED) {
                    const T (*te)[2][kTE] = sen[wib].en();
#pragma unroll
                    for (int k = 0; k < 3; ++k) {
                        Eo[0][k] = te[k][0][cl];
                        Eo[1][k] = te[k][0][cl + 1];
                        Eo[2][k] = te[k][1][cl];
                        Eo[3][k] = te[k][1][cl + 1];
                        sv[k] += beta * (Wn[0] * Eo[0][k] + Wn[1] * Eo[1][k] + Wn[2] * Eo[2][k] + Wn[3] * Eo[3][k]);
                    }
                }
                const A gb = sqrt(A(1) + sv[0] * sv[0] + sv[1] * sv[1] + sv[2] * sv[2]);
                const A a[3] = {beta * Bp[0] / gb, beta * Bp[1] / gb, beta * Bp[2] / gb};
                const A ia = A(1) / (A(1) + a[0] * a[0] + a[1] * a[1] + a[2] * a[2]);
                A al[3][3];
                al[0][0] = (A(1) + a[0] * a[0]) * ia; al[0][1] = (a[0] * a[1] + a[2]) * ia; al[0][2] = (a[0] * a[2] - a[1]) * ia;
                al[1][0] = (a[0] * a[1] - a[2]) * ia; al[1][1] = (A(1) + a[1] * a[1]) * ia; al[1][2] = (a[1] * a[2] + a[0]) * ia;
                al[2][0] = (a[0] * a[2] + a[1]) * ia; al[2][1] = (a[1] * a[2] - a[0]) * ia; al[2][2] = (A(1) + a[2] * a[2]) * ia;
                A au[3];
#pragma unroll
                for (int r = 0; r < 3; ++r) au[r] = al[r][0] * u0[0] + al[r][1] * u0[1] + al[r][2] * u0[2];
                const A rgb = A(1) / gb;
                const A cJ = wt * cJ0 * rgb, cM = wt * cM0 * rgb;   // with the 1/gbar of both terms
                const int i1 = wrap1(i + 1, nx), j1 = wrap1(j + 1, ny);
                const int64_t nodes[4] = {(int64_t)j * nx + i, (int64_t)j * nx + i1, (int64_t)j1 * nx + i,
                                          (int64_t)j1 * nx + i1};
                A ga_[3][3] = {{A(0), A(0), A(0)}, {A(0), A(0), A(0)}, {A(0), A(0), A(0)}};   // dL/dalpha
                A gW[4] = {A(0), A(0), A(0), A(0)}, gu[3] = {A(0), A(0), A(0)};
                A sg = A(0);   // sum of the terms' values: d/dgbar of each is -value/gbar
                A sJw = A(0), sMw = A(0);   // the same sums per unit weight (J and M are linear in w)
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    const A gj[3] = {(A)gJ[nodes[k]], (A)gJ[nc + nodes[k]], (A)gJ[2 * (int64_t)nc + nodes[k]]};
                    const A f = cJ * Wn[k];
                    A sJ = A(0);
#pragma unroll
                    for (int r = 0; r < 3; ++r) {
                        sJ += gj[r] * au[r];
#pragma unroll
                        for (int q = 0; q < 3; ++q) {
                            ga_[r][q] += f * gj[r] * u0[q];
                            gu[q] += f * al[r][q] * gj[r];
                        }
                    }
                    gW[k] += cJ * sJ;
                    sg += cJ * Wn[k] * sJ;
                    sJw += Wn[k] * sJ;
                }
#pragma unroll
                for (int pr = 0; pr < 10; ++pr) {
                    const double* G = gM + nodes[ps[pr]] * kMBlock + po[pr] * 9;
                    A Gv[9];
#pragma unroll
                    for (int e = 0; e < 9; ++e) Gv[e] = (A)G[e];
                    A s2 = A(0);
#pragma unroll
                    for (int r = 0; r < 3; ++r)
#pragma unroll
                        for (int q = 0; q < 3; ++q) s2 += Gv[r * 3 + q] * al[r][q];
                    const A wa = Wn[pa[pr]], wb = Wn[pb[pr]];
                    const A coef = cM * wa * wb;
#pragma unroll
                    for (int r = 0; r < 3; ++r)
#pragma unroll
                        for (int q = 0; q < 3; ++q) ga_[r][q] += coef * Gv[r * 3 + q];
                    gW[pa[pr]] += cM * wb * s2;
                    gW[pb[pr]] += cM * wa * s2;
                    sg += coef * s2;
                    sMw += wa * wb * s2;
                }
                A ggb = -sg * rgb;
                // Gm = -alpha^T ga_ alpha^T; gradient of a from <Gm, [da]x>
                A t1[3][3], Gm[3][3];
#pragma unroll
                for (int r = 0; r < 3; ++r)
#pragma unroll
                    for (int q = 0; q < 3; ++q)
                        t1[r][q] = al[0][r] * ga_[0][q] + al[1][r] * ga_[1][q] + al[2][r] * ga_[2][q];
#pragma unroll
                for (int r = 0; r < 3; ++r)
#pragma unroll
                    for (int q = 0; q < 3; ++q)
                        Gm[r][q] = -(t1[r][0] * al[q][0] + t1[r][1] * al[q][1] + t1[r][2] * al[q][2]);
                const A gav[3] = {Gm[2][1] - Gm[1][2], Gm[0][2] - Gm[2][0], Gm[1][0] - Gm[0][1]};
                const A gBp[3] = {beta * gav[0] * rgb, beta * gav[1] * rgb, beta * gav[2] * rgb};
                ggb -= (gav[0] * a[0] + gav[1] * a[1] + gav[2] * a[2]) * rgb;
                // dL/dgbar through gbar = gamma(s): to u^n and, predicted,
                // to E^n at the particle (beta dL/ds)
                A gs[3];
#pragma unroll
                for (int k = 0; k < 3; ++k) {
                    gs[k] = ggb * sv[k] * rgb;
                    gu[k] += gs[k];
                }
                A gxp = A(0), gyp = A(0);
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    A bg = A(0), eo = A(0);
#pragma unroll
                    for (int k = 0; k < 3; ++k) bg += Bc[q][k] * gBp[k];
                    if constexpr (PRED) {
#pragma unroll
                        for (int k = 0; k < 3; ++k) {
                            go[q][k] = Wn[q] * beta * gs[k];
                            eo += Eo[q][k] * beta * gs[k];
                        }
                    }
                    gxp += Wnx[q] * (gW[q] + eo) + Wcx[q] * bg;
                    gyp += Wny[q] * (gW[q] + eo) + Wcy[q] * bg;
                }
                A Cx[3], Ry[3];
                centre_factors(lx, ly, tx, ty, Cx, Ry);
#pragma unroll
                for (int k = 0; k < 3; ++k)
#pragma unroll
                    for (int r = 0; r < 3; ++r)
#pragma unroll
                        for (int c = 0; c < 3; ++c) gc[k][r][c] = Ry[r] * Cx[c] * gBp[k];
#pragma unroll
                for (int k = 0; k < 3; ++k) gu0[3 * (int64_t)p + k] = (double)gu[k];
                gx0[2 * (int64_t)p] = (double)gxp;
                gx0[2 * (int64_t)p + 1] = (double)gyp;
                if (gw0) gw0[p] = (double)((cJ0 * sJw + cM0 * sMw) * rgb);
            }
            const Runs rn = runs_of(act ? cl : -1, lane);
            flush_centres(gc, rn, act, gB, i, j, nx, ny, nc);
            if constexpr (PRED) {
                const int i1 = wrap1(i + 1, nx), j1 = wrap1(j + 1, ny);
                const int64_t nodes[4] = {(int64_t)j * nx + i, (int64_t)j * nx + i1, (int64_t)j1 * nx + i,
                                          (int64_t)j1 * nx + i1};
#pragma unroll
                for (int q = 0; q < 4; ++q)
#pragma unroll
                    for (int k = 0; k < 3; ++k) {
                        const A sq = run_sum(go[q][k], rn);
                        if (rn.head && act) atomicAdd(gEold + (int64_t)k * nc + nodes[q], (double)sq);
                    }
            }
        }
        __syncwarp();
    }
}

}  // namespace (the adjoints)

int row_units(GridP g) { return units_of(g.nx, g.ny); }

int push_grid_blocks(GridP g, int precision, int cap)
{
    return blocks_for(units_of(g.nx, g.ny), precision == 32 ? PushCfg<float>::warps : PushCfg<double>::warps,
                      cap > 0 ? cap : 152 * 16);
}

template <typename T>
cudaError_t load_convert(const double* x, const double* u, const double* w, int64_t n, GridP g,
                         PArrays<T> out, int32_t* key, int32_t* val, int* bad, cudaStream_t st)
{
    if (n <= 0) return cudaSuccess;
    count_launches(1);
    k_load_convert<T><<<blocks_for(n, 256, 152 * 32), 256, 0, st>>>(x, u, w, n, g, out, key, val, bad);
    return cudaGetLastError();
}

cudaError_t keys_unsorted(const int32_t* keys, int64_t n, int* flag, cudaStream_t st)
{
    if (n <= 1) return cudaSuccess;
    count_launches(1);
    k_keys_unsorted<<<blocks_for(n, 256, 152 * 8), 256, 0, st>>>(keys, n, flag);
    return cudaGetLastError();
}

template <typename T>
cudaError_t gather_particles(const int32_t* perm, PArrays<T> src, PArrays<T> dst, int64_t n,
                             bool ids_from_perm, cudaStream_t st)
{
    if (n <= 0) return cudaSuccess;
    count_launches(1);
    k_gather<T><<<blocks_for(n, 256, 152 * 32), 256, 0, st>>>(perm, src, dst, n, ids_from_perm);
    return cudaGetLastError();
}

template <typename T>
cudaError_t export_particles(PArrays<T> p, const int32_t* start, GridP g, double* x, double* u,
                             double* w, int32_t* id, cudaStream_t st)
{
    count_launches(1);
    k_export<T><<<blocks_for((int64_t)g.ncell * 32, 256, 152 * 16), 256, 0, st>>>(p, start, g, x, u, w, id);
    return cudaGetLastError();
}

template <typename T>
cudaError_t deposit(const DepositSpecies<T>& sp, const T* B, const T* En, T* M, T* J, GridP g, int* err,
                    cudaStream_t st, int max_blocks)
{
    const int nunits = units_of(g.nx, g.ny);
    int dev = 0, nsm = 152;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    nsm *= 2;   // two CTAs per SM
    if (max_blocks > 0) nsm = max_blocks;
    const size_t smem = (size_t)kDepBuf * 6 * kDepCap * sizeof(T);
    auto kern = En ? k_deposit<T, true> : k_deposit<T, false>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const int blocks = nunits < nsm ? nunits : nsm;
    count_launches(1);
    kern<<<blocks, kDepThreads, smem, st>>>(sp, B, En, M, J, g, err);
    return cudaGetLastError();
}

template <typename T>
cudaError_t push_sort(PArrays<T> src, PArrays<T> dst, const int32_t* start, int32_t* n9, int32_t* off9,
                      const T* Eth, const T* B, const T* En, GridP g, SpeciesConst sc, double* lsum_partial,
                      int lsum_blocks, int* err, cudaStream_t st)
{
    (void)err;   // the push has no bounded wait to report
    const T beta = (T)(sc.q * g.dt / (2.0 * sc.m));
    auto kern = En ? k_push_sort<T, true> : k_push_sort<T, false>;
    count_launches(1);
    kern<<<lsum_blocks, PushCfg<T>::threads, 0, st>>>(src, dst, start, n9, off9, Eth, B, En, g, beta,
                                                      (T)(g.dt / g.dx), (T)(g.dt / g.dy), (T)(sc.q * g.dt),
                                                      (T)sc.m, lsum_partial);
    return cudaGetLastError();
}

// shared launches over the instances of a batch (units numbered across them)
template <typename T>
cudaError_t deposit_batch(const DepDesc<T>* descs, int ninst, int total_units, bool pred, int* err, cudaStream_t st,
                          int blocks)
{
    const size_t smem = (size_t)kDepBuf * 6 * kDepCap * sizeof(T);
    auto kern = pred ? k_deposit_batch<T, true> : k_deposit_batch<T, false>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    if (blocks > total_units) blocks = total_units;
    if (blocks < 1) blocks = 1;
    count_launches(1);
    kern<<<blocks, kDepThreads, smem, st>>>(descs, ninst, total_units, err);
    return cudaGetLastError();
}

template <typename T>
cudaError_t push_sort_batch(const PushDesc<T>* descs, int ninst, int total_units, bool pred, int blocks,
                            cudaStream_t st)
{
    auto kern = pred ? k_push_sort_batch<T, true> : k_push_sort_batch<T, false>;
    const int need = blocks_for(total_units, PushCfg<T>::warps, blocks > 0 ? blocks : 152 * 16);
    count_launches(1);
    kern<<<need, PushCfg<T>::threads, 0, st>>>(descs, ninst, total_units);
    return cudaGetLastError();
}

template <typename T>
cudaError_t permute_batch(const PushDesc<T>* descs, int ninst, int total_units, cudaStream_t st)
{
    count_launches(1);
    k_permute_batch<T><<<blocks_for(total_units, 8, 152 * 16), 256, 0, st>>>(descs, ninst, total_units);
    return cudaGetLastError();
}

template <typename T>
cudaError_t deposit_adjoint(PArrays<T> src, const int32_t* start, const double* gJ, const double* gM, double* gu0,
                            double* gx0, double* gw0, double* gB, const T* B, GridP g, SpeciesConst sc, cudaStream_t st,
                            const T* En, double* gEn)
{
    const double beta = sc.q * g.dt / (2.0 * sc.m);
    count_launches(1);
    const int nb = push_grid_blocks(g, sizeof(T) == 4 ? 32 : 64, 152 * 16);
    if (En)
        k_deposit_adjoint<T, true><<<nb, PushCfg<T>::threads, 0, st>>>(src, start, gJ, gM, gu0, gx0, gw0, gB, B, g,
                                                                       beta, sc.q, En, gEn);
    else
        k_deposit_adjoint<T, false><<<nb, PushCfg<T>::threads, 0, st>>>(src, start, gJ, gM, gu0, gx0, gw0, gB, B, g,
                                                                        beta, sc.q, nullptr, nullptr);
    return cudaGetLastError();
}

template <typename T>
cudaError_t push_adjoint(PArrays<T> src, const int32_t* start, const double* gu1, const double* gx1, double* gu0,
                         double* gx0, double* gE, double* gB, const T* Eth, const T* B, GridP g, SpeciesConst sc,
                         cudaStream_t st, const T* En, double* gEn)
{
    const double beta = sc.q * g.dt / (2.0 * sc.m);
    count_launches(1);
    const int nb = push_grid_blocks(g, sizeof(T) == 4 ? 32 : 64, 152 * 16);
    if (En)
        k_push_adjoint<T, true><<<nb, PushCfg<T>::threads, 0, st>>>(src, start, gu1, gx1, gu0, gx0, gE, gB, Eth, B,
                                                                    g, beta, En, gEn);
    else
        k_push_adjoint<T, false><<<nb, PushCfg<T>::threads, 0, st>>>(src, start, gu1, gx1, gu0, gx0, gE, gB, Eth, B,
                                                                     g, beta, nullptr, nullptr);
    return cudaGetLastError();
}

template <typename T>
cudaError_t push_general(PArrays<T> src, PArrays<T> dst, const int32_t* start, int32_t* key, const T* Eth,
                         const T* B, const T* En, GridP g, SpeciesConst sc, double* lsum_partial, int lsum_blocks,
                         cudaStream_t st)
{
    const T beta = (T)(sc.q * g.dt / (2.0 * sc.m));
    auto kern = En ? k_push_general<T, true> : k_push_general<T, false>;
    count_launches(1);
    kern<<<lsum_blocks, PushCfg<T>::threads, 0, st>>>(src, dst, start, key, Eth, B, En, g, beta,
                                                      (T)(g.dt / g.dx), (T)(g.dt / g.dy), (T)(sc.q * g.dt),
                                                      (T)sc.m, lsum_partial);
    return cudaGetLastError();
}

template <typename T>
cudaError_t permute(PArrays<T> src, PArrays<T> dst, const int32_t* start_new, const int32_t* n9,
                    const int32_t* off9, GridP g, int* err, cudaStream_t st)
{
    count_launches(1);
    k_permute<T><<<blocks_for(units_of(g.nx, g.ny), 8, 152 * 16), 256, 0, st>>>(src, dst, start_new, n9, off9,
                                                                             g, err);
    return cudaGetLastError();
}

template <typename T>
cudaError_t kinetic_energy(PArrays<T> p, int64_t n, double m, double* partial, int nblocks,
                           cudaStream_t st)
{
    count_launches(1);
    k_kinetic<T><<<nblocks, 256, 0, st>>>(p, n, (T)m, partial);
    return cudaGetLastError();
}

template <typename T>
cudaError_t spectrum(PArrays<T> p, int64_t n, int variable, const T* edges, int nbins, double* wsum,
                     unsigned long long* cnt, cudaStream_t st)
{
    if (n <= 0) return cudaSuccess;
    const size_t smem = (size_t)(nbins + 2) * (sizeof(double) + sizeof(double)) + (size_t)(nbins + 1) * sizeof(T);
    cudaError_t e = cudaFuncSetAttribute(k_spectrum<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    count_launches(1);
    k_spectrum<T><<<blocks_for(n, 256, 152 * 4), 256, smem, st>>>(p, n, variable, edges, nbins, wsum, cnt);
    return cudaGetLastError();
}

#define RELSIM_INSTANTIATE(T)                                                                      \
    template cudaError_t load_convert<T>(const double*, const double*, const double*, int64_t,     \
                                         GridP, PArrays<T>, int32_t*, int32_t*, int*, cudaStream_t); \
    template cudaError_t gather_particles<T>(const int32_t*, PArrays<T>, PArrays<T>, int64_t, bool, \
                                             cudaStream_t);                                        \
    template cudaError_t export_particles<T>(PArrays<T>, const int32_t*, GridP, double*, double*,  \
                                             double*, int32_t*, cudaStream_t);                     \
    template cudaError_t deposit<T>(const DepositSpecies<T>&, const T*, const T*, T*, T*, GridP, int*,  \
                                    cudaStream_t, int);                                             \
    template cudaError_t deposit_batch<T>(const DepDesc<T>*, int, int, bool, int*, cudaStream_t, int); \
    template cudaError_t push_sort_batch<T>(const PushDesc<T>*, int, int, bool, int, cudaStream_t);  \
    template cudaError_t permute_batch<T>(const PushDesc<T>*, int, int, cudaStream_t);              \
    template cudaError_t push_sort<T>(PArrays<T>, PArrays<T>, const int32_t*, int32_t*, int32_t*,   \
                                      const T*, const T*, const T*, GridP, SpeciesConst, double*,   \
                                      int, int*, cudaStream_t);                                           \
    template cudaError_t push_general<T>(PArrays<T>, PArrays<T>, const int32_t*, int32_t*, const T*, \
                                         const T*, const T*, GridP, SpeciesConst, double*, int,      \
                                         cudaStream_t);                                              \
    template cudaError_t deposit_adjoint<T>(PArrays<T>, const int32_t*, const double*, const double*, \
                                            double*, double*, double*, double*, const T*, GridP,      \
                                            SpeciesConst, cudaStream_t, const T*, double*);           \
    template cudaError_t push_adjoint<T>(PArrays<T>, const int32_t*, const double*, const double*,   \
                                         double*, double*, double*, double*, const T*, const T*,     \
                                         GridP, SpeciesConst, cudaStream_t, const T*, double*);      \
    template cudaError_t permute<T>(PArrays<T>, PArrays<T>, const int32_t*, const int32_t*,         \
                                    const int32_t*, GridP, int*, cudaStream_t);                     \
    template cudaError_t kinetic_energy<T>(PArrays<T>, int64_t, double, double*, int, cudaStream_t); \
    template cudaError_t spectrum<T>(PArrays<T>, int64_t, int, const T*, int, double*, unsigned long long*, \
                                     cudaStream_t);

RELSIM_INSTANTIATE(float)
RELSIM_INSTANTIATE(double)

}  // namespace relsim
