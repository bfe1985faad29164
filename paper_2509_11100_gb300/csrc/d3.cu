// d3.cu -- the 3D form of the step: periodic nx x ny x nz grid, trilinear
// (CIC) shape functions, so a particle touches the 8 nodes of its cell and
// its mass-matrix contributions couple node pairs up to one cell apart in
// each direction (the 27-node stencil), of which 14 offsets are stored (the
// stored block of a pair serves both orders). The scheme is that of the 2D
// kernels (Sec. 2: explicit pusher, implicit field solve through the mass
// matrices); node and cell (i,j,k) have linear index (k ny + j) nx + i,
// centres sit at (i+1/2, j+1/2, k+1/2), and a particle is stored as its cell
// (implicit in the cell-sorted order) plus FP32 offsets fx, fy, fz.
//
// Kernels:
//   k_load3, k_gather3, k_export3   load, re-sort gather, read-back
//   k_deposit3   warp per row segment of cells; for each cell the lanes stage
//                their particles' weights, c alpha and c alpha u / gbar in
//                shared memory, then each lane accumulates the node pairs it
//                owns over the cell's particles in registers and flushes them
//                once per cell (FP32 or FP64 atomics)
//   k_op3        the operator A = I + (theta dt)^2 curl_n curl_c + theta dt M,
//                one thread per node, in the three modes of the 2D operator
//   k_rhs3, k_field_update3   the right-hand side, the field update with the
//                field ledger terms
//   k_push3      warp per row segment, the push with the cell change of the
//                general path (any move length), followed by the radix sort
#include "launch.cuh"

namespace relsim {
namespace {

unsigned grid3(int64_t n, int threads, int64_t cap)
{
    int64_t b = (n + threads - 1) / threads;
    if (b > cap) b = cap;
    return (unsigned)(b > 0 ? b : 1);
}

__host__ __device__ __forceinline__ int64_t node3(int i, int j, int k, const GridP& g)
{
    return ((int64_t)k * g.ny + j) * g.nx + i;
}

// the half-stored offset index of d = (di, dj, dk), or -1 when -d is the
// stored one
__host__ __device__ __forceinline__ int half3(int di, int dj, int dk)
{
    if (dk == 1) return 5 + (dj + 1) * 3 + (di + 1);
    if (dk == 0 && dj == 1) return 2 + (di + 1);
    if (dk == 0 && dj == 0 && di >= 0) return di;
    return -1;
}

// ---------------------------------------------------------------------------
// load, gather, export

template <typename T>
__global__ void k_load3(const double* __restrict__ x, const double* __restrict__ u, const double* __restrict__ w,
                        int64_t n, GridP g, PArrays<T> out, T* __restrict__ ofz, int32_t* __restrict__ key,
                        int32_t* __restrict__ val, int* bad)
{
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x) {
        double s[3] = {x[3 * p] / g.dx, x[3 * p + 1] / g.dy, x[3 * p + 2] / g.dz};
        const double ux = u[3 * p], uy = u[3 * p + 1], uz = u[3 * p + 2], ww = w[p];
        if (!isfinite(s[0]) || !isfinite(s[1]) || !isfinite(s[2]) || !isfinite(ux) || !isfinite(uy) ||
            !isfinite(uz) || !isfinite(ww)) {
            atomicOr(bad, 1);
            s[0] = s[1] = s[2] = 0.0;
        }
        const int nn[3] = {g.nx, g.ny, g.nz};
        int c[3];
        T f[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            if (s[a] < 0.0 || s[a] >= (double)nn[a]) s[a] -= nn[a] * floor(s[a] / nn[a]);
            const double fl = floor(s[a]);
            int ci = (int)fl;
            if (ci >= nn[a]) ci -= nn[a];
            if (ci < 0) ci = 0;
            c[a] = ci;
            f[a] = from_double_rz<T>(s[a] - fl);
        }
        out.fx[p] = f[0];
        out.fy[p] = f[1];
        ofz[p] = f[2];
        out.ux[p] = (T)ux;
        out.uy[p] = (T)uy;
        out.uz[p] = (T)uz;
        out.w[p] = (T)ww;
        key[p] = (int32_t)node3(c[0], c[1], c[2], g);
        val[p] = (int32_t)p;
    }
}

template <typename T>
__global__ void k_gather3(const int32_t* __restrict__ perm, PArrays<T> src, const T* __restrict__ sfz, PArrays<T> dst,
                          T* __restrict__ dfz, int64_t n, bool ids_from_perm)
{
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x) {
        const int32_t s = perm[p];
        dst.fx[p] = src.fx[s];
        dst.fy[p] = src.fy[s];
        dfz[p] = sfz[s];
        dst.ux[p] = src.ux[s];
        dst.uy[p] = src.uy[s];
        dst.uz[p] = src.uz[s];
        dst.w[p] = src.w[s];
        if (dst.id) dst.id[p] = ids_from_perm ? s : src.id[s];
    }
}

// one warp per cell: absolute positions back to FP64 (x, y, z interleaved)
template <typename T>
__global__ void k_export3(PArrays<T> pa, const T* __restrict__ fz, const int32_t* __restrict__ start, GridP g,
                          double* x, double* u, double* w, int32_t* id)
{
    const int lane = threadIdx.x & 31;
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nwarps = (gridDim.x * blockDim.x) >> 5;
    for (int c = warp; c < g.ncell; c += nwarps) {
        const int i = c % g.nx, j = (c / g.nx) % g.ny, k = c / (g.nx * g.ny);
        const int p1 = start[c + 1];
        for (int p = start[c] + lane; p < p1; p += 32) {
            if (x) {
                x[3 * (int64_t)p] = ((double)i + (double)pa.fx[p]) * g.dx;
                x[3 * (int64_t)p + 1] = ((double)j + (double)pa.fy[p]) * g.dy;
                x[3 * (int64_t)p + 2] = ((double)k + (double)fz[p]) * g.dz;
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
// per-particle arithmetic shared by the deposit and the push

// trilinear weights of the 8 corners a = (a&1, (a>>1)&1, (a>>2)&1)
template <typename T>
__device__ __forceinline__ void corner_weights(T fx, T fy, T fz, T (&W)[8])
{
    const T X[2] = {T(1) - fx, fx}, Y[2] = {T(1) - fy, fy}, Z[2] = {T(1) - fz, fz};
#pragma unroll
    for (int a = 0; a < 8; ++a) W[a] = X[a & 1] * Y[(a >> 1) & 1] * Z[(a >> 2) & 1];
}

// alpha = (I - [a]x + a a^T)/(1 + |a|^2), a = beta B/gbar (row-major)
template <typename T>
__device__ __forceinline__ void alpha3(const T (&Bp)[3], T beta, T gbar, T (&al)[9])
{
    const T ax = beta * Bp[0] / gbar, ay = beta * Bp[1] / gbar, az = beta * Bp[2] / gbar;
    const T ia = T(1) / (T(1) + ax * ax + ay * ay + az * az);
    al[0] = (T(1) + ax * ax) * ia; al[1] = (ax * ay + az) * ia; al[2] = (ax * az - ay) * ia;
    al[3] = (ax * ay - az) * ia; al[4] = (T(1) + ay * ay) * ia; al[5] = (ay * az + ax) * ia;
    al[6] = (ax * az + ay) * ia; al[7] = (ay * az - ax) * ia; al[8] = (T(1) + az * az) * ia;
}

// ---------------------------------------------------------------------------
// field tiles of a row segment (cells i0 .. i0+cn-1 of row (j, k)), staged in
// shared memory once per segment instead of 24 gathers per particle per field

template <typename T>
struct Tile3 {
    T E[3][2][2][33];   // [comp][dy][dz][c]: node (i0 + c, j + dy, k + dz)
    T B[3][3][3][34];   // [comp][dy][dz][c]: centre (i0 - 1 + c, j - 1 + dy, k - 1 + dz)
};

template <typename T>
__device__ __forceinline__ void load_tile3(Tile3<T>& tl, const T* __restrict__ E, const T* __restrict__ B, int i0,
                                           int cn, int j, int k, const GridP& g, int lane)
{
    const int64_t nc = g.ncell;
    if (E)
        for (int q = lane; q < 3 * 2 * 2 * 33; q += 32) {
            const int c = q % 33, dz = (q / 33) % 2, dy = (q / 66) % 2, comp = q / 132;
            if (c <= cn)
                tl.E[comp][dy][dz][c] =
                    ld(E + comp * nc + node3(wrap1(i0 + c, g.nx), wrap1(j + dy, g.ny), wrap1(k + dz, g.nz), g));
        }
    for (int q = lane; q < 3 * 3 * 3 * 34; q += 32) {
        const int c = q % 34, dz = (q / 34) % 3, dy = (q / 102) % 3, comp = q / 306;
        if (c <= cn + 1)
            tl.B[comp][dy][dz][c] =
                ld(B + comp * nc + node3(wrap1(i0 - 1 + c, g.nx), wrap1(j - 1 + dy, g.ny), wrap1(k - 1 + dz, g.nz), g));
    }
    __syncwarp();
}

// B^n at a particle of local cell cl with offsets f, from the tile
template <typename T>
__device__ __forceinline__ void tile_B3(const Tile3<T>& tl, int cl, T fx, T fy, T fz, T (&Bp)[3])
{
    const bool lx = fx < T(0.5), ly = fy < T(0.5), lz = fz < T(0.5);
    const T tx = lx ? fx + T(0.5) : fx - T(0.5);
    const T ty = ly ? fy + T(0.5) : fy - T(0.5);
    const T tz = lz ? fz + T(0.5) : fz - T(0.5);
    const int c0 = lx ? cl : cl + 1, y0 = ly ? 0 : 1, z0 = lz ? 0 : 1;
    T W[8];
    corner_weights(tx, ty, tz, W);
#pragma unroll
    for (int comp = 0; comp < 3; ++comp) {
        T b = T(0);
#pragma unroll
        for (int a = 0; a < 8; ++a) b += W[a] * tl.B[comp][y0 + ((a >> 1) & 1)][z0 + ((a >> 2) & 1)][c0 + (a & 1)];
        Bp[comp] = b;
    }
}

// ---------------------------------------------------------------------------
// deposit

template <typename T>
struct DepCfg3 {
    static constexpr int warps = sizeof(T) == 4 ? 4 : 2;   // static shared memory < 48 KB
};
constexpr int kStage3 = 22;   // staged values per particle (20, padded to an even stride for paired loads)

// a pair block's 9 sums; in FP32 as four pairs and one, accumulated with
// the paired FMA (one instruction for two sums)
template <typename T>
struct PairAcc {
    T v[9];
    __device__ __forceinline__ void zero()
    {
#pragma unroll
        for (int e = 0; e < 9; ++e) v[e] = T(0);
    }
    __device__ __forceinline__ void add(T w, const T* al)
    {
#pragma unroll
        for (int e = 0; e < 9; ++e) v[e] += w * al[e];
    }
    __device__ __forceinline__ void get(T (&o)[9]) const
    {
#pragma unroll
        for (int e = 0; e < 9; ++e) o[e] = v[e];
    }
};
template <>
struct PairAcc<float> {
    float2 v2[4];
    float v8;
    __device__ __forceinline__ void zero()
    {
#pragma unroll
        for (int k = 0; k < 4; ++k) v2[k] = make_float2(0.f, 0.f);
        v8 = 0.f;
    }
    // al: 8-byte aligned row of the 9 staged values
    __device__ __forceinline__ void add(float w, const float2 (&al2)[4], float al8)
    {
        const float2 ww = make_float2(w, w);
#pragma unroll
        for (int k = 0; k < 4; ++k) v2[k] = __ffma2_rn(ww, al2[k], v2[k]);
        v8 = fmaf(w, al8, v8);
    }
    __device__ __forceinline__ void get(float (&o)[9]) const
    {
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            o[2 * k] = v2[k].x;
            o[2 * k + 1] = v2[k].y;
        }
        o[8] = v8;
    }
};

// a 3x3 block added to the stored block at dst (offset index hs): in FP32
// as paired atomics (8-byte aligned pairs: the block starts on an even float
// when hs is even, as 126 per node is even), halving the atomic operations
__device__ __forceinline__ void add_block9(float* dst, const float (&v)[9], int hs)
{
    // constant indices in both branches keep v in registers
    if (hs & 1) {
        atomicAdd(dst, v[0]);
#pragma unroll
        for (int e = 0; e < 4; ++e)
            atomicAdd(reinterpret_cast<float2*>(dst + 1 + 2 * e), make_float2(v[1 + 2 * e], v[2 + 2 * e]));
    } else {
#pragma unroll
        for (int e = 0; e < 4; ++e)
            atomicAdd(reinterpret_cast<float2*>(dst + 2 * e), make_float2(v[2 * e], v[2 * e + 1]));
        atomicAdd(dst + 8, v[8]);
    }
}
__device__ __forceinline__ void add_block9(double* dst, const double (&v)[9], int)
{
#pragma unroll
    for (int e = 0; e < 9; ++e) atomicAdd(dst + e, v[e]);
}

// flush a cell's pair block: the block of pair (a, b) is stored at corner a
// with the offset b - a when that offset is in the stored half, else at
// corner b with a - b
template <typename T>
__device__ __forceinline__ void flush_pair3(T* M, int a, int b, const T (&acc)[9], int i, int j, int k, GridP g)
{
    const int di = (b & 1) - (a & 1), dj = ((b >> 1) & 1) - ((a >> 1) & 1), dk = ((b >> 2) & 1) - ((a >> 2) & 1);
    int hs = half3(di, dj, dk), at = a;
    if (hs < 0) {
        hs = half3(-di, -dj, -dk);
        at = b;
    }
    const int64_t gn =
        node3(wrap1(i + (at & 1), g.nx), wrap1(j + ((at >> 1) & 1), g.ny), wrap1(k + ((at >> 2) & 1), g.nz), g);
    add_block9(M + gn * kMBlock3 + hs * 9, acc, hs);
}

// the 36 unordered corner pairs (a <= b) of a cell, pair q
__device__ __forceinline__ void pair_of(int q, int& a, int& b)
{
    int r = q;
    a = 0;
    while (r >= 8 - a) {
        r -= 8 - a;
        ++a;
    }
    b = a + r;
}

template <typename T>
__global__ void __launch_bounds__(32 * DepCfg3<T>::warps)
k_deposit3(DepositSpecies<T> ds, FzArrays<T> fz, const T* __restrict__ B, T* __restrict__ M, T* __restrict__ J,
           GridP g)
{
    constexpr int kW = DepCfg3<T>::warps;
    __shared__ __align__(16) T sh[kW][32][kStage3];
    __shared__ Tile3<T> stl[kW];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nwarps = (gridDim.x * blockDim.x) >> 5;
    const int nseg = (g.nx + 31) / 32;
    const int64_t nunits = (int64_t)nseg * g.ny * g.nz;
    T (*st)[kStage3] = sh[wib];
    // the pairs this lane owns (q0 = lane, q1 = lane + 32 for lanes 0..3) and
    // the current component it owns (lanes 4..27: corner (lane-4)/3, component (lane-4)%3)
    int a0, b0, a1 = 0, b1 = 0;
    pair_of(lane, a0, b0);
    const bool two = lane < 4;
    if (two) pair_of(lane + 32, a1, b1);
    const bool ownj = lane >= 4 && lane < 28;
    const int ja = ownj ? (lane - 4) / 3 : 0, jc = ownj ? (lane - 4) % 3 : 0;
    for (int64_t u = warp; u < nunits; u += nwarps) {
        const int i0 = (int)(u % nseg) * 32;
        const int jk = (int)(u / nseg);
        const int j = jk % g.ny, k = jk / g.ny;
        const int cn = min(32, g.nx - i0);
        __syncwarp();
        load_tile3<T>(stl[wib], nullptr, B, i0, cn, j, k, g, lane);
        for (int cl = 0; cl < cn; ++cl) {
            const int i = i0 + cl;
            const int64_t c = node3(i, j, k, g);
            PairAcc<T> acc0, acc1;
            acc0.zero();
            acc1.zero();
            T accj = T(0);
            // the cell's particles of all species as one list (cum[s] = the
            // first list index of species s), staged 32 at a time
            // (fully unrolled over the species so the tables stay in registers)
            int cum[kMaxSpecies + 1], pst[kMaxSpecies];
            cum[0] = 0;
#pragma unroll
            for (int s = 0; s < kMaxSpecies; ++s) {
                pst[s] = s < ds.nsp ? ds.start[s][c] : 0;
                cum[s + 1] = cum[s] + (s < ds.nsp ? ds.start[s][c + 1] - pst[s] : 0);
            }
            const int total = cum[kMaxSpecies];
            if (total == 0) continue;
            for (int q0 = 0; q0 < total; q0 += 32) {
                const int t = q0 + lane;
                if (t < total) {
                    int s = 0, p = pst[0] + t;
#pragma unroll
                    for (int q = 1; q < kMaxSpecies; ++q)
                        if (t >= cum[q] && cum[q + 1] > cum[q]) {
                            s = q;
                            p = pst[q] + (t - cum[q]);
                        }
                    const T fx = ld(ds.fx[s] + p), fy = ld(ds.fy[s] + p), fzz = ld(fz.fz[s] + p);
                    const T ux = ld(ds.ux[s] + p), uy = ld(ds.uy[s] + p), uz = ld(ds.uz[s] + p);
                    const T wt = ld(ds.w[s] + p);
                    T W[8], Bp[3], al[9];
                    corner_weights(fx, fy, fzz, W);
                    tile_B3(stl[wib], cl, fx, fy, fzz, Bp);
                    const T gbar = sqrt(T(1) + ux * ux + uy * uy + uz * uz);
                    alpha3(Bp, ds.beta[s], gbar, al);
                    const T cM = wt * ds.cM[s] / gbar, cJ = wt * ds.cJ[s] / gbar;
#pragma unroll
                    for (int a = 0; a < 8; ++a) st[lane][a] = W[a];
#pragma unroll
                    for (int e = 0; e < 9; ++e) st[lane][8 + e] = cM * al[e];
#pragma unroll
                    for (int r = 0; r < 3; ++r)
                        st[lane][17 + r] = cJ * (al[3 * r] * ux + al[3 * r + 1] * uy + al[3 * r + 2] * uz);
                }
                __syncwarp();
                const int m = min(32, total - q0);
                for (int t2 = 0; t2 < m; ++t2) {
                    const T wab = st[t2][a0] * st[t2][b0];
                    const T w1 = two ? st[t2][a1] * st[t2][b1] : T(0);
                    if constexpr (sizeof(T) == 4) {
                        float2 al2[4];
                        const float2* r2 = reinterpret_cast<const float2*>(&st[t2][8]);
#pragma unroll
                        for (int q = 0; q < 4; ++q) al2[q] = r2[q];
                        const float al8 = st[t2][16];
                        acc0.add(wab, al2, al8);
                        if (two) acc1.add(w1, al2, al8);
                    } else {
                        T al[9];
#pragma unroll
                        for (int e = 0; e < 9; ++e) al[e] = st[t2][8 + e];
                        acc0.add(wab, al);
                        if (two) acc1.add(w1, al);
                    }
                    if (ownj) accj += st[t2][ja] * st[t2][17 + jc];
                }
                __syncwarp();
            }
            // flush: the block of pair (a, b) is stored at corner a with the
            // offset b - a when that offset is in the stored half, else at
            // corner b with a - b
            {
                T v[9];
                acc0.get(v);
                flush_pair3(M, a0, b0, v, i, j, k, g);
                if (two) {
                    acc1.get(v);
                    flush_pair3(M, a1, b1, v, i, j, k, g);
                }
            }
            if (ownj) {
                const int64_t gn = node3(wrap1(i + (ja & 1), g.nx), wrap1(j + ((ja >> 1) & 1), g.ny),
                                         wrap1(k + ((ja >> 2) & 1), g.nz), g);
                atomicAdd(J + (int64_t)jc * g.ncell + gn, accj);
            }
        }
    }
}

// ---------------------------------------------------------------------------
// the implicit operator, the right-hand side and the field update

enum { k3A = 0, k3Residual = 1, k3Arnoldi = 2 };
constexpr int kOpX3 = 32, kOpY3 = 4, kOpZ3 = 2;
constexpr int kOpT3 = kOpX3 * kOpY3 * kOpZ3;
constexpr int kOpChunk3 = 8;

// the offset of stored block h (0..13)
__device__ __forceinline__ void half_offset3(int h, int& di, int& dj, int& dk)
{
    if (h < 2) { di = h; dj = 0; dk = 0; }
    else if (h < 5) { di = h - 3; dj = 1; dk = 0; }
    else { di = (h - 5) % 3 - 1; dj = (h - 5) / 3 - 1; dk = 1; }
}

// (curl_n curl_c v) at a node from v on its 3x3x3 neighbourhood,
// f(comp, a, b, c) = component comp at node (i-1+a, j-1+b, k-1+c)
template <typename T, typename F>
__device__ __forceinline__ void curlcurl3(F f, T rdx4, T rdy4, T rdz4, T (&out)[3])
{
    // curl_c at the 8 cells around the node: cell (ci, cj, ck) spans local
    // nodes ci..ci+1, cj..cj+1, ck..ck+1 (ci = 0: the cell i-1)
    T C[3][2][2][2];
#pragma unroll
    for (int ci = 0; ci < 2; ++ci)
#pragma unroll
        for (int cj = 0; cj < 2; ++cj)
#pragma unroll
            for (int ck = 0; ck < 2; ++ck) {
                T d[3][3];   // d[axis][comp]
#pragma unroll
                for (int comp = 0; comp < 3; ++comp) {
                    T sx = T(0), sy = T(0), sz = T(0);
#pragma unroll
                    for (int e1 = 0; e1 < 2; ++e1)
#pragma unroll
                        for (int e2 = 0; e2 < 2; ++e2) {
                            sx += f(comp, ci + 1, cj + e1, ck + e2) - f(comp, ci, cj + e1, ck + e2);
                            sy += f(comp, ci + e1, cj + 1, ck + e2) - f(comp, ci + e1, cj, ck + e2);
                            sz += f(comp, ci + e1, cj + e2, ck + 1) - f(comp, ci + e1, cj + e2, ck);
                        }
                    d[0][comp] = sx * rdx4;
                    d[1][comp] = sy * rdy4;
                    d[2][comp] = sz * rdz4;
                }
                C[0][ci][cj][ck] = d[1][2] - d[2][1];
                C[1][ci][cj][ck] = d[2][0] - d[0][2];
                C[2][ci][cj][ck] = d[0][1] - d[1][0];
            }
    // curl_n at the node from the 8 cells
    T d[3][3];
#pragma unroll
    for (int comp = 0; comp < 3; ++comp) {
        T sx = T(0), sy = T(0), sz = T(0);
#pragma unroll
        for (int e1 = 0; e1 < 2; ++e1)
#pragma unroll
            for (int e2 = 0; e2 < 2; ++e2) {
                sx += C[comp][1][e1][e2] - C[comp][0][e1][e2];
                sy += C[comp][e1][1][e2] - C[comp][e1][0][e2];
                sz += C[comp][e1][e2][1] - C[comp][e1][e2][0];
            }
        d[0][comp] = sx * rdx4;
        d[1][comp] = sy * rdy4;
        d[2][comp] = sz * rdz4;
    }
    out[0] = d[1][2] - d[2][1];
    out[1] = d[2][0] - d[0][2];
    out[2] = d[0][1] - d[1][0];
}

// (M v) at node (i, j, k): its own 14 stored blocks times v at g + d(h), and
// the 13 neighbours' blocks M[g - d(h)][h] times v at g - d(h); with TR each
// block applied transposed
template <typename T, bool TR, typename F>
__device__ __forceinline__ void mv3(const T* __restrict__ M, int i, int j, int k, const GridP& g, F f, T (&out)[3])
{
    T r[3] = {T(0), T(0), T(0)};
    const T* Mg = M + node3(i, j, k, g) * kMBlock3;
#pragma unroll
    for (int h = 0; h < kHalf3; ++h) {
        int di, dj, dk;
        half_offset3(h, di, dj, dk);
        const T* Mo = Mg + h * 9;
        T vv[3];
#pragma unroll
        for (int s = 0; s < 3; ++s) vv[s] = f(s, 1 + di, 1 + dj, 1 + dk);
#pragma unroll
        for (int rr = 0; rr < 3; ++rr)
#pragma unroll
            for (int s = 0; s < 3; ++s) r[rr] += ld(Mo + (TR ? s * 3 + rr : rr * 3 + s)) * vv[s];
        if (h == 0) continue;
        const T* Mn = M + node3(wrap1(i - di, g.nx), wrap1(j - dj, g.ny), wrap1(k - dk, g.nz), g) * kMBlock3 + h * 9;
#pragma unroll
        for (int s = 0; s < 3; ++s) vv[s] = f(s, 1 - di, 1 - dj, 1 - dk);
#pragma unroll
        for (int rr = 0; rr < 3; ++rr)
#pragma unroll
            for (int s = 0; s < 3; ++s) r[rr] += ld(Mn + (TR ? s * 3 + rr : rr * 3 + s)) * vv[s];
    }
    out[0] = r[0];
    out[1] = r[1];
    out[2] = r[2];
}

// The operator on tiles of 32 x 4 x 2 nodes, the input staged in T on the
// tile's 1-node halo (one FP64 load and conversion per staged value); the
// modes and the per-block partial sums are those of the 2D operator:
//   A:        out = in + B in
//   Residual: out = b - (in + B in), partial |out|^2
//   Arnoldi:  v = s in (to vj when vj is not null), out = B v, partials
//             <out, V_q> (q < nv), <out, v>, <out, out>
template <typename T, int MODE, bool TR>
__global__ void __launch_bounds__(kOpT3)
k_op3(const T* __restrict__ M, const double* __restrict__ in, double s, const double* __restrict__ b,
      double* __restrict__ out, double* __restrict__ vj, const double* __restrict__ V, int64_t ldv, int nv, GridP g,
      double* __restrict__ partial, const GmDyn* __restrict__ dyn)
{
    if (MODE == k3Arnoldi && dyn) {
        if (!dyn->live) return;
        in = dyn->in;
        s = dyn->s;
        vj = dyn->vj;
        out = dyn->out;
        nv = dyn->nv;
    }
    constexpr int HX = kOpX3 + 2, HY = kOpY3 + 2, HZ = kOpZ3 + 2;
    __shared__ T sv[3][HZ][HY][HX];
    __shared__ double buf[kOpChunk3][kOpT3];
    const int nx = g.nx, ny = g.ny, nz = g.nz;
    const int64_t nc = g.ncell;
    const int tx_n = (nx + kOpX3 - 1) / kOpX3, ty_n = (ny + kOpY3 - 1) / kOpY3;
    const int bx = blockIdx.x % tx_n, by = (blockIdx.x / tx_n) % ty_n, bz = blockIdx.x / (tx_n * ty_n);
    const int i0 = bx * kOpX3, j0 = by * kOpY3, k0 = bz * kOpZ3;
    const int tid = threadIdx.x, tx = tid % kOpX3, ty = (tid / kOpX3) % kOpY3, tz = tid / (kOpX3 * kOpY3);
    const int i = i0 + tx, j = j0 + ty, k = k0 + tz;
    const bool active = i < nx && j < ny && k < nz;
    const int64_t gidx = active ? node3(i, j, k, g) : 0;
    const T sT = (T)s;
    for (int q = tid; q < 3 * HZ * HY * HX; q += kOpT3) {
        const int comp = q / (HZ * HY * HX), rem = q % (HZ * HY * HX);
        const int zz = rem / (HY * HX), yy = (rem / HX) % HY, xx = rem % HX;
        const int gi = wrap1(min(i0 - 1 + xx, 2 * nx - 1), nx), gj = wrap1(min(j0 - 1 + yy, 2 * ny - 1), ny);
        const int gk = wrap1(min(k0 - 1 + zz, 2 * nz - 1), nz);
        T val = (T)__ldg(in + comp * nc + node3(gi, gj, gk, g));
        if (MODE == k3Arnoldi) val *= sT;
        sv[comp][zz][yy][xx] = val;
    }
    __syncthreads();
    double own[3] = {0.0, 0.0, 0.0}, wv[3] = {0.0, 0.0, 0.0};
    if (active) {
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            own[c] = __ldg(in + c * nc + gidx);
            if (MODE == k3Arnoldi && !is_one(s)) own[c] *= s;
        }
        auto f = [&](int comp, int a, int bb, int cc) -> T { return sv[comp][tz + cc][ty + bb][tx + a]; };
        T cc3[3], mv[3];
        curlcurl3<T>(f, gc<T>(g).qdx, gc<T>(g).qdy, gc<T>(g).qdz, cc3);
        mv3<T, TR>(M, i, j, k, g, f, mv);
        const T td = gc<T>(g).td;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const double bv = (double)(td * td * cc3[c] + td * mv[c]);
            if (MODE == k3A) wv[c] = own[c] + bv;
            else if (MODE == k3Residual) wv[c] = b[c * nc + gidx] - (own[c] + bv);
            else wv[c] = bv;
            out[c * nc + gidx] = wv[c];
            if (MODE == k3Arnoldi && vj) vj[c * nc + gidx] = own[c];
        }
    }
    if (MODE == k3A) return;
    const int nq = MODE == k3Residual ? 1 : nv + 2;
    const int lane = tid & 31, wid = tid >> 5;
    for (int q0 = 0; q0 < nq; q0 += kOpChunk3) {
        const int kc = min(kOpChunk3, nq - q0);
        for (int c = 0; c < kc; ++c) {
            const int q = q0 + c;
            double d = 0.0;
            if (active) {
                if (MODE == k3Residual || q == nv + 1) d = wv[0] * wv[0] + wv[1] * wv[1] + wv[2] * wv[2];
                else if (q == nv) d = wv[0] * own[0] + wv[1] * own[1] + wv[2] * own[2];
                else {
                    const double* Vq = V + (int64_t)q * ldv + gidx;
                    d = wv[0] * __ldg(Vq) + wv[1] * __ldg(Vq + nc) + wv[2] * __ldg(Vq + 2 * nc);
                }
            }
            buf[c][tid] = d;
        }
        __syncthreads();
        for (int c = wid; c < kc; c += kOpT3 / 32) {
            double t = 0.0;
#pragma unroll
            for (int m = 0; m < kOpT3 / 32; ++m) t += buf[c][m * 32 + lane];
            t = warp_sum(t);
            if (lane == 0) partial[(int64_t)blockIdx.x * nq + q0 + c] = t;
        }
        __syncthreads();
    }
}

// b = E^n + theta dt curl_n B^n - theta dt Jhat
template <typename T>
__global__ void k_rhs3(const T* __restrict__ E, const T* __restrict__ B, const T* __restrict__ J,
                       double* __restrict__ b, GridP g)
{
    const int64_t nc = g.ncell;
    for (int64_t gi = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; gi < nc; gi += (int64_t)gridDim.x * blockDim.x) {
        const int i = (int)(gi % g.nx), j = (int)((gi / g.nx) % g.ny), k = (int)(gi / ((int64_t)g.nx * g.ny));
        const int ii[2] = {wrap1(i - 1, g.nx), i}, jj[2] = {wrap1(j - 1, g.ny), j}, kk[2] = {wrap1(k - 1, g.nz), k};
        T d[3][3];
#pragma unroll
        for (int comp = 0; comp < 3; ++comp) {
            const T* f = B + comp * nc;
            T sx = T(0), sy = T(0), sz = T(0);
#pragma unroll
            for (int e1 = 0; e1 < 2; ++e1)
#pragma unroll
                for (int e2 = 0; e2 < 2; ++e2) {
                    sx += f[node3(ii[1], jj[e1], kk[e2], g)] - f[node3(ii[0], jj[e1], kk[e2], g)];
                    sy += f[node3(ii[e1], jj[1], kk[e2], g)] - f[node3(ii[e1], jj[0], kk[e2], g)];
                    sz += f[node3(ii[e1], jj[e2], kk[1], g)] - f[node3(ii[e1], jj[e2], kk[0], g)];
                }
            d[0][comp] = sx * gc<T>(g).qdx;
            d[1][comp] = sy * gc<T>(g).qdy;
            d[2][comp] = sz * gc<T>(g).qdz;
        }
        const T cn[3] = {d[1][2] - d[2][1], d[2][0] - d[0][2], d[0][1] - d[1][0]};
        const T td = gc<T>(g).td;
#pragma unroll
        for (int comp = 0; comp < 3; ++comp)
            b[comp * nc + gi] = (double)(E[comp * nc + gi] + td * cn[comp] - td * J[comp * nc + gi]);
    }
}

constexpr int kFieldLedger3 = 6;

// E^{n+theta} (FP64 solution) -> Eth, E^{n+1}, B^{n+1} of cell (i,j,k) and the
// field ledger terms 0..4 (as the 2D field update); term 5 (the work) by
// k_work3 from Eth in T
template <typename T>
__global__ void __launch_bounds__(256)
k_field_update3(const double* __restrict__ x, T* __restrict__ Eth, T* __restrict__ E, const T* __restrict__ B0,
                T* __restrict__ B1, GridP g, double* __restrict__ partial)
{
    __shared__ double red[32 * 5];
    const int64_t nc = g.ncell;
    const int64_t gidx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    T acc[5] = {T(0), T(0), T(0), T(0), T(0)};
    if (gidx < nc) {
        const int i = (int)(gidx % g.nx), j = (int)((gidx / g.nx) % g.ny), k = (int)(gidx / ((int64_t)g.nx * g.ny));
        const T th = gc<T>(g).theta, hdV = gc<T>(g).hdV;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const T et = (T)x[c * nc + gidx];
            const T e0 = E[c * nc + gidx];
            const T e1 = (et - (T(1) - th) * e0) / th;
            Eth[c * nc + gidx] = et;
            E[c * nc + gidx] = e1;
            acc[0] += hdV * (e1 - e0) * (e1 + e0);
            acc[2] += (e1 - e0) * (e1 - e0);
            acc[3] += hdV * e1 * e1;
        }
        const int ii[2] = {i, wrap1(i + 1, g.nx)}, jj[2] = {j, wrap1(j + 1, g.ny)}, kk[2] = {k, wrap1(k + 1, g.nz)};
        T d[3][3];
#pragma unroll
        for (int comp = 0; comp < 3; ++comp) {
            T sx = T(0), sy = T(0), sz = T(0);
#pragma unroll
            for (int e1 = 0; e1 < 2; ++e1)
#pragma unroll
                for (int e2 = 0; e2 < 2; ++e2) {
                    sx += (T)x[comp * nc + node3(ii[1], jj[e1], kk[e2], g)] - (T)x[comp * nc + node3(ii[0], jj[e1], kk[e2], g)];
                    sy += (T)x[comp * nc + node3(ii[e1], jj[1], kk[e2], g)] - (T)x[comp * nc + node3(ii[e1], jj[0], kk[e2], g)];
                    sz += (T)x[comp * nc + node3(ii[e1], jj[e2], kk[1], g)] - (T)x[comp * nc + node3(ii[e1], jj[e2], kk[0], g)];
                }
            d[0][comp] = sx * gc<T>(g).qdx;
            d[1][comp] = sy * gc<T>(g).qdy;
            d[2][comp] = sz * gc<T>(g).qdz;
        }
        const T curl[3] = {d[1][2] - d[2][1], d[2][0] - d[0][2], d[0][1] - d[1][0]};
        const T dt = gc<T>(g).dt;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const T b0 = B0[c * nc + gidx];
            const T b1 = b0 - dt * curl[c];
            B1[c * nc + gidx] = b1;
            acc[1] += hdV * (b1 - b0) * (b1 + b0);
            acc[2] += (b1 - b0) * (b1 - b0);
            acc[4] += hdV * b1 * b1;
        }
        acc[2] *= gc<T>(g).thdV;
    }
    double v[5], o[5];
#pragma unroll
    for (int q = 0; q < 5; ++q) v[q] = (double)acc[q];
    block_sum<5>(v, red, o);
    if (threadIdx.x == 0)
#pragma unroll
        for (int q = 0; q < 5; ++q) partial[(int64_t)blockIdx.x * kFieldLedger3 + q] = o[q];
}

// ledger term 5: dt dV (Jhat + M E^{n+theta}) . E^{n+theta}, with the same
// blocks as k_field_update3
template <typename T>
__global__ void __launch_bounds__(256)
k_work3(const T* __restrict__ M, const T* __restrict__ J, const T* __restrict__ Eth, GridP g,
        double* __restrict__ partial)
{
    __shared__ double red[32];
    const int64_t nc = g.ncell;
    const int64_t gidx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    T wk = T(0);
    if (gidx < nc) {
        const int i = (int)(gidx % g.nx), j = (int)((gidx / g.nx) % g.ny), k = (int)(gidx / ((int64_t)g.nx * g.ny));
        auto f = [&](int comp, int a, int b, int c) -> T {
            return ld(Eth + comp * nc + node3(wrap1(i - 1 + a, g.nx), wrap1(j - 1 + b, g.ny), wrap1(k - 1 + c, g.nz), g));
        };
        T mv[3];
        mv3<T, false>(M, i, j, k, g, f, mv);
#pragma unroll
        for (int c = 0; c < 3; ++c) wk += (J[c * nc + gidx] + mv[c]) * Eth[c * nc + gidx];
        wk *= gc<T>(g).dtdV;
    }
    double v[1] = {(double)wk}, o[1];
    block_sum<1>(v, red, o);
    if (threadIdx.x == 0) partial[(int64_t)blockIdx.x * kFieldLedger3 + 5] = o[0];
}

// ---------------------------------------------------------------------------
// push

constexpr int kPushWarps3 = 4;

// The explicit push with E^{n+theta} and B^n at x^{n+1/2}: ubar = alpha (u +
// beta E), u^{n+1} = 2 ubar - u^n, x^{n+3/2} = x^{n+1/2} + dt u^{n+1}/gamma^{n+1}
// as a cell shift plus offsets; the pushed particle goes to the same index
// of dst with its new cell in key. Ledger sums per block: dK, work,
// mismatch, K1 (as the 2D push). Warp per row segment of up to 32 cells, the
// lanes over the segment's particles. With rank non-null each particle also
// takes a slot among its new cell's particles, rank[p] = count[key]++ (one
// atomic per new cell and warp: the lanes with equal keys found by
// match-any), for the unstable counting sort that follows.
template <typename T>
__global__ void __launch_bounds__(32 * kPushWarps3)
k_push3(PArrays<T> src, const T* __restrict__ sfz, PArrays<T> dst, T* __restrict__ dfz,
        const int32_t* __restrict__ start, int32_t* __restrict__ key, int32_t* __restrict__ rank,
        int32_t* __restrict__ count, const T* __restrict__ Eth, const T* __restrict__ B, GridP g, T beta, T qdt,
        T m, double* __restrict__ lsum)
{
    __shared__ int sst[kPushWarps3][33];
    __shared__ Tile3<T> stl[kPushWarps3];
    __shared__ double red[32 * 4];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nwarps = (gridDim.x * blockDim.x) >> 5;
    const int nseg = (g.nx + 31) / 32;
    const int64_t nunits = (int64_t)nseg * g.ny * g.nz;
    int* ss = sst[wib];
    const T dt = gc<T>(g).dt, rdx = gc<T>(g).rdx, rdy = gc<T>(g).rdy, rdz = gc<T>(g).rdz;
    T acc[4] = {T(0), T(0), T(0), T(0)};
    for (int64_t u = warp; u < nunits; u += nwarps) {
        const int i0 = (int)(u % nseg) * 32;
        const int jk = (int)(u / nseg);
        const int j = jk % g.ny, k = jk / g.ny;
        const int cn = min(32, g.nx - i0);
        const int64_t c0 = node3(i0, j, k, g);
        __syncwarp();
        if (lane <= cn) ss[lane] = start[c0 + lane];
        if (lane == 0 && cn == 32) ss[32] = start[c0 + 32];
        load_tile3<T>(stl[wib], Eth, B, i0, cn, j, k, g, lane);
        const Tile3<T>& tl = stl[wib];
        const int P0 = ss[0], P1 = ss[cn];
        int cl = 0;
        for (int p0 = P0; p0 < P1; p0 += 32) {
            const int p = p0 + lane;
            const bool act = p < P1;
            int newkey = -1 - lane;   // distinct for idle lanes
            if (act) {
            while (ss[cl + 1] <= p) ++cl;
            const int i = i0 + cl;
            const T fx = ld(src.fx + p), fy = ld(src.fy + p), fz = ld(sfz + p);
            const T ux = ld(src.ux + p), uy = ld(src.uy + p), uz = ld(src.uz + p), w = ld(src.w + p);
            T W[8];
            corner_weights(fx, fy, fz, W);
            T E[3];
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                T e = T(0);
#pragma unroll
                for (int a = 0; a < 8; ++a) e += W[a] * tl.E[c][(a >> 1) & 1][(a >> 2) & 1][cl + (a & 1)];
                E[c] = e;
            }
            T Bp[3];
            tile_B3(tl, cl, fx, fy, fz, Bp);
            const T u02 = ux * ux + uy * uy + uz * uz;
            const T g0 = sqrt(T(1) + u02);
            const T ax = beta * Bp[0] / g0, ay = beta * Bp[1] / g0, az = beta * Bp[2] / g0;
            const T sa = T(1) / (T(1) + ax * ax + ay * ay + az * az);
            const T wx = ux + beta * E[0], wy = uy + beta * E[1], wz = uz + beta * E[2];
            const T wa = wx * ax + wy * ay + wz * az;
            const T ubx = sa * (wx + (wy * az - wz * ay) + wa * ax);
            const T uby = sa * (wy + (wz * ax - wx * az) + wa * ay);
            const T ubz = sa * (wz + (wx * ay - wy * ax) + wa * az);
            const T u1x = T(2) * ubx - ux, u1y = T(2) * uby - uy, u1z = T(2) * ubz - uz;
            const T u12 = u1x * u1x + u1y * u1y + u1z * u1z;
            const T g1 = sqrt(T(1) + u12);
            const T t[3] = {fx + dt * rdx * (u1x / g1), fy + dt * rdy * (u1y / g1), fz + dt * rdz * (u1z / g1)};
            const int nn[3] = {g.nx, g.ny, g.nz}, cc[3] = {i, j, k};
            T fn[3];
            int cnew[3];
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                const T fl = floor(t[a]);
                int sh = (int)fl;
                T f = t[a] - fl;
                if (f >= T(1)) { f -= T(1); sh += 1; }
                fn[a] = f;
                int q = (cc[a] + sh) % nn[a];
                if (q < 0) q += nn[a];
                cnew[a] = q;
            }
            dst.fx[p] = fn[0];
            dst.fy[p] = fn[1];
            dfz[p] = fn[2];
            dst.ux[p] = u1x;
            dst.uy[p] = u1y;
            dst.uz[p] = u1z;
            dst.w[p] = w;
            if (dst.id) dst.id[p] = src.id[p];
            newkey = (int32_t)node3(cnew[0], cnew[1], cnew[2], g);
            key[p] = newkey;
            // ledger: g0 - g1 = (u0 - u1).(u0 + u1)/(g0 + g1)
            const T ue = ubx * E[0] + uby * E[1] + ubz * E[2];
            const T du = (ux - u1x) * (ux + u1x) + (uy - u1y) * (uy + u1y) + (uz - u1z) * (uz + u1z);
            const T igs = T(1) / (g0 + g1);
            acc[0] -= w * m * du * igs;
            acc[1] += qdt * w * ue / g0;
            acc[2] += qdt * w * ue * du * igs * igs / g0;
            acc[3] += w * m * u12 / (g1 + T(1));
            }
            if (rank) {
                const unsigned peers = __match_any_sync(0xffffffffu, newkey);
                const int leader = __ffs(peers) - 1;
                int base = 0;
                if (act && lane == leader) base = atomicAdd(count + newkey, __popc(peers));
                base = __shfl_sync(0xffffffffu, base, leader);
                if (act) rank[p] = base + __popc(peers & ((1u << lane) - 1u));
            }
        }
        __syncwarp();
    }
    double v[4], o[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) v[q] = (double)acc[q];
    block_sum<4>(v, red, o);
    if (threadIdx.x == 0)
#pragma unroll
        for (int q = 0; q < 4; ++q) lsum[(int64_t)blockIdx.x * 4 + q] = o[q];
}

// the counting sort's placement: particle p to start[key[p]] + rank[p]
template <typename T>
__global__ void k_place3(PArrays<T> src, const T* __restrict__ sfz, PArrays<T> dst, T* __restrict__ dfz,
                         const int32_t* __restrict__ key, const int32_t* __restrict__ rank,
                         const int32_t* __restrict__ start, int64_t n)
{
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x) {
        const int64_t q = (int64_t)start[key[p]] + rank[p];
        dst.fx[q] = src.fx[p];
        dst.fy[q] = src.fy[p];
        if (dfz) dfz[q] = sfz[p];   // null for 2D particles
        dst.ux[q] = src.ux[p];
        dst.uy[q] = src.uy[p];
        dst.uz[q] = src.uz[p];
        dst.w[q] = src.w[p];
        if (dst.id) dst.id[q] = src.id[p];
    }
}

}  // namespace

template <typename T>
cudaError_t load_convert3(const double* x, const double* u, const double* w, int64_t n, GridP g, PArrays<T> out,
                          T* ofz, int32_t* key, int32_t* val, int* bad, cudaStream_t st)
{
    if (n <= 0) return cudaSuccess;
    count_launches(1);
    k_load3<T><<<grid3(n, 256, 152 * 32), 256, 0, st>>>(x, u, w, n, g, out, ofz, key, val, bad);
    return cudaGetLastError();
}

template <typename T>
cudaError_t gather_particles3(const int32_t* perm, PArrays<T> src, const T* sfz, PArrays<T> dst, T* dfz, int64_t n,
                              bool ids_from_perm, cudaStream_t st)
{
    if (n <= 0) return cudaSuccess;
    count_launches(1);
    k_gather3<T><<<grid3(n, 256, 152 * 32), 256, 0, st>>>(perm, src, sfz, dst, dfz, n, ids_from_perm);
    return cudaGetLastError();
}

template <typename T>
cudaError_t export_particles3(PArrays<T> p, const T* fz, const int32_t* start, GridP g, double* x, double* u,
                              double* w, int32_t* id, cudaStream_t st)
{
    count_launches(1);
    k_export3<T><<<grid3((int64_t)g.ncell * 32, 256, 152 * 16), 256, 0, st>>>(p, fz, start, g, x, u, w, id);
    return cudaGetLastError();
}

template <typename T>
cudaError_t deposit3(const DepositSpecies<T>& ds, const FzArrays<T>& fz, const T* B, T* M, T* J, GridP g,
                     cudaStream_t st, int blocks)
{
    const int64_t units = (int64_t)((g.nx + 31) / 32) * g.ny * g.nz;
    count_launches(1);
    k_deposit3<T><<<grid3(units, DepCfg3<T>::warps, blocks > 0 ? blocks : 152 * 8), 32 * DepCfg3<T>::warps, 0, st>>>(
        ds, fz, B, M, J, g);
    return cudaGetLastError();
}

int op_blocks3(GridP g)
{
    return ((g.nx + kOpX3 - 1) / kOpX3) * ((g.ny + kOpY3 - 1) / kOpY3) * ((g.nz + kOpZ3 - 1) / kOpZ3);
}

template <typename T, int MODE, bool TR>
cudaError_t launch_op3(const T* M, const double* in, double sc, const double* b, double* out, double* vj,
                       const double* V, int64_t ldv, int nv, GridP g, double* partial, cudaStream_t st,
                       const GmDyn* dyn)
{
    count_launches(1);
    k_op3<T, MODE, TR><<<op_blocks3(g), kOpT3, 0, st>>>(M, in, sc, b, out, vj, V, ldv, nv, g, partial, dyn);
    return cudaGetLastError();
}

template <typename T>
cudaError_t rhs3(const T* E, const T* B, const T* J, double* b, GridP g, cudaStream_t st)
{
    count_launches(1);
    k_rhs3<T><<<grid3(g.ncell, 256, 152 * 32), 256, 0, st>>>(E, B, J, b, g);
    return cudaGetLastError();
}

template <typename T>
cudaError_t field_update3(const double* x, const T* M, const T* J, T* Eth, T* E, const T* B0, T* B1, GridP g,
                          double* partial, int nblocks, cudaStream_t st)
{
    count_launches(2);
    k_field_update3<T><<<nblocks, 256, 0, st>>>(x, Eth, E, B0, B1, g, partial);
    k_work3<T><<<nblocks, 256, 0, st>>>(M, J, Eth, g, partial);
    return cudaGetLastError();
}

int push_blocks3(GridP g, int cap)
{
    const int64_t units = (int64_t)((g.nx + 31) / 32) * g.ny * g.nz;
    return (int)grid3(units, kPushWarps3, cap > 0 ? cap : 152 * 16);
}

template <typename T>
cudaError_t push3(PArrays<T> src, const T* sfz, PArrays<T> dst, T* dfz, const int32_t* start, int32_t* key,
                  int32_t* rank, int32_t* count, const T* Eth, const T* B, GridP g, SpeciesConst sc, double* lsum,
                  int nblocks, cudaStream_t st)
{
    count_launches(1);
    k_push3<T><<<nblocks, 32 * kPushWarps3, 0, st>>>(src, sfz, dst, dfz, start, key, rank, count, Eth, B, g,
                                                       (T)(sc.q * g.dt / (2.0 * sc.m)), (T)(sc.q * g.dt), (T)sc.m,
                                                       lsum);
    return cudaGetLastError();
}

template <typename T>
cudaError_t place3(PArrays<T> src, const T* sfz, PArrays<T> dst, T* dfz, const int32_t* key, const int32_t* rank,
                   const int32_t* start, int64_t n, cudaStream_t st)
{
    if (n <= 0) return cudaSuccess;
    count_launches(1);
    k_place3<T><<<grid3(n, 256, 152 * 32), 256, 0, st>>>(src, sfz, dst, dfz, key, rank, start, n);
    return cudaGetLastError();
}

#define RELSIM_D3_INSTANTIATE(T)                                                                                   \
    template cudaError_t load_convert3<T>(const double*, const double*, const double*, int64_t, GridP, PArrays<T>, \
                                          T*, int32_t*, int32_t*, int*, cudaStream_t);                             \
    template cudaError_t gather_particles3<T>(const int32_t*, PArrays<T>, const T*, PArrays<T>, T*, int64_t, bool, \
                                              cudaStream_t);                                                       \
    template cudaError_t export_particles3<T>(PArrays<T>, const T*, const int32_t*, GridP, double*, double*,       \
                                              double*, int32_t*, cudaStream_t);                                    \
    template cudaError_t deposit3<T>(const DepositSpecies<T>&, const FzArrays<T>&, const T*, T*, T*, GridP,        \
                                     cudaStream_t, int);                                                                \
    template cudaError_t rhs3<T>(const T*, const T*, const T*, double*, GridP, cudaStream_t);                      \
    template cudaError_t field_update3<T>(const double*, const T*, const T*, T*, T*, const T*, T*, GridP, double*, \
                                          int, cudaStream_t);                                                      \
    template cudaError_t push3<T>(PArrays<T>, const T*, PArrays<T>, T*, const int32_t*, int32_t*, int32_t*,        \
                                  int32_t*, const T*, const T*, GridP, SpeciesConst, double*, int, cudaStream_t);  \
    template cudaError_t place3<T>(PArrays<T>, const T*, PArrays<T>, T*, const int32_t*, const int32_t*,           \
                                   const int32_t*, int64_t, cudaStream_t);                                         \
    template cudaError_t launch_op3<T, 0, false>(const T*, const double*, double, const double*, double*, double*, \
                                                 const double*, int64_t, int, GridP, double*, cudaStream_t,        \
                                                 const GmDyn*);                                                    \
    template cudaError_t launch_op3<T, 1, false>(const T*, const double*, double, const double*, double*, double*, \
                                                 const double*, int64_t, int, GridP, double*, cudaStream_t,        \
                                                 const GmDyn*);                                                    \
    template cudaError_t launch_op3<T, 2, false>(const T*, const double*, double, const double*, double*, double*, \
                                                 const double*, int64_t, int, GridP, double*, cudaStream_t,        \
                                                 const GmDyn*);                                                    \
    template cudaError_t launch_op3<T, 0, true>(const T*, const double*, double, const double*, double*, double*,  \
                                                const double*, int64_t, int, GridP, double*, cudaStream_t,         \
                                                const GmDyn*);                                                     \
    template cudaError_t launch_op3<T, 1, true>(const T*, const double*, double, const double*, double*, double*,  \
                                                const double*, int64_t, int, GridP, double*, cudaStream_t,         \
                                                const GmDyn*);                                                     \
    template cudaError_t launch_op3<T, 2, true>(const T*, const double*, double, const double*, double*, double*,  \
                                                const double*, int64_t, int, GridP, double*, cudaStream_t,         \
                                                const GmDyn*);

RELSIM_D3_INSTANTIATE(float)
RELSIM_D3_INSTANTIATE(double)

}  // namespace relsim
