// quad.cu -- the 2D step with quadratic (triangular-shaped-cloud) shape
// functions, the higher-order variant of the linear shape of the other 2D
// kernels (same scheme, Sec. 2). Along each axis a particle at lattice
// coordinate s touches the nearest node n = floor(s + 1/2) and its two
// neighbours with weights 1/2 (1/2 - d)^2, 3/4 - d^2, 1/2 (1/2 + d)^2,
// d = s - n. In cell i with offset f that is nodes i-1 .. i+1 (f < 1/2, d =
// f) or i .. i+2 (f >= 1/2, d = f - 1); B on the centre lattice is gathered
// from centres i-1 .. i+1 with d = f - 1/2, whatever f. Node pairs of a
// particle lie up to two cells apart: 25 offsets, 13 stored per node in the
// order (0,0), (1,0), (2,0), (di,1) for di = -2..2, (di,2) for di = -2..2
// (a stored block serves both orders of its pair).
//
// Kernels:
//   k_deposit_q   warp per row segment of cells, the segment's B staged in
//                 shared memory; per cell the particles of all species staged
//                 in four groups by the half of the cell they sit in (each
//                 group touches a fixed 3 x 3 of the cell's 4 x 4 nodes); per
//                 group each lane sums up to 2 of the 45 node pairs of 3 x 3
//                 nodes with paired FP32 FMAs and adds them to the cell's 106
//                 pair sums in shared memory, flushed once per cell
//   k_op_q        the operator on 32 x 8-node tiles, the input staged on a
//                 2-node halo, the 25 blocks per node from global memory, the
//                 modes and partial dot products of the other operators
//   k_field_update_q, k_work_q   the field update and the ledger terms
//   k_push_q      warp per row segment with E and B tiles, the push, the new
//                 cell and its slot for the counting sort (k_place3 places)
#include "launch.cuh"

namespace relsim {
namespace {

constexpr int kQX = 32;   // cells per row segment

unsigned gridq(int64_t n, int threads, int64_t cap)
{
    int64_t b = (n + threads - 1) / threads;
    if (b > cap) b = cap;
    return (unsigned)(b > 0 ? b : 1);
}

// the stored index of offset (di, dj), or -1 when (-di, -dj) is stored
__host__ __device__ __forceinline__ int halfq(int di, int dj)
{
    if (dj == 2) return 8 + di + 2;
    if (dj == 1) return 3 + di + 2;
    if (dj == 0 && di >= 0) return di;
    return -1;
}

__device__ __forceinline__ void halfq_offset(int h, int& di, int& dj)
{
    if (h < 3) { di = h; dj = 0; }
    else if (h < 8) { di = h - 5; dj = 1; }
    else { di = h - 10; dj = 2; }
}

// the three weights of a particle along one axis (d in [-1/2, 1/2))
template <typename T>
__device__ __forceinline__ void quad3(T d, T (&w)[3])
{
    const T a = T(0.5) - d, b = T(0.5) + d;
    w[0] = T(0.5) * a * a;
    w[1] = T(0.75) - d * d;
    w[2] = T(0.5) * b * b;
}

// the weights on the 4 nodes i-1 .. i+2 of the axis (one of them zero)
template <typename T>
__device__ __forceinline__ void node4(T f, T (&w4)[4])
{
    T w[3];
    const bool hi = f >= T(0.5);
    quad3(hi ? f - T(1) : f, w);
    w4[0] = hi ? T(0) : w[0];
    w4[1] = hi ? w[0] : w[1];
    w4[2] = hi ? w[1] : w[2];
    w4[3] = hi ? w[2] : T(0);
}

// field tiles of a row segment (cells i0 .. i0+cn-1 of row j)
template <typename T>
struct TileQ {
    T E[3][4][kQX + 3];   // node (i0 - 1 + c, j - 1 + r)
    T B[3][3][kQX + 2];   // centre (i0 - 1 + c, j - 1 + r)
};

template <typename T>
__device__ __forceinline__ void load_tileq(TileQ<T>& tl, const T* __restrict__ E, const T* __restrict__ B, int i0,
                                           int cn, int j, const GridP& g, int lane)
{
    const int nc = g.ncell;
    if (E)
        for (int q = lane; q < 3 * 4 * (kQX + 3); q += 32) {
            const int c = q % (kQX + 3), r = (q / (kQX + 3)) % 4, comp = q / (4 * (kQX + 3));
            if (c <= cn + 2)
                tl.E[comp][r][c] = ld(E + comp * nc + wrap1(j - 1 + r, g.ny) * g.nx + wrap1(i0 - 1 + c, g.nx));
        }
    for (int q = lane; q < 3 * 3 * (kQX + 2); q += 32) {
        const int c = q % (kQX + 2), r = (q / (kQX + 2)) % 3, comp = q / (3 * (kQX + 2));
        if (c <= cn + 1)
            tl.B[comp][r][c] = ld(B + comp * nc + wrap1(j - 1 + r, g.ny) * g.nx + wrap1(i0 - 1 + c, g.nx));
    }
    __syncwarp();
}

// B^n at a particle of local cell cl: centres cl-1 .. cl+1 (tile columns
// cl .. cl+2), rows j-1 .. j+1
template <typename T>
__device__ __forceinline__ void tile_Bq(const TileQ<T>& tl, int cl, T fx, T fy, T (&Bp)[3])
{
    T wx[3], wy[3];
    quad3(fx - T(0.5), wx);
    quad3(fy - T(0.5), wy);
#pragma unroll
    for (int comp = 0; comp < 3; ++comp) {
        T b = T(0);
#pragma unroll
        for (int r = 0; r < 3; ++r)
#pragma unroll
            for (int c = 0; c < 3; ++c) b += wy[r] * wx[c] * tl.B[comp][r][cl + c];
        Bp[comp] = b;
    }
}

template <typename T>
__device__ __forceinline__ void alphaq(const T (&Bp)[3], T beta, T gbar, T (&al)[9])
{
    const T ax = beta * Bp[0] / gbar, ay = beta * Bp[1] / gbar, az = beta * Bp[2] / gbar;
    const T ia = T(1) / (T(1) + ax * ax + ay * ay + az * az);
    al[0] = (T(1) + ax * ax) * ia; al[1] = (ax * ay + az) * ia; al[2] = (ax * az - ay) * ia;
    al[3] = (ax * ay - az) * ia; al[4] = (T(1) + ay * ay) * ia; al[5] = (ay * az + ax) * ia;
    al[6] = (ax * az + ay) * ia; al[7] = (ay * az - ax) * ia; al[8] = (T(1) + az * az) * ia;
}

// ---------------------------------------------------------------------------
// deposit

constexpr int kPairsQ = 106;  // node pairs of the 4 x 4 union at most two apart per axis

template <typename T>
struct DepCfgQ {
    static constexpr int warps = sizeof(T) == 4 ? 4 : 2;
    static constexpr int min_blocks = sizeof(T) == 4 ? 4 : 1;   // FP32: at most 128 registers
};

template <typename T>
struct AccQ {
    T v[9];
    __device__ __forceinline__ void zero()
    {
#pragma unroll
        for (int e = 0; e < 9; ++e) v[e] = T(0);
    }
    __device__ __forceinline__ void add(T w, const T* row)
    {
#pragma unroll
        for (int e = 0; e < 9; ++e) v[e] += w * row[e];
    }
    __device__ __forceinline__ void get(T (&o)[9]) const
    {
#pragma unroll
        for (int e = 0; e < 9; ++e) o[e] = v[e];
    }
};
template <>
struct AccQ<float> {
    float2 v2[4];
    float v8;
    __device__ __forceinline__ void zero()
    {
#pragma unroll
        for (int k = 0; k < 4; ++k) v2[k] = make_float2(0.f, 0.f);
        v8 = 0.f;
    }
    __device__ __forceinline__ void add(float w, const float* row)   // row 8-byte aligned
    {
        const float2 ww = make_float2(w, w);
        const float2* r2 = reinterpret_cast<const float2*>(row);
#pragma unroll
        for (int k = 0; k < 4; ++k) v2[k] = __ffma2_rn(ww, r2[k], v2[k]);
        v8 = fmaf(w, row[8], v8);
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

// a 3x3 block added to the stored block at dst; in FP32 as paired atomics on
// 8-byte aligned pairs (odd: dst starts on an odd float, as 117 values per
// node and 9 per block are odd), constant indices in both branches
__device__ __forceinline__ void add_block9q(float* dst, const float (&v)[9], int odd)
{
    if (odd) {
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
__device__ __forceinline__ void add_block9q(double* dst, const double (&v)[9], int)
{
#pragma unroll
    for (int e = 0; e < 9; ++e) atomicAdd(dst + e, v[e]);
}

// the q-th pair (a <= b, node index 4 y + x in the 4 x 4 union, at most two
// apart per axis)
__device__ __forceinline__ void pair_q(int q, int& a, int& b)
{
    int n = 0;
    a = b = 0;
    for (int aa = 0; aa < 16; ++aa)
        for (int bb = aa; bb < 16; ++bb) {
            const int dx = (bb & 3) - (aa & 3), dy = (bb >> 2) - (aa >> 2);
            if (dx > 2 || dx < -2 || dy > 2) continue;
            if (n == q) {
                a = aa;
                b = bb;
            }
            ++n;
        }
}

template <typename T>
__device__ __forceinline__ void flush_q_vals(T* M, int a, int b, const T (&v)[9], int i, int j, const GridP& g)
{
    const int di = (b & 3) - (a & 3), dj = (b >> 2) - (a >> 2);
    int hs = halfq(di, dj), at = a;
    if (hs < 0) {
        hs = halfq(-di, -dj);
        at = b;
    }
    const int64_t gn = (int64_t)wrap1(j - 1 + (at >> 2), g.ny) * g.nx + wrap1(i - 1 + (at & 3), g.nx);
    add_block9q(M + gn * kMBlockQ + hs * 9, v, (int)((gn + hs) & 1));
}

template <typename T>
__global__ void __launch_bounds__(32 * DepCfgQ<T>::warps, DepCfgQ<T>::min_blocks)
k_deposit_q(DepositSpecies<T> ds, const T* __restrict__ B, T* __restrict__ M, T* __restrict__ J, GridP g)
{
    // The particles of a cell are taken in four groups by the half of the
    // cell they sit in along x and y (hx, hy): a group's particles touch the
    // same 3 x 3 nodes, the union nodes (x + hx, y + hy) of the frame nodes
    // x, y = 0..2. Each lane owns frame pairs lane and lane + 32 of the 45
    // pairs of a frame and frame current component lane (of 27), sums a
    // group's particles in registers and adds the sums to the cell's union
    // accumulators in shared memory (one owner per entry and group); the
    // union sums are flushed to M and Jhat once per cell.
    constexpr int kW = DepCfgQ<T>::warps;
    constexpr int kSt = 22;   // 9 frame weights, pad, 9 c alpha at 10, 3 currents at 19
    __shared__ __align__(16) T sh[kW][32][kSt];
    __shared__ __align__(16) T um[kW][kPairsQ][9];
    __shared__ T uj[kW][48];
    __shared__ TileQ<T> stl[kW];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nwarps = (gridDim.x * blockDim.x) >> 5;
    const int nseg = (g.nx + kQX - 1) / kQX;
    const int nunits = nseg * g.ny;
    T (*st)[kSt] = sh[wib];
    T (*U)[9] = um[wib];
    T* UJ = uj[wib];
    // this lane's frame pairs (a <= b in the frame order 3 y + x)
    int fa[2] = {0, 0}, fb[2] = {0, 0};
#pragma unroll
    for (int t = 0; t < 2; ++t) {
        const int q = lane + 32 * t;
        int n = 0;
        for (int a = 0; a < 9; ++a)
            for (int b = a; b < 9; ++b) {
                if (n == q) {
                    fa[t] = a;
                    fb[t] = b;
                }
                ++n;
            }
    }
    const bool two = lane + 32 < 45;
    // their union pair index per group
    int uq[2][4];
#pragma unroll
    for (int t = 0; t < 2; ++t)
#pragma unroll
        for (int gq = 0; gq < 4; ++gq) {
            const int hx = gq & 1, hy = gq >> 1;
            const int ua = 4 * (fa[t] / 3 + hy) + fa[t] % 3 + hx, ub = 4 * (fb[t] / 3 + hy) + fb[t] % 3 + hx;
            int n = 0, found = 0;
            for (int a = 0; a < 16; ++a)
                for (int b = a; b < 16; ++b) {
                    const int dx = (b & 3) - (a & 3), dy = (b >> 2) - (a >> 2);
                    if (dx > 2 || dx < -2 || dy > 2) continue;
                    if (a == ua && b == ub) found = n;
                    ++n;
                }
            uq[t][gq] = found;
        }
    // the union pairs this lane flushes
    int pa[4], pb[4];
#pragma unroll
    for (int t = 0; t < 4; ++t) {
        const int q = lane + 32 * t;
        if (q < kPairsQ) pair_q(q, pa[t], pb[t]);
        else pa[t] = pb[t] = 0;
    }
    const bool ownj = lane < 27;
    const int jf = lane / 3, jc = lane % 3;   // frame node and component
    for (int q = lane; q < kPairsQ * 9; q += 32) (&U[0][0])[q] = T(0);
    for (int q = lane; q < 48; q += 32) UJ[q] = T(0);
    for (int u = warp; u < nunits; u += nwarps) {
        const int i0 = (u % nseg) * kQX, j = u / nseg;
        const int cn = min(kQX, g.nx - i0);
        __syncwarp();
        load_tileq<T>(stl[wib], nullptr, B, i0, cn, j, g, lane);
        for (int cl = 0; cl < cn; ++cl) {
            const int i = i0 + cl;
            const int c = j * g.nx + i;
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
                const bool act = t < total;
                int grp = -1;
                T row[kSt];
                if (act) {
                    int s = 0, p = pst[0] + t;
#pragma unroll
                    for (int q = 1; q < kMaxSpecies; ++q)
                        if (t >= cum[q] && cum[q + 1] > cum[q]) {
                            s = q;
                            p = pst[q] + (t - cum[q]);
                        }
                    const T fx = ld(ds.fx[s] + p), fy = ld(ds.fy[s] + p);
                    const T ux = ld(ds.ux[s] + p), uy = ld(ds.uy[s] + p), uz = ld(ds.uz[s] + p);
                    const T wt = ld(ds.w[s] + p);
                    const int hx = fx >= T(0.5), hy = fy >= T(0.5);
                    grp = 2 * hy + hx;
                    T wx[3], wy[3], Bp[3], al[9];
                    quad3(hx ? fx - T(1) : fx, wx);
                    quad3(hy ? fy - T(1) : fy, wy);
                    tile_Bq(stl[wib], cl, fx, fy, Bp);
                    const T gbar = sqrt(T(1) + ux * ux + uy * uy + uz * uz);
                    alphaq(Bp, ds.beta[s], gbar, al);
                    const T cM = wt * ds.cM[s] / gbar, cJ = wt * ds.cJ[s] / gbar;
#pragma unroll
                    for (int r = 0; r < 3; ++r)
#pragma unroll
                        for (int c2 = 0; c2 < 3; ++c2) row[3 * r + c2] = wy[r] * wx[c2];
                    row[9] = T(0);
#pragma unroll
                    for (int e = 0; e < 9; ++e) row[10 + e] = cM * al[e];
#pragma unroll
                    for (int r = 0; r < 3; ++r)
                        row[19 + r] = cJ * (al[3 * r] * ux + al[3 * r + 1] * uy + al[3 * r + 2] * uz);
                }
                // staging rows grouped by g (ballot prefix sums)
                unsigned bal[4];
                int gb[5];
                gb[0] = 0;
#pragma unroll
                for (int gq = 0; gq < 4; ++gq) {
                    bal[gq] = __ballot_sync(0xffffffffu, grp == gq);
                    gb[gq + 1] = gb[gq] + __popc(bal[gq]);
                }
                if (act) {
                    int r = 0;
#pragma unroll
                    for (int gq = 0; gq < 4; ++gq)
                        if (grp == gq) r = gb[gq] + __popc(bal[gq] & ((1u << lane) - 1u));
#pragma unroll
                    for (int e = 0; e < kSt; ++e) st[r][e] = row[e];
                }
                __syncwarp();
#pragma unroll
                for (int gq = 0; gq < 4; ++gq) {
                    if (gb[gq + 1] == gb[gq]) continue;   // warp-uniform
                    AccQ<T> a0, a1;
                    a0.zero();
                    a1.zero();
                    T aj = T(0);
                    for (int r = gb[gq]; r < gb[gq + 1]; ++r) {
                        const T* rw = st[r];
                        a0.add(rw[fa[0]] * rw[fb[0]], rw + 10);
                        if (two) a1.add(rw[fa[1]] * rw[fb[1]], rw + 10);
                        if (ownj) aj += rw[jf] * rw[19 + jc];
                    }
                    // into the union accumulators (distinct entries per lane)
                    T v[9];
                    a0.get(v);
#pragma unroll
                    for (int e = 0; e < 9; ++e) U[uq[0][gq]][e] += v[e];
                    if (two) {
                        a1.get(v);
#pragma unroll
                        for (int e = 0; e < 9; ++e) U[uq[1][gq]][e] += v[e];
                    }
                    if (ownj) {
                        const int hx = gq & 1, hy = gq >> 1;
                        UJ[3 * (4 * (jf / 3 + hy) + jf % 3 + hx) + jc] += aj;
                    }
                    __syncwarp();   // another lane may own these entries in the next group
                }
                __syncwarp();
            }
            // flush the cell's union sums and clear them
#pragma unroll
            for (int t2 = 0; t2 < 4; ++t2) {
                const int q = lane + 32 * t2;
                if (q < kPairsQ) {
                    T v[9];
#pragma unroll
                    for (int e = 0; e < 9; ++e) {
                        v[e] = U[q][e];
                        U[q][e] = T(0);
                    }
                    flush_q_vals(M, pa[t2], pb[t2], v, i, j, g);
                }
            }
            for (int q = lane; q < 48; q += 32) {
                const T val = UJ[q];
                UJ[q] = T(0);
                const int un = q / 3, comp = q % 3;
                const int64_t gn = (int64_t)wrap1(j - 1 + (un >> 2), g.ny) * g.nx + wrap1(i - 1 + (un & 3), g.nx);
                if (val != T(0)) atomicAdd(J + (int64_t)comp * g.ncell + gn, val);
            }
            __syncwarp();
        }
    }
}

// ---------------------------------------------------------------------------
// the operator and the field update

enum { kqA = 0, kqResidual = 1, kqArnoldi = 2 };
constexpr int kOpXq = 32, kOpYq = 8, kOpTq = kOpXq * kOpYq;
constexpr int kOpChunkq = 8;

// (curl_n curl_c v) at a node from v on its 3 x 3 neighbourhood,
// f(comp, a, b) = component comp at node (i-1+a, j-1+b)
template <typename T, typename F>
__device__ __forceinline__ void curlcurl_q(F f, T rdx2, T rdy2, T (&out)[3])
{
    T C[3][2][2];
#pragma unroll
    for (int ci = 0; ci < 2; ++ci)
#pragma unroll
        for (int cj = 0; cj < 2; ++cj) {
            T dxf[3], dyf[3];
#pragma unroll
            for (int comp = 0; comp < 3; ++comp) {
                dxf[comp] = (f(comp, ci + 1, cj) - f(comp, ci, cj) + f(comp, ci + 1, cj + 1) - f(comp, ci, cj + 1)) * rdx2;
                dyf[comp] = (f(comp, ci, cj + 1) - f(comp, ci, cj) + f(comp, ci + 1, cj + 1) - f(comp, ci + 1, cj)) * rdy2;
            }
            C[0][ci][cj] = dyf[2];
            C[1][ci][cj] = -dxf[2];
            C[2][ci][cj] = dxf[1] - dyf[0];
        }
    T dxn[3], dyn[3];
#pragma unroll
    for (int comp = 0; comp < 3; ++comp) {
        dxn[comp] = (C[comp][1][1] - C[comp][0][1] + C[comp][1][0] - C[comp][0][0]) * rdx2;
        dyn[comp] = (C[comp][1][1] - C[comp][1][0] + C[comp][0][1] - C[comp][0][0]) * rdy2;
    }
    out[0] = dyn[2];
    out[1] = -dxn[2];
    out[2] = dxn[1] - dyn[0];
}

// (M v) at node (i, j): own 13 stored blocks times v at g + d(h), the 12
// neighbours' blocks M[g - d(h)][h] times v at g - d(h); f(comp, a, b) = v
// at node (i-2+a, j-2+b); with TR each block transposed
template <typename T, bool TR, typename F>
__device__ __forceinline__ void mv_q(const T* __restrict__ M, int i, int j, const GridP& g, F f, T (&out)[3])
{
    T r[3] = {T(0), T(0), T(0)};
    const T* Mg = M + ((int64_t)j * g.nx + i) * kMBlockQ;
#pragma unroll
    for (int h = 0; h < kHalfQ; ++h) {
        int di, dj;
        halfq_offset(h, di, dj);
        const T* Mo = Mg + h * 9;
        T vv[3];
#pragma unroll
        for (int s = 0; s < 3; ++s) vv[s] = f(s, 2 + di, 2 + dj);
#pragma unroll
        for (int rr = 0; rr < 3; ++rr)
#pragma unroll
            for (int s = 0; s < 3; ++s) r[rr] += ld(Mo + (TR ? s * 3 + rr : rr * 3 + s)) * vv[s];
        if (h == 0) continue;
        const T* Mn = M + ((int64_t)wrap1(j - dj, g.ny) * g.nx + wrap1(i - di, g.nx)) * kMBlockQ + h * 9;
#pragma unroll
        for (int s = 0; s < 3; ++s) vv[s] = f(s, 2 - di, 2 - dj);
#pragma unroll
        for (int rr = 0; rr < 3; ++rr)
#pragma unroll
            for (int s = 0; s < 3; ++s) r[rr] += ld(Mn + (TR ? s * 3 + rr : rr * 3 + s)) * vv[s];
    }
    out[0] = r[0];
    out[1] = r[1];
    out[2] = r[2];
}

template <typename T, int MODE, bool TR>
__global__ void __launch_bounds__(kOpTq)
k_op_q(const T* __restrict__ M, const double* __restrict__ in, double s, const double* __restrict__ b,
       double* __restrict__ out, double* __restrict__ vj, const double* __restrict__ V, int64_t ldv, int nv, GridP g,
       double* __restrict__ partial, const GmDyn* __restrict__ dyn)
{
    if (MODE == kqArnoldi && dyn) {
        if (!dyn->live) return;
        in = dyn->in;
        s = dyn->s;
        vj = dyn->vj;
        out = dyn->out;
        nv = dyn->nv;
    }
    constexpr int HX = kOpXq + 4, HY = kOpYq + 4;
    __shared__ T sv[3][HY][HX];
    __shared__ double buf[kOpChunkq][kOpTq];
    const int nx = g.nx, ny = g.ny;
    const int64_t nc = g.ncell;
    const int tx_n = (nx + kOpXq - 1) / kOpXq;
    const int i0 = (blockIdx.x % tx_n) * kOpXq, j0 = (blockIdx.x / tx_n) * kOpYq;
    const int tid = threadIdx.x, tx = tid % kOpXq, ty = tid / kOpXq;
    const int i = i0 + tx, j = j0 + ty;
    const bool active = i < nx && j < ny;
    const int64_t gidx = active ? (int64_t)j * nx + i : 0;
    const T sT = (T)s;
    for (int q = tid; q < 3 * HY * HX; q += kOpTq) {
        const int comp = q / (HY * HX), rem = q % (HY * HX), yy = rem / HX, xx = rem % HX;
        // positions past the tile's last used column/row are clamped (unused)
        const int gi = wrap1(min(i0 - 2 + xx, 2 * nx - 1), nx), gj = wrap1(min(j0 - 2 + yy, 2 * ny - 1), ny);
        T val = (T)__ldg(in + comp * nc + (int64_t)gj * nx + gi);
        if (MODE == kqArnoldi) val *= sT;
        sv[comp][yy][xx] = val;
    }
    __syncthreads();
    double own[3] = {0.0, 0.0, 0.0}, wv[3] = {0.0, 0.0, 0.0};
    if (active) {
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            own[c] = __ldg(in + c * nc + gidx);
            if (MODE == kqArnoldi && !is_one(s)) own[c] *= s;
        }
        auto f1 = [&](int comp, int a, int bb) -> T { return sv[comp][ty + 1 + bb][tx + 1 + a]; };
        auto f2 = [&](int comp, int a, int bb) -> T { return sv[comp][ty + bb][tx + a]; };
        T cc[3], mv[3];
        curlcurl_q<T>(f1, gc<T>(g).hdx, gc<T>(g).hdy, cc);
        mv_q<T, TR>(M, i, j, g, f2, mv);
        const T td = gc<T>(g).td;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const double bv = (double)(td * td * cc[c] + td * mv[c]);
            if (MODE == kqA) wv[c] = own[c] + bv;
            else if (MODE == kqResidual) wv[c] = b[c * nc + gidx] - (own[c] + bv);
            else wv[c] = bv;
            out[c * nc + gidx] = wv[c];
            if (MODE == kqArnoldi && vj) vj[c * nc + gidx] = own[c];
        }
    }
    if (MODE == kqA) return;
    const int nq = MODE == kqResidual ? 1 : nv + 2;
    const int lane = tid & 31, wid = tid >> 5;
    for (int q0 = 0; q0 < nq; q0 += kOpChunkq) {
        const int kc = min(kOpChunkq, nq - q0);
        for (int c = 0; c < kc; ++c) {
            const int q = q0 + c;
            double d = 0.0;
            if (active) {
                if (MODE == kqResidual || q == nv + 1) d = wv[0] * wv[0] + wv[1] * wv[1] + wv[2] * wv[2];
                else if (q == nv) d = wv[0] * own[0] + wv[1] * own[1] + wv[2] * own[2];
                else {
                    const double* Vq = V + (int64_t)q * ldv + gidx;
                    d = wv[0] * __ldg(Vq) + wv[1] * __ldg(Vq + nc) + wv[2] * __ldg(Vq + 2 * nc);
                }
            }
            buf[c][tid] = d;
        }
        __syncthreads();
        for (int c = wid; c < kc; c += kOpTq / 32) {
            double t = 0.0;
#pragma unroll
            for (int mm = 0; mm < kOpTq / 32; ++mm) t += buf[c][mm * 32 + lane];
            t = warp_sum(t);
            if (lane == 0) partial[(int64_t)blockIdx.x * nq + q0 + c] = t;
        }
        __syncthreads();
    }
}

constexpr int kFieldLedgerQ = 6;

// E^{n+theta} -> Eth, E^{n+1}, B^{n+1} of cell (i, j) and the ledger terms
// 0..4 of the 2D field update; term 5 (the work) by k_work_q
template <typename T>
__global__ void __launch_bounds__(256)
k_field_update_q(const double* __restrict__ x, T* __restrict__ Eth, T* __restrict__ E, const T* __restrict__ B0,
                 T* __restrict__ B1, GridP g, double* __restrict__ partial)
{
    __shared__ double red[32 * 5];
    const int64_t nc = g.ncell;
    const int64_t gidx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    T acc[5] = {T(0), T(0), T(0), T(0), T(0)};
    if (gidx < nc) {
        const int i = (int)(gidx % g.nx), j = (int)(gidx / g.nx);
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
        const int i1 = wrap1(i + 1, g.nx), j1 = wrap1(j + 1, g.ny);
        const int64_t n00 = (int64_t)j * g.nx + i, n10 = (int64_t)j * g.nx + i1;
        const int64_t n01 = (int64_t)j1 * g.nx + i, n11 = (int64_t)j1 * g.nx + i1;
        const T idx2 = gc<T>(g).hdx, idy2 = gc<T>(g).hdy;
        T dxE[3], dyE[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const T a = (T)x[c * nc + n00], bq = (T)x[c * nc + n10], cq = (T)x[c * nc + n01], d = (T)x[c * nc + n11];
            dxE[c] = (bq - a + d - cq) * idx2;
            dyE[c] = (cq - a + d - bq) * idy2;
        }
        const T curl[3] = {dyE[2], -dxE[2], dxE[1] - dyE[0]};
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
        for (int q = 0; q < 5; ++q) partial[(int64_t)blockIdx.x * kFieldLedgerQ + q] = o[q];
}

template <typename T>
__global__ void __launch_bounds__(256)
k_work_q(const T* __restrict__ M, const T* __restrict__ J, const T* __restrict__ Eth, GridP g,
         double* __restrict__ partial)
{
    __shared__ double red[32];
    const int64_t nc = g.ncell;
    const int64_t gidx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    T wk = T(0);
    if (gidx < nc) {
        const int i = (int)(gidx % g.nx), j = (int)(gidx / g.nx);
        auto f = [&](int comp, int a, int b) -> T {
            return ld(Eth + comp * nc + (int64_t)wrap1(j - 2 + b, g.ny) * g.nx + wrap1(i - 2 + a, g.nx));
        };
        T mv[3];
        mv_q<T, false>(M, i, j, g, f, mv);
#pragma unroll
        for (int c = 0; c < 3; ++c) wk += (J[c * nc + gidx] + mv[c]) * Eth[c * nc + gidx];
        wk *= gc<T>(g).dtdV;
    }
    double v[1] = {(double)wk}, o[1];
    block_sum<1>(v, red, o);
    if (threadIdx.x == 0) partial[(int64_t)blockIdx.x * kFieldLedgerQ + 5] = o[0];
}

// ---------------------------------------------------------------------------
// push

constexpr int kPushWarpsQ = 4;

template <typename T>
__global__ void __launch_bounds__(32 * kPushWarpsQ)
k_push_q(PArrays<T> src, PArrays<T> dst, const int32_t* __restrict__ start, int32_t* __restrict__ key,
         int32_t* __restrict__ rank, int32_t* __restrict__ count, const T* __restrict__ Eth, const T* __restrict__ B,
         GridP g, T beta, T qdt, T m, double* __restrict__ lsum)
{
    __shared__ int sst[kPushWarpsQ][kQX + 1];
    __shared__ TileQ<T> stl[kPushWarpsQ];
    __shared__ double red[32 * 4];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nwarps = (gridDim.x * blockDim.x) >> 5;
    const int nseg = (g.nx + kQX - 1) / kQX;
    const int nunits = nseg * g.ny;
    int* ss = sst[wib];
    const T dt = gc<T>(g).dt, rdx = gc<T>(g).rdx, rdy = gc<T>(g).rdy;
    T acc[4] = {T(0), T(0), T(0), T(0)};
    for (int u = warp; u < nunits; u += nwarps) {
        const int i0 = (u % nseg) * kQX, j = u / nseg;
        const int cn = min(kQX, g.nx - i0);
        const int c0 = j * g.nx + i0;
        __syncwarp();
        if (lane <= cn) ss[lane] = start[c0 + lane];
        if (lane == 0 && cn == kQX) ss[kQX] = start[c0 + kQX];
        load_tileq<T>(stl[wib], Eth, B, i0, cn, j, g, lane);
        const TileQ<T>& tl = stl[wib];
        const int P0 = ss[0], P1 = ss[cn];
        int cl = 0;
        for (int p0 = P0; p0 < P1; p0 += 32) {
            const int p = p0 + lane;
            const bool act = p < P1;
            int newkey = -1 - lane;
            if (act) {
                while (ss[cl + 1] <= p) ++cl;
                const int i = i0 + cl;
                const T fx = ld(src.fx + p), fy = ld(src.fy + p);
                const T ux = ld(src.ux + p), uy = ld(src.uy + p), uz = ld(src.uz + p), w = ld(src.w + p);
                T wx[4], wy[4];
                node4(fx, wx);
                node4(fy, wy);
                T E[3];
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    T e = T(0);
#pragma unroll
                    for (int r = 0; r < 4; ++r)
#pragma unroll
                        for (int cc = 0; cc < 4; ++cc) e += wy[r] * wx[cc] * tl.E[c][r][cl + cc];
                    E[c] = e;
                }
                T Bp[3];
                tile_Bq(tl, cl, fx, fy, Bp);
                const T u02 = ux * ux + uy * uy + uz * uz;
                const T g0 = sqrt(T(1) + u02);
                const T ax = beta * Bp[0] / g0, ay = beta * Bp[1] / g0, az = beta * Bp[2] / g0;
                const T sa = T(1) / (T(1) + ax * ax + ay * ay + az * az);
                const T wxv = ux + beta * E[0], wyv = uy + beta * E[1], wzv = uz + beta * E[2];
                const T wa = wxv * ax + wyv * ay + wzv * az;
                const T ubx = sa * (wxv + (wyv * az - wzv * ay) + wa * ax);
                const T uby = sa * (wyv + (wzv * ax - wxv * az) + wa * ay);
                const T ubz = sa * (wzv + (wxv * ay - wyv * ax) + wa * az);
                const T u1x = T(2) * ubx - ux, u1y = T(2) * uby - uy, u1z = T(2) * ubz - uz;
                const T u12 = u1x * u1x + u1y * u1y + u1z * u1z;
                const T g1 = sqrt(T(1) + u12);
                const T t[2] = {fx + dt * rdx * (u1x / g1), fy + dt * rdy * (u1y / g1)};
                const int nn[2] = {g.nx, g.ny}, cc0[2] = {i, j};
                T fn[2];
                int cnew[2];
#pragma unroll
                for (int a = 0; a < 2; ++a) {
                    const T fl = floor(t[a]);
                    int sh = (int)fl;
                    T f = t[a] - fl;
                    if (f >= T(1)) { f -= T(1); sh += 1; }
                    fn[a] = f;
                    int q = (cc0[a] + sh) % nn[a];
                    if (q < 0) q += nn[a];
                    cnew[a] = q;
                }
                dst.fx[p] = fn[0];
                dst.fy[p] = fn[1];
                dst.ux[p] = u1x;
                dst.uy[p] = u1y;
                dst.uz[p] = u1z;
                dst.w[p] = w;
                if (dst.id) dst.id[p] = src.id[p];
                newkey = cnew[1] * g.nx + cnew[0];
                key[p] = newkey;
                const T ue = ubx * E[0] + uby * E[1] + ubz * E[2];
                const T du = (ux - u1x) * (ux + u1x) + (uy - u1y) * (uy + u1y) + (uz - u1z) * (uz + u1z);
                const T igs = T(1) / (g0 + g1);
                acc[0] -= w * m * du * igs;
                acc[1] += qdt * w * ue / g0;
                acc[2] += qdt * w * ue * du * igs * igs / g0;
                acc[3] += w * m * u12 / (g1 + T(1));
            }
            const unsigned peers = __match_any_sync(0xffffffffu, newkey);
            const int leader = __ffs(peers) - 1;
            int base = 0;
            if (act && lane == leader) base = atomicAdd(count + newkey, __popc(peers));
            base = __shfl_sync(0xffffffffu, base, leader);
            if (act) rank[p] = base + __popc(peers & ((1u << lane) - 1u));
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

}  // namespace

template <typename T>
cudaError_t deposit_q(const DepositSpecies<T>& ds, const T* B, T* M, T* J, GridP g, cudaStream_t st, int blocks)
{
    const int units = ((g.nx + kQX - 1) / kQX) * g.ny;
    count_launches(1);
    k_deposit_q<T><<<gridq(units, DepCfgQ<T>::warps, blocks > 0 ? blocks : 152 * 8), 32 * DepCfgQ<T>::warps, 0, st>>>(
        ds, B, M, J, g);
    return cudaGetLastError();
}

int op_blocks_q(GridP g) { return ((g.nx + kOpXq - 1) / kOpXq) * ((g.ny + kOpYq - 1) / kOpYq); }

template <typename T, int MODE, bool TR>
cudaError_t launch_op_q(const T* M, const double* in, double sc, const double* b, double* out, double* vj,
                        const double* V, int64_t ldv, int nv, GridP g, double* partial, cudaStream_t st,
                        const GmDyn* dyn)
{
    count_launches(1);
    k_op_q<T, MODE, TR><<<op_blocks_q(g), kOpTq, 0, st>>>(M, in, sc, b, out, vj, V, ldv, nv, g, partial, dyn);
    return cudaGetLastError();
}

template <typename T>
cudaError_t field_update_q(const double* x, const T* M, const T* J, T* Eth, T* E, const T* B0, T* B1, GridP g,
                           double* partial, int nblocks, cudaStream_t st)
{
    count_launches(2);
    k_field_update_q<T><<<nblocks, 256, 0, st>>>(x, Eth, E, B0, B1, g, partial);
    k_work_q<T><<<nblocks, 256, 0, st>>>(M, J, Eth, g, partial);
    return cudaGetLastError();
}

int push_blocks_q(GridP g, int cap)
{
    const int64_t units = (int64_t)((g.nx + kQX - 1) / kQX) * g.ny;
    return (int)gridq(units, kPushWarpsQ, cap > 0 ? cap : 152 * 16);
}

template <typename T>
cudaError_t push_q(PArrays<T> src, PArrays<T> dst, const int32_t* start, int32_t* key, int32_t* rank,
                   int32_t* count, const T* Eth, const T* B, GridP g, SpeciesConst sc, double* lsum, int nblocks,
                   cudaStream_t st)
{
    count_launches(1);
    k_push_q<T><<<nblocks, 32 * kPushWarpsQ, 0, st>>>(src, dst, start, key, rank, count, Eth, B, g,
                                                        (T)(sc.q * g.dt / (2.0 * sc.m)), (T)(sc.q * g.dt), (T)sc.m,
                                                        lsum);
    return cudaGetLastError();
}

#define RELSIM_Q_OP(T, MODE, TR)                                                                                  \
    template cudaError_t launch_op_q<T, MODE, TR>(const T*, const double*, double, const double*, double*,        \
                                                  double*, const double*, int64_t, int, GridP, double*,           \
                                                  cudaStream_t, const GmDyn*);
#define RELSIM_Q_INSTANTIATE(T)                                                                                   \
    template cudaError_t deposit_q<T>(const DepositSpecies<T>&, const T*, T*, T*, GridP, cudaStream_t, int);           \
    template cudaError_t field_update_q<T>(const double*, const T*, const T*, T*, T*, const T*, T*, GridP,        \
                                           double*, int, cudaStream_t);                                           \
    template cudaError_t push_q<T>(PArrays<T>, PArrays<T>, const int32_t*, int32_t*, int32_t*, int32_t*,         \
                                   const T*, const T*, GridP, SpeciesConst, double*, int, cudaStream_t);          \
    RELSIM_Q_OP(T, 0, false) RELSIM_Q_OP(T, 1, false) RELSIM_Q_OP(T, 2, false)                                   \
    RELSIM_Q_OP(T, 0, true) RELSIM_Q_OP(T, 1, true) RELSIM_Q_OP(T, 2, true)

RELSIM_Q_INSTANTIATE(float)
RELSIM_Q_INSTANTIATE(double)

}  // namespace relsim
