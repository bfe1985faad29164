// particles.cu -- particle kernels: load conversion, gather/export, the
// mass-matrix and predicted-current deposit, and the explicit push with the
// cell re-sort.
//
// Particles of a species are stored sorted by cell (SoA, offsets fx, fy in
// [0,1) within the cell, momenta u = gamma v, weight w). Cell c owns the
// index range [start[c], start[c+1]).
#include "launch.cuh"

namespace relsim {

namespace {

// ---------------------------------------------------------------------------
// load: absolute FP64 positions -> (cell key, offsets), FP64 -> T

template <typename T>
__global__ void k_load_convert(const double* __restrict__ x, const double* __restrict__ u,
                               const double* __restrict__ w, int64_t n, GridP g, PArrays<T> out,
                               int32_t* key, int32_t* val, int* bad)
{
    int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (; p < n; p += stride) {
        double xs = x[2 * p] / g.dx, ys = x[2 * p + 1] / g.dy;
        double ux = u[3 * p], uy = u[3 * p + 1], uz = u[3 * p + 2], ww = w[p];
        if (!isfinite(xs) || !isfinite(ys) || !isfinite(ux) || !isfinite(uy) || !isfinite(uz) ||
            !isfinite(ww)) {
            atomicOr(bad, 1);
            xs = ys = 0.0;
        }
        // periodic wrap into [0, n) then split into cell + offset
        xs -= g.nx * floor(xs / g.nx);
        ys -= g.ny * floor(ys / g.ny);
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

// B^n at the particle from the cell-centre lattice. The centre lattice
// coordinate is i + fx - 1/2: the two centres are (i-1, i) when fx < 1/2 and
// (i, i+1) otherwise.
template <typename T>
__device__ __forceinline__ void gather_B(const T* __restrict__ B, int nc, int nx, int i, int im,
                                         int ip, int jr, int jmr, int jpr, T fx, T fy, T& Bx, T& By,
                                         T& Bz)
{
    // jr, jmr, jpr are row offsets j*nx, (j-1)*nx, (j+1)*nx (wrapped)
    const bool lx = fx < T(0.5), ly = fy < T(0.5);
    const T tx = lx ? fx + T(0.5) : fx - T(0.5);
    const T ty = ly ? fy + T(0.5) : fy - T(0.5);
    const int c0x = lx ? im : i, c1x = lx ? i : ip;
    const int r0 = ly ? jmr : jr, r1 = ly ? jr : jpr;
    const T w00 = (T(1) - tx) * (T(1) - ty), w10 = tx * (T(1) - ty);
    const T w01 = (T(1) - tx) * ty, w11 = tx * ty;
    const int a = r0 + c0x, b = r0 + c1x, c = r1 + c0x, d = r1 + c1x;
    Bx = w00 * ld(B + a) + w10 * ld(B + b) + w01 * ld(B + c) + w11 * ld(B + d);
    By = w00 * ld(B + nc + a) + w10 * ld(B + nc + b) + w01 * ld(B + nc + c) + w11 * ld(B + nc + d);
    Bz = w00 * ld(B + 2 * nc + a) + w10 * ld(B + 2 * nc + b) + w01 * ld(B + 2 * nc + c) +
         w11 * ld(B + 2 * nc + d);
}

// ---------------------------------------------------------------------------
// deposit: G lanes per cell accumulate 81 mass-matrix moments and 12 current
// values in registers, reduce across the group, then flush with atomics.
//
// Moments: S[k][e] = sum_p c_p XX_xx YY_yy alpha'_e with k = xx*3 + yy,
// XX = ((1-fx)^2, (1-fx) fx, fx^2), YY likewise in y, alpha' = alpha (1+|a|^2)
// and c_p = w q beta /(gbar dV (1+|a|^2)). The ten node pairs of a cell take
// nine distinct weight products; (n00,n11) and (n10,n01) share k = 4.

template <typename T, int G>
__global__ void __launch_bounds__(256)
k_deposit(DepositSpecies<T> sp, const T* __restrict__ B, T* __restrict__ M, T* __restrict__ J,
          GridP g)
{
    constexpr int GPW = 32 / G;   // groups per warp
    const int lane = threadIdx.x & 31;
    const int gl = lane % G;      // lane within group
    const int gw = lane / G;      // group within warp
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nwarps = (gridDim.x * blockDim.x) >> 5;
    const int nx = g.nx, ny = g.ny, nc = g.ncell;

    for (int cb = warp * GPW; cb < nc; cb += nwarps * GPW) {
        const int c = cb + gw;
        const bool valid = c < nc;
        T S[81];
        T Jm[12];
#pragma unroll
        for (int k = 0; k < 81; ++k) S[k] = T(0);
#pragma unroll
        for (int k = 0; k < 12; ++k) Jm[k] = T(0);
        int i = 0, j = 0;
        if (valid) {
            i = c % nx;
            j = c / nx;
            const int im = wrap1(i - 1, nx), ip = wrap1(i + 1, nx);
            const int jr = j * nx, jmr = wrap1(j - 1, ny) * nx, jpr = wrap1(j + 1, ny) * nx;
            for (int s = 0; s < sp.nsp; ++s) {
                const int p0 = sp.start[s][c], p1 = sp.start[s][c + 1];
                const T beta = sp.beta[s], cJ = sp.cJ[s], cM = sp.cM[s];
                const T* __restrict__ pfx = sp.fx[s];
                const T* __restrict__ pfy = sp.fy[s];
                const T* __restrict__ pux = sp.ux[s];
                const T* __restrict__ puy = sp.uy[s];
                const T* __restrict__ puz = sp.uz[s];
                const T* __restrict__ pw = sp.w[s];
                for (int p = p0 + gl; p < p1; p += G) {
                    const T fx = ld(pfx + p), fy = ld(pfy + p);
                    const T ux = ld(pux + p), uy = ld(puy + p), uz = ld(puz + p);
                    const T w = ld(pw + p);
                    T Bx, By, Bz;
                    gather_B(B, nc, nx, i, im, ip, jr, jmr, jpr, fx, fy, Bx, By, Bz);
                    const T u2 = ux * ux + uy * uy + uz * uz;
                    const T ig = T(1) / sqrt(T(1) + u2);
                    const T bg = beta * ig;
                    const T ax = bg * Bx, ay = bg * By, az = bg * Bz;
                    const T sa = T(1) / (T(1) + ax * ax + ay * ay + az * az);
                    T e[9];
                    e[0] = T(1) + ax * ax; e[1] = ax * ay + az;   e[2] = ax * az - ay;
                    e[3] = ax * ay - az;   e[4] = T(1) + ay * ay; e[5] = ay * az + ax;
                    e[6] = ax * az + ay;   e[7] = ay * az - ax;   e[8] = T(1) + az * az;
                    // predicted current: w q alpha u / gbar / dV at the 4 nodes
                    const T cj = w * cJ * sa * ig;
                    const T vx = cj * (e[0] * ux + e[1] * uy + e[2] * uz);
                    const T vy = cj * (e[3] * ux + e[4] * uy + e[5] * uz);
                    const T vz = cj * (e[6] * ux + e[7] * uy + e[8] * uz);
                    const T X0 = T(1) - fx, X1 = fx, Y0 = T(1) - fy, Y1 = fy;
                    const T W[4] = {X0 * Y0, X1 * Y0, X0 * Y1, X1 * Y1};
#pragma unroll
                    for (int a = 0; a < 4; ++a) {
                        Jm[a * 3 + 0] += W[a] * vx;
                        Jm[a * 3 + 1] += W[a] * vy;
                        Jm[a * 3 + 2] += W[a] * vz;
                    }
                    const T cm = w * cM * sa * ig;
                    const T xx[3] = {cm * X0 * X0, cm * X0 * X1, cm * X1 * X1};
                    const T yy[3] = {Y0 * Y0, Y0 * Y1, Y1 * Y1};
#pragma unroll
                    for (int a = 0; a < 3; ++a)
#pragma unroll
                        for (int b = 0; b < 3; ++b) {
                            const T t = xx[a] * yy[b];
#pragma unroll
                            for (int q = 0; q < 9; ++q) S[(a * 3 + b) * 9 + q] += t * e[q];
                        }
                }
            }
        }
        // reduce across the G lanes of the group
        if (G > 1) {
#pragma unroll
            for (int o = G / 2; o >= 1; o >>= 1) {
#pragma unroll
                for (int k = 0; k < 81; ++k) S[k] += __shfl_xor_sync(0xffffffffu, S[k], o);
#pragma unroll
                for (int k = 0; k < 12; ++k) Jm[k] += __shfl_xor_sync(0xffffffffu, Jm[k], o);
            }
        }
        if (!valid) continue;
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
                atomicAdd(M + (int64_t)pn[pr] * kMBlock + po[pr] * 9 + q, S[pk[pr] * 9 + q]);
            }
        }
        const int jn[4] = {n00, n10, n01, n11};
#pragma unroll
        for (int it = 0; it < 12; ++it) {
            if ((90 + it) % G == gl) atomicAdd(J + (int64_t)(it % 3) * nc + jn[it / 3], Jm[it]);
        }
    }
}

// ---------------------------------------------------------------------------
// push. One warp per (cell, species); the lanes walk the cell's particles in
// order, so ranks within a (cell, direction) group follow the old order.

constexpr int kPushThreads = 256;
constexpr int kLedger = 5;   // K0, dK, work, mismatch, K1

template <typename T>
__global__ void __launch_bounds__(kPushThreads)
k_push(int phase, PArrays<T> src, PArrays<T> dst, const int32_t* __restrict__ start,
       int32_t* __restrict__ n9, const int32_t* __restrict__ off9, int32_t* __restrict__ key,
       const T* __restrict__ Eth, const T* __restrict__ B, GridP g, T beta, T dt_dx, T dt_dy,
       T qw_dt, T m, double* __restrict__ lsum, int npart, int* __restrict__ err)
{
    __shared__ int rankbase[kPushThreads / 32][kNDir];
    __shared__ double red[32 * kLedger];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nwarps = (gridDim.x * blockDim.x) >> 5;
    const int nx = g.nx, ny = g.ny, nc = g.ncell;
    const unsigned lt = (1u << lane) - 1u;
    T acc[kLedger] = {T(0), T(0), T(0), T(0), T(0)};

    for (int c = warp; c < nc; c += nwarps) {
        const int i = c % nx, j = c / nx;
        const int im = wrap1(i - 1, nx), ip = wrap1(i + 1, nx);
        const int jr = j * nx, jmr = wrap1(j - 1, ny) * nx, jpr = wrap1(j + 1, ny) * nx;
        // E^{n+theta} at the four nodes of the cell
        const int n00 = jr + i, n10 = jr + ip, n01 = jpr + i, n11 = jpr + ip;
        T En[3][4];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            En[k][0] = ld(Eth + k * nc + n00);
            En[k][1] = ld(Eth + k * nc + n10);
            En[k][2] = ld(Eth + k * nc + n01);
            En[k][3] = ld(Eth + k * nc + n11);
        }
        const int p0 = start[c], p1 = start[c + 1];
        int cnt[kNDir];
#pragma unroll
        for (int d = 0; d < kNDir; ++d) cnt[d] = 0;
        if (phase != 0) {
            if (lane < kNDir) rankbase[wib][lane] = 0;
            __syncwarp();
        }
        for (int base = p0; base < p1; base += 32) {
            const int p = base + lane;
            const bool act = p < p1;
            int dir = kNDir;   // inactive lanes use a direction no active lane has
            T fxn = T(0), fyn = T(0), u1x = T(0), u1y = T(0), u1z = T(0), w = T(0);
            int sx = 0, sy = 0;
            if (act) {
                const T fx = src.fx[p], fy = src.fy[p];
                const T ux = src.ux[p], uy = src.uy[p], uz = src.uz[p];
                w = src.w[p];
                T Bx, By, Bz;
                gather_B(B, nc, nx, i, im, ip, jr, jmr, jpr, fx, fy, Bx, By, Bz);
                const T X0 = T(1) - fx, Y0 = T(1) - fy;
                const T W0 = X0 * Y0, W1 = fx * Y0, W2 = X0 * fy, W3 = fx * fy;
                const T Ex = W0 * En[0][0] + W1 * En[0][1] + W2 * En[0][2] + W3 * En[0][3];
                const T Ey = W0 * En[1][0] + W1 * En[1][1] + W2 * En[1][2] + W3 * En[1][3];
                const T Ez = W0 * En[2][0] + W1 * En[2][1] + W2 * En[2][2] + W3 * En[2][3];
                const T u02 = ux * ux + uy * uy + uz * uz;
                const T g0 = sqrt(T(1) + u02);
                const T bg = beta / g0;
                const T ax = bg * Bx, ay = bg * By, az = bg * Bz;
                const T sa = T(1) / (T(1) + ax * ax + ay * ay + az * az);
                // ubar = alpha w = (w + w x a + (w.a) a)/(1 + |a|^2), w = u + beta E
                const T wx = ux + beta * Ex, wy = uy + beta * Ey, wz = uz + beta * Ez;
                const T wa = wx * ax + wy * ay + wz * az;
                const T ubx = sa * (wx + (wy * az - wz * ay) + wa * ax);
                const T uby = sa * (wy + (wz * ax - wx * az) + wa * ay);
                const T ubz = sa * (wz + (wx * ay - wy * ax) + wa * az);
                u1x = T(2) * ubx - ux;
                u1y = T(2) * uby - uy;
                u1z = T(2) * ubz - uz;
                const T u12 = u1x * u1x + u1y * u1y + u1z * u1z;
                const T g1 = sqrt(T(1) + u12);
                const T ig1 = T(1) / g1;
                // position: x^{n+3/2} = x^{n+1/2} + dt u^{n+1}/gamma^{n+1}
                T tx = fx + dt_dx * (u1x * ig1);
                T ty = fy + dt_dy * (u1y * ig1);
                T flx = floor(tx), fly = floor(ty);
                sx = (int)flx;
                sy = (int)fly;
                fxn = tx - flx;
                fyn = ty - fly;
                if (fxn >= T(1)) { fxn -= T(1); sx += 1; }
                if (fyn >= T(1)) { fyn -= T(1); sy += 1; }
                if (phase != 2) {
                    // with c dt <= dx a move of more than one cell can only come
                    // from rounding at |v| = c; keep the particle on the last
                    // representable point of the neighbour cell
                    if (sx > 1) { sx = 1; fxn = Consts<T>::one_below(); }
                    if (sx < -1) { sx = -1; fxn = T(0); }
                    if (sy > 1) { sy = 1; fyn = Consts<T>::one_below(); }
                    if (sy < -1) { sy = -1; fyn = T(0); }
                    dir = (sy + 1) * 3 + (sx + 1);
                } else {
                    dir = 0;
                }
                if (phase == 0) {
                    const T ue = ubx * Ex + uby * Ey + ubz * Ez;
                    // g0 - g1 = (u0 - u1).(u0 + u1)/(g0 + g1)
                    const T du = (ux - u1x) * (ux + u1x) + (uy - u1y) * (uy + u1y) +
                                 (uz - u1z) * (uz + u1z);
                    const T gs = g0 + g1;
                    acc[0] += w * m * (u02 / (g0 + T(1)));      // K0
                    acc[1] += -w * m * (du / gs);               // dK
                    acc[2] += qw_dt * w * ue / g0;              // work (qw_dt = q dt)
                    acc[3] += qw_dt * w * ue * (du / gs) / (g0 * gs);   // mismatch
                    acc[4] += w * m * (u12 / (g1 + T(1)));      // K1
                }
            }
            if (phase == 0) {
#pragma unroll
                for (int d = 0; d < kNDir; ++d) cnt[d] += __popc(__ballot_sync(0xffffffffu, dir == d));
            } else {
                const unsigned peers = __match_any_sync(0xffffffffu, dir);
                const int rk = __popc(peers & lt);
                int rb = 0;
                if (act) rb = rankbase[wib][dir];
                __syncwarp();
                if (act && rk == 0) rankbase[wib][dir] = rb + __popc(peers);
                __syncwarp();
                if (act) {
                    int ni, nj;
                    if (phase == 1) {
                        ni = wrap1(i + sx, nx);
                        nj = wrap1(j + sy, ny);
                    } else {
                        ni = (i + sx) % nx;
                        nj = (j + sy) % ny;
                        if (ni < 0) ni += nx;
                        if (nj < 0) nj += ny;
                    }
                    const int k = nj * nx + ni;
                    if (phase == 1) {
                        const int dpos = off9[(int64_t)k * kNDir + dir] + rb + rk;
                        // the count pass and this pass must agree move by move;
                        // if they ever did not, flag it instead of writing
                        if (rb + rk >= n9[(int64_t)c * kNDir + dir] || dpos < 0 || dpos >= npart) {
                            atomicOr(err, 1);
                            continue;
                        }
                        dst.fx[dpos] = fxn;
                        dst.fy[dpos] = fyn;
                        dst.ux[dpos] = u1x;
                        dst.uy[dpos] = u1y;
                        dst.uz[dpos] = u1z;
                        dst.w[dpos] = w;
                        if (dst.id) dst.id[dpos] = src.id[p];
                    } else {
                        dst.fx[p] = fxn;
                        dst.fy[p] = fyn;
                        dst.ux[p] = u1x;
                        dst.uy[p] = u1y;
                        dst.uz[p] = u1z;
                        dst.w[p] = w;
                        if (dst.id) dst.id[p] = src.id[p];
                        key[p] = k;
                    }
                }
            }
        }
        if (phase == 0 && lane < kNDir) {
            int v = 0;
#pragma unroll
            for (int d = 0; d < kNDir; ++d) v = lane == d ? cnt[d] : v;
            n9[(int64_t)c * kNDir + lane] = v;
        }
    }
    if (phase == 0) {
        double v[kLedger], out[kLedger];
#pragma unroll
        for (int s = 0; s < kLedger; ++s) v[s] = (double)acc[s];
        block_sum<kLedger>(v, red, out);
        if (threadIdx.x == 0)
#pragma unroll
            for (int s = 0; s < kLedger; ++s) lsum[(int64_t)blockIdx.x * kLedger + s] = out[s];
    }
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

int blocks_for(int64_t n, int threads, int cap)
{
    int64_t b = (n + threads - 1) / threads;
    if (b < 1) b = 1;
    if (b > cap) b = cap;
    return (int)b;
}

}  // namespace

int push_grid_blocks() { return 152 * 8; }

template <typename T>
cudaError_t load_convert(const double* x, const double* u, const double* w, int64_t n, GridP g,
                         PArrays<T> out, int32_t* key, int32_t* val, int* bad, cudaStream_t st)
{
    if (n <= 0) return cudaSuccess;
    count_launches(1);
    k_load_convert<T><<<blocks_for(n, 256, 152 * 32), 256, 0, st>>>(x, u, w, n, g, out, key, val, bad);
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
cudaError_t deposit(const DepositSpecies<T>& sp, const T* B, T* M, T* J, GridP g, cudaStream_t st)
{
    constexpr int G = 8;
    const int threads = 256;
    int64_t groups = g.ncell;
    int blocks = blocks_for(groups * G, threads, 152 * 16);
    count_launches(1);
    k_deposit<T, G><<<blocks, threads, 0, st>>>(sp, B, M, J, g);
    return cudaGetLastError();
}

template <typename T>
cudaError_t push(int phase, PArrays<T> src, PArrays<T> dst, const int32_t* start, int32_t* n9,
                 const int32_t* off9, int32_t* key, const T* Eth, const T* B, GridP g,
                 SpeciesConst sc, double* lsum_partial, int lsum_blocks, int64_t npart, int* err,
                 cudaStream_t st)
{
    const T beta = (T)(sc.q * g.dt / (2.0 * sc.m));
    count_launches(1);
    k_push<T><<<lsum_blocks, kPushThreads, 0, st>>>(phase, src, dst, start, n9, off9, key, Eth, B, g,
                                                    beta, (T)(g.dt / g.dx), (T)(g.dt / g.dy),
                                                    (T)(sc.q * g.dt), (T)sc.m, lsum_partial,
                                                    (int)npart, err);
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

#define RELSIM_INSTANTIATE(T)                                                                      \
    template cudaError_t load_convert<T>(const double*, const double*, const double*, int64_t,     \
                                         GridP, PArrays<T>, int32_t*, int32_t*, int*, cudaStream_t); \
    template cudaError_t gather_particles<T>(const int32_t*, PArrays<T>, PArrays<T>, int64_t, bool, \
                                             cudaStream_t);                                        \
    template cudaError_t export_particles<T>(PArrays<T>, const int32_t*, GridP, double*, double*,  \
                                             double*, int32_t*, cudaStream_t);                     \
    template cudaError_t deposit<T>(const DepositSpecies<T>&, const T*, T*, T*, GridP, cudaStream_t); \
    template cudaError_t push<T>(int, PArrays<T>, PArrays<T>, const int32_t*, int32_t*,            \
                                 const int32_t*, int32_t*, const T*, const T*, GridP, SpeciesConst, \
                                 double*, int, int64_t, int*, cudaStream_t);                       \
    template cudaError_t kinetic_energy<T>(PArrays<T>, int64_t, double, double*, int, cudaStream_t);

RELSIM_INSTANTIATE(float)
RELSIM_INSTANTIATE(double)

}  // namespace relsim
