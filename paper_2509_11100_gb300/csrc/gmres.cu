// gmres.cu -- the control of the restarted GMRES solve (Sec. 2: the field
// solver is the implicit part of the method) decided on the device.
//
// The Arnoldi process runs on B = A - I with an FP64 Krylov basis (double-
// float pairs in the FP32 form of the 2D scheme with linear shapes). Its
// heavy kernels (operator with fused dot products, their reduction, the
// fused basis update) are in fields.cu; the single-thread kernels here keep
// the small dense part on the device: the Hessenberg column, the Givens
// rotations, the residual estimate, the stop tests, the triangular solve
// for the update, and the launch arguments of the next iteration (GmDyn).
// With nothing left for the host to decide between iterations, the whole
// solve can run as a CUDA graph whose loops are conditional while nodes
// (the kernels set the loop conditions), or be driven from the host.
//
// When the norm of w - V h loses most of its digits (|w - V h|^2 < 1e-4
// |w|^2, so the new basis vector would not be orthogonal to the others), the
// cycle ends without that column and GMRES restarts from the true residual
// (at j = 0 the column is kept: the Krylov space is then nearly invariant).
#include "launch.cuh"

namespace relsim {
namespace {

__global__ void k_gm_begin(GmState* st, const double* __restrict__ sums)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    const double bn = sqrt(sums[0]);
    st->bnorm = bn;
    st->beta = 0.0;
    st->relres = 0.0;
    st->total = 0;
    st->restarts = 0;
    st->kdim = 0;
    st->run = 0;
    st->inner = 0;
    st->status = isfinite(bn) ? kGmOk : kGmNonfinite;
    st->zero = bn == 0.0 ? 1 : 0;
    st->dyn.live = 0;
}

__global__ void k_gm_zero_x(const GmState* __restrict__ st, double* __restrict__ x, int64_t n)
{
    if (!st->zero) return;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
        x[e] = 0.0;
}

__global__ void k_gm_cycle(GmState* st, const double* __restrict__ sums, GmPtrs p, GmParams q,
                           cudaGraphConditionalHandle cond, int has_cond)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    int run = 0;
    if (st->status == kGmOk) {
        const double beta = sqrt(sums[0]);
        if (!isfinite(beta)) {
            st->status = kGmNonfinite;
        } else {
            st->beta = beta;
            const double rr = st->zero ? 0.0 : beta / st->bnorm;
            st->relres = rr;
            if (st->zero || rr <= q.tol) {
                // converged
            } else if (st->total >= q.maxit || st->restarts > q.maxit) {
                // (every cycle runs at least one iteration, so the second
                // bound only backs up the first: the loop always ends)
                st->status = kGmNotConverged;
            } else {
                run = 1;
                st->gv[0] = beta;
                for (int k = 1; k <= q.m; ++k) st->gv[k] = 0.0;
                st->kdim = 0;
                GmDyn& d = st->dyn;
                d.in = p.r;      // v_0 = r / beta, written to V_0 by iteration 0
                d.vj = p.V;
                d.out = p.w0;
                d.ds = p.ds0;
                d.s = 1.0 / beta;
                d.nv = 0;
            }
        }
    }
    st->run = run;
    st->inner = run;
    st->dyn.live = run;
    if (has_cond) cudaGraphSetConditional(cond, run);
}

__global__ void k_gm_arm(const GmState* __restrict__ st, cudaGraphConditionalHandle cond, int has_cond)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    if (has_cond) cudaGraphSetConditional(cond, st->run);
}

__global__ void k_gm_tail(GmState* st, GmPtrs p, GmParams q, cudaGraphConditionalHandle cond, int has_cond)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    GmDyn& d = st->dyn;
    int inner = 0;
    if (d.live) {
        const int j = d.nv, m = q.m;
        const double* hj = d.ds;
        const double ww = hj[j + 1];
        double hn2 = ww;
        for (int i = 0; i <= j; ++i) hn2 -= hj[i] * hj[i];
        st->total += 1;
        if (!isfinite(hn2)) {
            st->status = kGmNonfinite;
            st->kdim = 0;
            st->run = 0;
        } else if (j > 0 && hn2 < 1e-4 * ww) {
            st->kdim = j;   // end the cycle without column j; restart from the true residual
        } else {
            double* H = st->H;
            double* cs = st->cs;
            double* sn = st->sn;
            double* gv = st->gv;
            const double hn = sqrt(hn2 > 0.0 ? hn2 : 0.0);
            for (int i = 0; i <= j; ++i) H[i * m + j] = hj[i];
            H[j * m + j] += 1.0;   // A = I + B
            H[(j + 1) * m + j] = hn;
            for (int i = 0; i < j; ++i) {
                const double t = cs[i] * H[i * m + j] + sn[i] * H[(i + 1) * m + j];
                H[(i + 1) * m + j] = -sn[i] * H[i * m + j] + cs[i] * H[(i + 1) * m + j];
                H[i * m + j] = t;
            }
            const double a = H[j * m + j], b = H[(j + 1) * m + j];
            const double r = hypot(a, b);
            cs[j] = r == 0.0 ? 1.0 : a / r;
            sn[j] = r == 0.0 ? 0.0 : b / r;
            H[j * m + j] = r;
            H[(j + 1) * m + j] = 0.0;
            gv[j + 1] = -sn[j] * gv[j];
            gv[j] = cs[j] * gv[j];
            st->kdim = j + 1;
            const bool stop = fabs(gv[j + 1]) <= q.tol * st->bnorm || st->total >= q.maxit || hn == 0.0 ||
                              j + 1 >= m;
            if (!stop) {
                const int jn = j + 1;
                inner = 1;
                d.in = p.V + (int64_t)jn * p.ldv;
                d.vj = nullptr;
                d.out = jn % 2 == 0 ? p.w0 : p.r;
                d.ds = jn % 2 == 0 ? p.ds0 : p.ds1;
                d.s = 1.0;
                d.nv = jn;
            }
        }
    }
    d.live = inner;
    st->inner = inner;
    if (has_cond) cudaGraphSetConditional(cond, inner);
}

// back substitution R y = g over the finished cycle's kdim columns
__global__ void k_gm_solve_y(GmState* st, int m)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    if (!st->run) {
        st->kdim = 0;
        return;
    }
    const int kdim = st->kdim;
    const double* H = st->H;
    for (int i = kdim - 1; i >= 0; --i) {
        double s = st->gv[i];
        for (int k = i + 1; k < kdim; ++k) s -= H[i * m + k] * st->y[k];
        st->y[i] = H[i * m + i] != 0.0 ? s / H[i * m + i] : 0.0;
    }
    st->restarts += 1;
}

}  // namespace

cudaError_t gm_begin(GmState* st, const double* sums, cudaStream_t s)
{
    count_launches(1);
    k_gm_begin<<<1, 32, 0, s>>>(st, sums);
    return cudaGetLastError();
}

cudaError_t gm_zero_x(const GmState* st, double* x, int64_t n, cudaStream_t s)
{
    count_launches(1);
    const int64_t b = (n + 255) / 256;
    k_gm_zero_x<<<(int)(b < 152 * 4 ? (b < 1 ? 1 : b) : 152 * 4), 256, 0, s>>>(st, x, n);
    return cudaGetLastError();
}

cudaError_t gm_cycle(GmState* st, const double* sums, GmPtrs p, GmParams q, GmCond cond, cudaStream_t s)
{
    count_launches(1);
    k_gm_cycle<<<1, 32, 0, s>>>(st, sums, p, q, (cudaGraphConditionalHandle)cond.h, cond.has);
    return cudaGetLastError();
}

cudaError_t gm_arm(const GmState* st, GmCond cond, cudaStream_t s)
{
    count_launches(1);
    k_gm_arm<<<1, 32, 0, s>>>(st, (cudaGraphConditionalHandle)cond.h, cond.has);
    return cudaGetLastError();
}

cudaError_t gm_tail(GmState* st, GmPtrs p, GmParams q, GmCond cond, cudaStream_t s)
{
    count_launches(1);
    k_gm_tail<<<1, 32, 0, s>>>(st, p, q, (cudaGraphConditionalHandle)cond.h, cond.has);
    return cudaGetLastError();
}

cudaError_t gm_finish_cycle(GmState* st, double* x, const double* V, int64_t ldv, int64_t n, int m,
                            cudaStream_t s, int df)
{
    count_launches(1);
    k_gm_solve_y<<<1, 32, 0, s>>>(st, m);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return gm_combine_dev(x, V, ldv, &st->kdim, st->y, n, s, df);
}

}  // namespace relsim
