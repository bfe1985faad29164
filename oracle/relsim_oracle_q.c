/*
 * relsim_oracle_q.c -- the plain FP64 CPU oracle of one 2D RelSIM step with
 * quadratic (triangular-shaped-cloud, TSC) shape functions.
 *
 * TEST INFRASTRUCTURE ONLY (see relsim_oracle.h): the tests and the
 * benchmark's CPU-baseline leg are its only users; the CUDA library never
 * links or calls it.
 *
 * The scheme of relsim_oracle.c (Sec. 2: explicit pusher, implicit field
 * solve through the mass matrices) with the linear shape replaced by the
 * quadratic B-spline: along each axis a particle at lattice coordinate s
 * touches the nearest node n = floor(s + 1/2) and its two neighbours with
 * weights 1/2 (1/2 - d)^2, 3/4 - d^2, 1/2 (1/2 + d)^2 for nodes n-1, n, n+1,
 * d = s - n in [-1/2, 1/2). The same shape, on the centre lattice (shifted
 * by half a cell), gathers B. A particle touches 3 x 3 nodes, so its
 * mass-matrix contributions couple node pairs up to two cells apart along
 * each axis (25 neighbour offsets). The curls, the right-hand side, the
 * field update and the energies do not depend on the shape and are the 2D
 * oracle's. The base scheme only (gbar = gamma(u^n)).
 *
 * M is stored for all 25 offsets: M[((g*25 + o)*3 + r)*3 + s] with
 * o = (dj+2)*5 + (di+2) for node g + (di, dj).
 */
#include "relsim_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

static int64_t wrapq(int64_t i, int64_t n)
{
    i %= n;
    return i < 0 ? i + n : i;
}

/* the three quadratic weights around the nearest lattice point of s */
static void quad1(double s, int n, int64_t idx[3], double w[3])
{
    double fl = floor(s + 0.5);
    double d = s - fl;
    int64_t c = (int64_t)fl;
    idx[0] = wrapq(c - 1, n);
    idx[1] = wrapq(c, n);
    idx[2] = wrapq(c + 1, n);
    w[0] = 0.5 * (0.5 - d) * (0.5 - d);
    w[1] = 0.75 - d * d;
    w[2] = 0.5 * (0.5 + d) * (0.5 + d);
}

/* 9 nodes (shift 0) or centres (shift 1/2) with their weights; a = 3*ay + ax */
static void weightsq(const orc_config* c, double x, double y, double shift, int64_t g[9], double W[9])
{
    int64_t ix[3], iy[3];
    double wx[3], wy[3];
    quad1(x / c->dx - shift, c->nx, ix, wx);
    quad1(y / c->dy - shift, c->ny, iy, wy);
    for (int ay = 0; ay < 3; ++ay)
        for (int ax = 0; ax < 3; ++ax) {
            g[3 * ay + ax] = iy[ay] * c->nx + ix[ax];
            W[3 * ay + ax] = wx[ax] * wy[ay];
        }
}

void orcq_node_weights(const orc_config* c, double x, double y, int64_t g[9], double W[9])
{
    weightsq(c, x, y, 0.0, g, W);
}

void orcq_gather_E(const orc_config* c, const double* E, double x, double y, double out[3])
{
    int64_t g[9];
    double W[9];
    int64_t nn = (int64_t)c->nx * c->ny;
    weightsq(c, x, y, 0.0, g, W);
    for (int k = 0; k < 3; ++k) {
        out[k] = 0.0;
        for (int a = 0; a < 9; ++a) out[k] += W[a] * E[k * nn + g[a]];
    }
}

void orcq_gather_B(const orc_config* c, const double* B, double x, double y, double out[3])
{
    int64_t g[9];
    double W[9];
    int64_t nn = (int64_t)c->nx * c->ny;
    weightsq(c, x, y, 0.5, g, W);
    for (int k = 0; k < 3; ++k) {
        out[k] = 0.0;
        for (int a = 0; a < 9; ++a) out[k] += W[a] * B[k * nn + g[a]];
    }
}

static double gammaq(const double u[3]) { return sqrt(1.0 + u[0] * u[0] + u[1] * u[1] + u[2] * u[2]); }

static double gammaq_m1(const double u[3])
{
    double u2 = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    return u2 / (sqrt(1.0 + u2) + 1.0);
}

/* Steps 1-5 with the quadratic shape: Jhat[3 nn], M[25*9 nn]. Node a and b of
   a particle's 3x3 set are (bx-ax, by-ay) apart. */
void orcq_deposit(const orc_config* c, const int64_t* off, const double* x, const double* y, const double* ux,
                  const double* uy, const double* uz, const double* w, const double* B, double* J, double* M)
{
    int64_t nn = (int64_t)c->nx * c->ny;
    double dV = c->dx * c->dy;
    memset(J, 0, sizeof(double) * 3 * nn);
    memset(M, 0, sizeof(double) * 225 * nn);
    for (int s = 0; s < c->nspecies; ++s) {
        double q = c->q[s], m = c->m[s];
        double beta = q * c->dt / (2.0 * m);
        for (int64_t p = off[s]; p < off[s + 1]; ++p) {
            double Bp[3], alpha[9], u[3] = {ux[p], uy[p], uz[p]};
            orcq_gather_B(c, B, x[p], y[p], Bp);
            double gbar = gammaq(u);
            orc_alpha(beta, gbar, Bp, alpha);
            double vJ[3];
            for (int r = 0; r < 3; ++r) {
                vJ[r] = 0.0;
                for (int k = 0; k < 3; ++k) vJ[r] += alpha[r * 3 + k] * u[k];
                vJ[r] /= gbar;
            }
            int64_t g[9];
            double W[9];
            weightsq(c, x[p], y[p], 0.0, g, W);
            double cJ = w[p] * q / dV;
            double cM = w[p] * q * beta / (gbar * dV);
            for (int a = 0; a < 9; ++a) {
                for (int k = 0; k < 3; ++k) J[k * nn + g[a]] += cJ * W[a] * vJ[k];
                for (int b = 0; b < 9; ++b) {
                    int di = (b % 3) - (a % 3), dj = (b / 3) - (a / 3);
                    int o = (dj + 2) * 5 + (di + 2);
                    double* blk = M + (g[a] * 25 + o) * 9;
                    for (int rs = 0; rs < 9; ++rs) blk[rs] += cM * W[a] * W[b] * alpha[rs];
                }
            }
        }
    }
}

/* (M v)_g = sum over the 25 offsets o of M[g][o] v_{g+o} */
void orcq_apply_M(const orc_config* c, const double* M, const double* v, double* out)
{
    int nx = c->nx, ny = c->ny;
    int64_t nn = (int64_t)nx * ny;
    for (int j = 0; j < ny; ++j)
        for (int i = 0; i < nx; ++i) {
            int64_t g = (int64_t)j * nx + i;
            double acc[3] = {0.0, 0.0, 0.0};
            for (int dj = -2; dj <= 2; ++dj)
                for (int di = -2; di <= 2; ++di) {
                    int o = (dj + 2) * 5 + (di + 2);
                    int64_t h = wrapq(j + dj, ny) * nx + wrapq(i + di, nx);
                    const double* blk = M + (g * 25 + o) * 9;
                    for (int r = 0; r < 3; ++r)
                        for (int s = 0; s < 3; ++s) acc[r] += blk[r * 3 + s] * v[s * nn + h];
                }
            for (int r = 0; r < 3; ++r) out[r * nn + g] = acc[r];
        }
}

void orcq_apply_A(const orc_config* c, const double* M, const double* v, double* out)
{
    int64_t nn = (int64_t)c->nx * c->ny;
    double* cc = (double*)malloc(sizeof(double) * 3 * nn);
    double* cn = (double*)malloc(sizeof(double) * 3 * nn);
    double* mv = (double*)malloc(sizeof(double) * 3 * nn);
    double td = c->theta * c->dt;
    orc_curl_c(c, v, cc);
    orc_curl_n(c, cc, cn);
    orcq_apply_M(c, M, v, mv);
    for (int64_t k = 0; k < 3 * nn; ++k) out[k] = v[k] + td * td * cn[k] + td * mv[k];
    free(cc);
    free(cn);
    free(mv);
}

static double dotq(int64_t n, const double* a, const double* b)
{
    double s = 0.0;
    for (int64_t k = 0; k < n; ++k) s += a[k] * b[k];
    return s;
}

/* Restarted GMRES(m), modified Gram-Schmidt, Givens rotations (the textbook
   algorithm, as in the 2D oracle), on the quadratic-shape operator. */
int orcq_gmres(const orc_config* c, const double* M, const double* b, double* x, int* iters, double* relres)
{
    int64_t n = 3 * (int64_t)c->nx * c->ny;
    int m = c->gmres_restart > 0 ? c->gmres_restart : 50;
    int maxit = c->gmres_maxit > 0 ? c->gmres_maxit : 1000;
    double tol = c->gmres_tol;
    double* V = (double*)malloc(sizeof(double) * n * (m + 1));
    double* H = (double*)calloc((size_t)(m + 1) * m, sizeof(double));
    double *cs = (double*)malloc(sizeof(double) * m), *sn = (double*)malloc(sizeof(double) * m);
    double* g = (double*)malloc(sizeof(double) * (m + 1));
    double* y = (double*)malloc(sizeof(double) * m);
    double* r = (double*)malloc(sizeof(double) * n);
    double* w = (double*)malloc(sizeof(double) * n);
    int total = 0, status = 1;
    double bnorm = sqrt(dotq(n, b, b));
    if (bnorm == 0.0) {
        memset(x, 0, sizeof(double) * n);
        *iters = 0;
        *relres = 0.0;
        status = 0;
        goto done;
    }
    for (;;) {
        orcq_apply_A(c, M, x, w);
        for (int64_t k = 0; k < n; ++k) r[k] = b[k] - w[k];
        double beta = sqrt(dotq(n, r, r));
        *relres = beta / bnorm;
        if (*relres <= tol) {
            status = 0;
            break;
        }
        if (total >= maxit) break;
        for (int64_t k = 0; k < n; ++k) V[k] = r[k] / beta;
        memset(g, 0, sizeof(double) * (m + 1));
        g[0] = beta;
        int kdim = 0;
        for (int j = 0; j < m; ++j) {
            orcq_apply_A(c, M, V + (int64_t)j * n, w);
            for (int i = 0; i <= j; ++i) {
                double* vi = V + (int64_t)i * n;
                double h = dotq(n, w, vi);
                H[i * m + j] = h;
                for (int64_t k = 0; k < n; ++k) w[k] -= h * vi[k];
            }
            double hn = sqrt(dotq(n, w, w));
            H[(j + 1) * m + j] = hn;
            if (hn != 0.0)
                for (int64_t k = 0; k < n; ++k) V[(int64_t)(j + 1) * n + k] = w[k] / hn;
            for (int i = 0; i < j; ++i) {
                double t = cs[i] * H[i * m + j] + sn[i] * H[(i + 1) * m + j];
                H[(i + 1) * m + j] = -sn[i] * H[i * m + j] + cs[i] * H[(i + 1) * m + j];
                H[i * m + j] = t;
            }
            double aa = H[j * m + j], bb = H[(j + 1) * m + j];
            double rr = hypot(aa, bb);
            cs[j] = rr == 0.0 ? 1.0 : aa / rr;
            sn[j] = rr == 0.0 ? 0.0 : bb / rr;
            H[j * m + j] = rr;
            H[(j + 1) * m + j] = 0.0;
            g[j + 1] = -sn[j] * g[j];
            g[j] = cs[j] * g[j];
            ++total;
            kdim = j + 1;
            if (fabs(g[j + 1]) <= tol * bnorm || total >= maxit || hn == 0.0) break;
        }
        for (int i = kdim - 1; i >= 0; --i) {
            double s = g[i];
            for (int k = i + 1; k < kdim; ++k) s -= H[i * m + k] * y[k];
            y[i] = s / H[i * m + i];
        }
        for (int i = 0; i < kdim; ++i)
            for (int64_t k = 0; k < n; ++k) x[k] += y[i] * V[(int64_t)i * n + k];
    }
    *iters = total;
done:
    free(V); free(H); free(cs); free(sn); free(g); free(y); free(r); free(w);
    return status;
}

static double wrap_posq(double s, double L)
{
    double t = s - L * floor(s / L);
    if (t >= L) t = 0.0;
    if (t < 0.0) t = 0.0;
    return t;
}

/* Steps 9 and 10 and the ledger's particle sums {K0, K1, work, mismatch}. */
void orcq_push(const orc_config* c, const int64_t* off, double* x, double* y, double* ux, double* uy, double* uz,
               const double* w, const double* Etheta, const double* B, double sums[4])
{
    double Lx = c->nx * c->dx, Ly = c->ny * c->dy;
    for (int k = 0; k < 4; ++k) sums[k] = 0.0;
    for (int s = 0; s < c->nspecies; ++s) {
        double q = c->q[s], m = c->m[s];
        double beta = q * c->dt / (2.0 * m);
        for (int64_t p = off[s]; p < off[s + 1]; ++p) {
            double Ep[3], Bp[3], alpha[9];
            double u0[3] = {ux[p], uy[p], uz[p]};
            orcq_gather_E(c, Etheta, x[p], y[p], Ep);
            orcq_gather_B(c, B, x[p], y[p], Bp);
            double gbar = gammaq(u0);
            orc_alpha(beta, gbar, Bp, alpha);
            double wv[3], ub[3], u1[3];
            for (int k = 0; k < 3; ++k) wv[k] = u0[k] + beta * Ep[k];
            for (int r = 0; r < 3; ++r) {
                ub[r] = 0.0;
                for (int k = 0; k < 3; ++k) ub[r] += alpha[r * 3 + k] * wv[k];
            }
            for (int k = 0; k < 3; ++k) u1[k] = 2.0 * ub[k] - u0[k];
            double g1 = gammaq(u1);
            double ue = ub[0] * Ep[0] + ub[1] * Ep[1] + ub[2] * Ep[2];
            double du = 0.0;
            for (int k = 0; k < 3; ++k) du += (u0[k] - u1[k]) * (u0[k] + u1[k]);
            double g01 = du / (gbar + g1);
            sums[0] += w[p] * m * gammaq_m1(u0);
            sums[1] += w[p] * m * gammaq_m1(u1);
            sums[2] += c->dt * w[p] * q * ue / gbar;
            sums[3] += c->dt * w[p] * q * ue * g01 / (gbar * (gbar + g1));
            ux[p] = u1[0];
            uy[p] = u1[1];
            uz[p] = u1[2];
            x[p] = wrap_posq(x[p] + c->dt * u1[0] / g1, Lx);
            y[p] = wrap_posq(y[p] + c->dt * u1[1] / g1, Ly);
        }
    }
}

int orcq_step(const orc_config* c, const int64_t* off, double* x, double* y, double* ux, double* uy, double* uz,
              const double* w, double* E, double* B, orc_ledger* led, double* J_out, double* M_out,
              double* Etheta_out)
{
    int64_t nn = (int64_t)c->nx * c->ny;
    double dV = c->dx * c->dy;
    double* J = (double*)malloc(sizeof(double) * 3 * nn);
    double* M = (double*)malloc(sizeof(double) * 225 * nn);
    double* b = (double*)malloc(sizeof(double) * 3 * nn);
    double* Et = (double*)malloc(sizeof(double) * 3 * nn);
    double* E0 = (double*)malloc(sizeof(double) * 3 * nn);
    double* B0 = (double*)malloc(sizeof(double) * 3 * nn);
    double* Jbar = (double*)malloc(sizeof(double) * 3 * nn);
    double en0[3], en1[3], sums[4];
    orc_energies(c, off, ux, uy, uz, w, E, B, en0);
    memcpy(E0, E, sizeof(double) * 3 * nn);
    memcpy(B0, B, sizeof(double) * 3 * nn);

    orcq_deposit(c, off, x, y, ux, uy, uz, w, B, J, M);          /* steps 1-5 */
    orc_rhs(c, E, B, J, b);                                       /* step 6 */
    memcpy(Et, E, sizeof(double) * 3 * nn);
    int iters = 0;
    double relres = 0.0;
    int st = orcq_gmres(c, M, b, Et, &iters, &relres);
    orc_field_update(c, Et, E, B);                                /* steps 7-8 */
    orcq_push(c, off, x, y, ux, uy, uz, w, Et, B0, sums);         /* steps 9-10 */
    orc_energies(c, off, ux, uy, uz, w, E, B, en1);

    if (led) {
        orcq_apply_M(c, M, Et, Jbar);
        for (int64_t k = 0; k < 3 * nn; ++k) Jbar[k] += J[k];
        double dE2 = 0.0, dB2 = 0.0;
        for (int64_t k = 0; k < 3 * nn; ++k) {
            dE2 += (E[k] - E0[k]) * (E[k] - E0[k]);
            dB2 += (B[k] - B0[k]) * (B[k] - B0[k]);
        }
        led->W_E0 = en0[0]; led->W_B0 = en0[1]; led->K0 = en0[2];
        led->W_E1 = en1[0]; led->W_B1 = en1[1]; led->K1 = en1[2];
        led->work_grid = c->dt * dV * dotq(3 * nn, Jbar, Et);
        led->work_particles = sums[2];
        led->mismatch = sums[3];
        led->dissipation = (c->theta - 0.5) * dV * (dE2 + dB2);
        led->residual = (en1[0] + en1[1] + en1[2]) - (en0[0] + en0[1] + en0[2]) - led->mismatch + led->dissipation;
        led->gmres_iters = iters;
        led->gmres_relres = relres;
    }
    if (J_out) memcpy(J_out, J, sizeof(double) * 3 * nn);
    if (M_out) memcpy(M_out, M, sizeof(double) * 225 * nn);
    if (Etheta_out) memcpy(Etheta_out, Et, sizeof(double) * 3 * nn);
    free(J); free(M); free(b); free(Et); free(E0); free(B0); free(Jbar);
    return st;
}
