/*
 * relsim_oracle.c -- plain FP64 CPU oracle of one RelSIM step.
 *
 * TEST INFRASTRUCTURE ONLY (see relsim_oracle.h): the tests, the smoke check
 * and the benchmark's CPU-baseline leg are its only users; the CUDA library
 * never links or calls it.
 *
 * The paper (Sec. 2, "Methods and Simulation Setup") states the structure of
 * the method: the particle pusher is explicit, only the field solver is
 * implicit, and the field solver uses a mass-matrix formulation that
 * conserves energy exactly in the non-relativistic limit. It does not print
 * the equations; they are those of the energy-conserving semi-implicit
 * method (ECSIM) it builds on, extended to relativistic momenta. This file
 * writes that scheme out step by step, in this order (the readings where the
 * paper is silent are listed in the repository's design notes):
 *
 *   state: x^{n+1/2}, u^n (u = gamma v), E^n on nodes, B^n on cell centres
 *   1. gbar = sqrt(1 + |u^n|^2)  (or, with gamma_pred, the Lorentz factor of
 *      the predicted half-step momentum u^n + beta E^n(x): the magnetic
 *      rotation keeps |u| and E^n stands in for E^{n+theta})
 *   2. a = beta B^n(x)/gbar, beta = q dt/(2m)
 *   3. alpha = (I - [a]x + a a^T)/(1 + |a|^2), the solution operator of
 *      ubar - ubar x a = w (the implicit-midpoint rotation)
 *   4. Jhat_g = sum_p w q W_g alpha u^n/gbar / dV
 *   5. M_gg'  = sum_p w q beta/gbar W_g W_g' alpha / dV
 *   6. (I + (theta dt)^2 curl_n curl_c + theta dt M) E^{n+theta}
 *        = E^n + theta dt curl_n B^n - theta dt Jhat        (GMRES)
 *   7. E^{n+1} = (E^{n+theta} - (1-theta) E^n)/theta
 *   8. B^{n+1} = B^n - dt curl_c E^{n+theta}
 *   9. ubar = alpha (u^n + beta E^{n+theta}(x)); u^{n+1} = 2 ubar - u^n
 *  10. x^{n+3/2} = x^{n+1/2} + dt u^{n+1}/sqrt(1 + |u^{n+1}|^2), periodic
 *
 * Everything is FP64, single-threaded, with no blocking or fusion.
 */
#include "relsim_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

int orc_version(void) { return 1; }

static int64_t wrapi(int64_t i, int64_t n)
{
    i %= n;
    return i < 0 ? i + n : i;
}

/* Cell (i,j) holding the point and the fractional offsets inside it. */
static void locate(double s, double d, int n, int64_t* i, double* f)
{
    double t = s / d;
    double fl = floor(t);
    *f = t - fl;
    *i = wrapi((int64_t)fl, n);
}

/* Linear (CIC) node weights: the four nodes of the cell holding (x,y). */
void orc_node_weights(const orc_config* c, double x, double y, int64_t g[4], double W[4])
{
    int64_t i, j;
    double fx, fy;
    locate(x, c->dx, c->nx, &i, &fx);
    locate(y, c->dy, c->ny, &j, &fy);
    int64_t i1 = wrapi(i + 1, c->nx), j1 = wrapi(j + 1, c->ny);
    g[0] = j * c->nx + i;   W[0] = (1.0 - fx) * (1.0 - fy);
    g[1] = j * c->nx + i1;  W[1] = fx * (1.0 - fy);
    g[2] = j1 * c->nx + i;  W[2] = (1.0 - fx) * fy;
    g[3] = j1 * c->nx + i1; W[3] = fx * fy;
}

/* Linear weights on the cell-centre lattice (centres at (i+1/2, j+1/2)). */
static void centre_weights(const orc_config* c, double x, double y, int64_t g[4], double W[4])
{
    int64_t i, j;
    double fx, fy;
    locate(x - 0.5 * c->dx, c->dx, c->nx, &i, &fx);
    locate(y - 0.5 * c->dy, c->dy, c->ny, &j, &fy);
    int64_t i1 = wrapi(i + 1, c->nx), j1 = wrapi(j + 1, c->ny);
    g[0] = j * c->nx + i;   W[0] = (1.0 - fx) * (1.0 - fy);
    g[1] = j * c->nx + i1;  W[1] = fx * (1.0 - fy);
    g[2] = j1 * c->nx + i;  W[2] = (1.0 - fx) * fy;
    g[3] = j1 * c->nx + i1; W[3] = fx * fy;
}

void orc_gather_E(const orc_config* c, const double* E, double x, double y, double out[3])
{
    int64_t g[4];
    double W[4];
    int64_t nn = (int64_t)c->nx * c->ny;
    orc_node_weights(c, x, y, g, W);
    for (int k = 0; k < 3; ++k) {
        out[k] = 0.0;
        for (int a = 0; a < 4; ++a) out[k] += W[a] * E[k * nn + g[a]];
    }
}

void orc_gather_B(const orc_config* c, const double* B, double x, double y, double out[3])
{
    int64_t g[4];
    double W[4];
    int64_t nn = (int64_t)c->nx * c->ny;
    centre_weights(c, x, y, g, W);
    for (int k = 0; k < 3; ++k) {
        out[k] = 0.0;
        for (int a = 0; a < 4; ++a) out[k] += W[a] * B[k * nn + g[a]];
    }
}

/* alpha = (I - [a]x + a a^T)/(1 + |a|^2) with a = beta Bp / gbar, where
   [a]x v = a x v. Row-major alpha[r*3 + s]. */
void orc_alpha(double beta, double gbar, const double Bp[3], double alpha[9])
{
    double a[3];
    for (int k = 0; k < 3; ++k) a[k] = beta * Bp[k] / gbar;
    double a2 = a[0] * a[0] + a[1] * a[1] + a[2] * a[2];
    /* cross-product matrix: ([a]x)_{rs} with (a x v)_r = sum_s ([a]x)_{rs} v_s */
    double ax[9] = {0.0, -a[2], a[1],
                    a[2], 0.0, -a[0],
                    -a[1], a[0], 0.0};
    for (int r = 0; r < 3; ++r)
        for (int s = 0; s < 3; ++s)
            alpha[r * 3 + s] = ((r == s ? 1.0 : 0.0) - ax[r * 3 + s] + a[r] * a[s]) / (1.0 + a2);
}

static double gamma_of(double ux, double uy, double uz)
{
    return sqrt(1.0 + ux * ux + uy * uy + uz * uz);
}

/* gamma - 1 written as |u|^2/(gamma + 1): the same number without the
   cancellation of sqrt(1+u^2) - 1 for slow particles. */
static double gamma_m1(double ux, double uy, double uz)
{
    double u2 = ux * ux + uy * uy + uz * uz;
    return u2 / (sqrt(1.0 + u2) + 1.0);
}

/* the Lorentz factor in alpha and M (step 1) */
static double gbar_of(const orc_config* c, double beta, const double* E, double x, double y,
                      const double u[3])
{
    if (!c->gamma_pred) return gamma_of(u[0], u[1], u[2]);
    double Ep[3];
    orc_gather_E(c, E, x, y, Ep);
    return gamma_of(u[0] + beta * Ep[0], u[1] + beta * Ep[1], u[2] + beta * Ep[2]);
}

/* Offset slot of node b relative to node a, both nodes of one cell. */
static int pair_slot(const orc_config* c, int64_t ga, int64_t gb)
{
    int64_t ia = ga % c->nx, ja = ga / c->nx, ib = gb % c->nx, jb = gb / c->nx;
    int64_t di = ib - ia, dj = jb - ja;
    /* undo the periodic wrap: the two nodes are at most one cell apart */
    if (di > 1) di -= c->nx;
    if (di < -1) di += c->nx;
    if (dj > 1) dj -= c->ny;
    if (dj < -1) dj += c->ny;
    return (int)((dj + 1) * 3 + (di + 1));
}

/* Steps 1-5: predicted current and mass matrices from x^{n+1/2}, u^n, B^n. */
void orc_deposit(const orc_config* c, const int64_t* off,
                 const double* x, const double* y,
                 const double* ux, const double* uy, const double* uz,
                 const double* w, const double* B, const double* E, double* J, double* M)
{
    int64_t nn = (int64_t)c->nx * c->ny;
    double dV = c->dx * c->dy;
    memset(J, 0, sizeof(double) * 3 * nn);
    memset(M, 0, sizeof(double) * 81 * nn);
    for (int s = 0; s < c->nspecies; ++s) {
        double q = c->q[s], m = c->m[s];
        double beta = q * c->dt / (2.0 * m);
        for (int64_t p = off[s]; p < off[s + 1]; ++p) {
            double Bp[3], alpha[9], u[3] = {ux[p], uy[p], uz[p]};
            orc_gather_B(c, B, x[p], y[p], Bp);
            double gbar = gbar_of(c, beta, E, x[p], y[p], u);
            orc_alpha(beta, gbar, Bp, alpha);
            double vJ[3];
            for (int r = 0; r < 3; ++r) {
                vJ[r] = 0.0;
                for (int k = 0; k < 3; ++k) vJ[r] += alpha[r * 3 + k] * u[k];
                vJ[r] /= gbar;
            }
            int64_t g[4];
            double W[4];
            orc_node_weights(c, x[p], y[p], g, W);
            double cJ = w[p] * q / dV;
            double cM = w[p] * q * beta / (gbar * dV);
            for (int a = 0; a < 4; ++a) {
                for (int k = 0; k < 3; ++k) J[k * nn + g[a]] += cJ * W[a] * vJ[k];
                for (int b = 0; b < 4; ++b) {
                    int o = pair_slot(c, g[a], g[b]);
                    double* blk = M + ((g[a] * 9 + o) * 9);
                    for (int rs = 0; rs < 9; ++rs) blk[rs] += cM * W[a] * W[b] * alpha[rs];
                }
            }
        }
    }
}

/* node -> centre curl. Differences across the cell, averaged over its two
   edges in the other direction. */
void orc_curl_c(const orc_config* c, const double* E, double* out)
{
    int nx = c->nx, ny = c->ny;
    int64_t nn = (int64_t)nx * ny;
    const double *Ex = E, *Ey = E + nn, *Ez = E + 2 * nn;
    for (int j = 0; j < ny; ++j)
        for (int i = 0; i < nx; ++i) {
            int64_t n00 = (int64_t)j * nx + i;
            int64_t n10 = (int64_t)j * nx + wrapi(i + 1, nx);
            int64_t n01 = wrapi(j + 1, ny) * nx + i;
            int64_t n11 = wrapi(j + 1, ny) * nx + wrapi(i + 1, nx);
#define DX(f) (((f)[n10] - (f)[n00] + (f)[n11] - (f)[n01]) / (2.0 * c->dx))
#define DY(f) (((f)[n01] - (f)[n00] + (f)[n11] - (f)[n10]) / (2.0 * c->dy))
            out[n00] = DY(Ez);
            out[nn + n00] = -DX(Ez);
            out[2 * nn + n00] = DX(Ey) - DY(Ex);
#undef DX
#undef DY
        }
}

/* centre -> node curl, over the four centres around the node. */
void orc_curl_n(const orc_config* c, const double* B, double* out)
{
    int nx = c->nx, ny = c->ny;
    int64_t nn = (int64_t)nx * ny;
    const double *Bx = B, *By = B + nn, *Bz = B + 2 * nn;
    for (int j = 0; j < ny; ++j)
        for (int i = 0; i < nx; ++i) {
            int64_t c11 = (int64_t)j * nx + i;                              /* (i, j)     */
            int64_t c01 = (int64_t)j * nx + wrapi(i - 1, nx);               /* (i-1, j)   */
            int64_t c10 = wrapi(j - 1, ny) * nx + i;                        /* (i, j-1)   */
            int64_t c00 = wrapi(j - 1, ny) * nx + wrapi(i - 1, nx);         /* (i-1, j-1) */
#define DX(f) (((f)[c11] - (f)[c01] + (f)[c10] - (f)[c00]) / (2.0 * c->dx))
#define DY(f) (((f)[c11] - (f)[c10] + (f)[c01] - (f)[c00]) / (2.0 * c->dy))
            out[c11] = DY(Bz);
            out[nn + c11] = -DX(Bz);
            out[2 * nn + c11] = DX(By) - DY(Bx);
#undef DX
#undef DY
        }
}

/* (M v)_g = sum_o M[g][o] v_{g+o} */
void orc_apply_M(const orc_config* c, const double* M, const double* v, double* out)
{
    int nx = c->nx, ny = c->ny;
    int64_t nn = (int64_t)nx * ny;
    for (int j = 0; j < ny; ++j)
        for (int i = 0; i < nx; ++i) {
            int64_t g = (int64_t)j * nx + i;
            double acc[3] = {0.0, 0.0, 0.0};
            for (int dj = -1; dj <= 1; ++dj)
                for (int di = -1; di <= 1; ++di) {
                    int o = (dj + 1) * 3 + (di + 1);
                    int64_t h = wrapi(j + dj, ny) * nx + wrapi(i + di, nx);
                    const double* blk = M + (g * 9 + o) * 9;
                    for (int r = 0; r < 3; ++r)
                        for (int s = 0; s < 3; ++s) acc[r] += blk[r * 3 + s] * v[s * nn + h];
                }
            for (int r = 0; r < 3; ++r) out[r * nn + g] = acc[r];
        }
}

/* A v = v + (theta dt)^2 curl_n curl_c v + theta dt M v  (step 6) */
void orc_apply_A(const orc_config* c, const double* M, const double* v, double* out)
{
    int64_t nn = (int64_t)c->nx * c->ny;
    double* cc = (double*)malloc(sizeof(double) * 3 * nn);
    double* cn = (double*)malloc(sizeof(double) * 3 * nn);
    double* mv = (double*)malloc(sizeof(double) * 3 * nn);
    double td = c->theta * c->dt;
    orc_curl_c(c, v, cc);
    orc_curl_n(c, cc, cn);
    orc_apply_M(c, M, v, mv);
    for (int64_t k = 0; k < 3 * nn; ++k) out[k] = v[k] + td * td * cn[k] + td * mv[k];
    free(cc);
    free(cn);
    free(mv);
}

/* b = E^n + theta dt curl_n B^n - theta dt Jhat */
void orc_rhs(const orc_config* c, const double* E, const double* B, const double* J, double* b)
{
    int64_t nn = (int64_t)c->nx * c->ny;
    double td = c->theta * c->dt;
    double* cn = (double*)malloc(sizeof(double) * 3 * nn);
    orc_curl_n(c, B, cn);
    for (int64_t k = 0; k < 3 * nn; ++k) b[k] = E[k] + td * cn[k] - td * J[k];
    free(cn);
}

static double dot(int64_t n, const double* a, const double* b)
{
    double s = 0.0;
    for (int64_t k = 0; k < n; ++k) s += a[k] * b[k];
    return s;
}

/* Restarted GMRES(m) with modified Gram-Schmidt and Givens rotations
   (the textbook algorithm). x holds the initial guess on entry. Stops when
   ||b - A x|| <= tol ||b|| or after maxit Arnoldi steps. Returns 0 when
   converged, 1 otherwise; *relres is the true relative residual. */
int orc_gmres(const orc_config* c, const double* M, const double* b, double* x,
              int* iters, double* relres)
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
    double bnorm = sqrt(dot(n, b, b));
    if (bnorm == 0.0) {
        memset(x, 0, sizeof(double) * n);
        *iters = 0;
        *relres = 0.0;
        status = 0;
        goto done;
    }
    for (;;) {
        orc_apply_A(c, M, x, w);
        for (int64_t k = 0; k < n; ++k) r[k] = b[k] - w[k];
        double beta = sqrt(dot(n, r, r));
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
            double* vj = V + (int64_t)j * n;
            orc_apply_A(c, M, vj, w);
            for (int i = 0; i <= j; ++i) {
                double* vi = V + (int64_t)i * n;
                double h = dot(n, w, vi);
                H[i * m + j] = h;
                for (int64_t k = 0; k < n; ++k) w[k] -= h * vi[k];
            }
            double hn = sqrt(dot(n, w, w));
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

/* Steps 7 and 8. */
void orc_field_update(const orc_config* c, const double* Etheta, double* E, double* B)
{
    int64_t nn = (int64_t)c->nx * c->ny;
    double th = c->theta;
    double* cc = (double*)malloc(sizeof(double) * 3 * nn);
    orc_curl_c(c, Etheta, cc);
    for (int64_t k = 0; k < 3 * nn; ++k) {
        E[k] = (Etheta[k] - (1.0 - th) * E[k]) / th;
        B[k] = B[k] - c->dt * cc[k];
    }
    free(cc);
}

static double wrap_pos(double s, double L)
{
    double t = s - L * floor(s / L);
    if (t >= L) t = 0.0;
    if (t < 0.0) t = 0.0;
    return t;
}

/* Steps 9 and 10, plus the per-particle energy sums of the ledger. */
void orc_push(const orc_config* c, const int64_t* off,
              double* x, double* y, double* ux, double* uy, double* uz,
              const double* w, const double* Etheta, const double* B, const double* E,
              double sums[4])
{
    double Lx = c->nx * c->dx, Ly = c->ny * c->dy;
    for (int k = 0; k < 4; ++k) sums[k] = 0.0;
    for (int s = 0; s < c->nspecies; ++s) {
        double q = c->q[s], m = c->m[s];
        double beta = q * c->dt / (2.0 * m);
        for (int64_t p = off[s]; p < off[s + 1]; ++p) {
            double Ep[3], Bp[3], alpha[9];
            double u0[3] = {ux[p], uy[p], uz[p]};
            double Ep0[3] = {0.0, 0.0, 0.0};
            orc_gather_E(c, Etheta, x[p], y[p], Ep);
            orc_gather_B(c, B, x[p], y[p], Bp);
            if (c->gamma_pred) orc_gather_E(c, E, x[p], y[p], Ep0);
            double gbar = gbar_of(c, beta, E, x[p], y[p], u0);
            orc_alpha(beta, gbar, Bp, alpha);
            double wv[3], ub[3], u1[3];
            for (int k = 0; k < 3; ++k) wv[k] = u0[k] + beta * Ep[k];
            for (int r = 0; r < 3; ++r) {
                ub[r] = 0.0;
                for (int k = 0; k < 3; ++k) ub[r] += alpha[r * 3 + k] * wv[k];
            }
            for (int k = 0; k < 3; ++k) u1[k] = 2.0 * ub[k] - u0[k];
            double g1 = gamma_of(u1[0], u1[1], u1[2]);
            double ue = ub[0] * Ep[0] + ub[1] * Ep[1] + ub[2] * Ep[2];
            /* 2/(g0+g1) - 1/gbar with gbar = g0 equals (g0-g1)/(g0 (g0+g1)),
               and g0 - g1 = (u0-u1).(u0+u1)/(g0+g1) */
            double du = 0.0;
            for (int k = 0; k < 3; ++k) du += (u0[k] - u1[k]) * (u0[k] + u1[k]);
            double g01 = du / (gbar + g1);
            sums[0] += w[p] * m * gamma_m1(u0[0], u0[1], u0[2]);
            sums[1] += w[p] * m * gamma_m1(u1[0], u1[1], u1[2]);
            sums[2] += c->dt * w[p] * q * ue / gbar;
            if (!c->gamma_pred) {
                sums[3] += c->dt * w[p] * q * ue * g01 / (gbar * (gbar + g1));
            } else {
                /* 2/(g0+g1) - 1/gbar = ((gbar-g0) + (gbar-g1))/(gbar (g0+g1)),
                   each difference from squares: gbar^2 - g^2 = |u*|^2 - |u|^2 */
                double g0 = gamma_of(u0[0], u0[1], u0[2]);
                double d0 = 0.0, d1 = 0.0;
                for (int k = 0; k < 3; ++k) {
                    double us = u0[k] + beta * (Ep0[k]);
                    d0 += (us - u0[k]) * (us + u0[k]);
                    d1 += (us - u1[k]) * (us + u1[k]);
                }
                double diff = d0 / (gbar + g0) + d1 / (gbar + g1);
                sums[3] += c->dt * w[p] * q * ue * diff / (gbar * (g0 + g1));
            }
            ux[p] = u1[0];
            uy[p] = u1[1];
            uz[p] = u1[2];
            x[p] = wrap_pos(x[p] + c->dt * u1[0] / g1, Lx);
            y[p] = wrap_pos(y[p] + c->dt * u1[1] / g1, Ly);
        }
    }
}

void orc_energies(const orc_config* c, const int64_t* off, const double* ux,
                  const double* uy, const double* uz, const double* w,
                  const double* E, const double* B, double out[3])
{
    int64_t nn = (int64_t)c->nx * c->ny;
    double dV = c->dx * c->dy;
    out[0] = 0.5 * dV * dot(3 * nn, E, E);
    out[1] = 0.5 * dV * dot(3 * nn, B, B);
    out[2] = 0.0;
    for (int s = 0; s < c->nspecies; ++s)
        for (int64_t p = off[s]; p < off[s + 1]; ++p)
            out[2] += w[p] * c->m[s] * gamma_m1(ux[p], uy[p], uz[p]);
}

void orc_cell_keys(const orc_config* c, int64_t n, const double* x, const double* y,
                   int32_t* keys)
{
    for (int64_t p = 0; p < n; ++p) {
        int64_t i, j;
        double f;
        locate(x[p], c->dx, c->nx, &i, &f);
        locate(y[p], c->dy, c->ny, &j, &f);
        keys[p] = (int32_t)(j * c->nx + i);
    }
}

/* Stable counting sort: histogram, exclusive scan, in-order placement. */
void orc_stable_sort(int64_t n, const int32_t* keys, int32_t nkeys, int64_t* perm,
                     int64_t* start)
{
    int64_t* cursor = (int64_t*)calloc((size_t)nkeys, sizeof(int64_t));
    memset(start, 0, sizeof(int64_t) * ((size_t)nkeys + 1));
    for (int64_t p = 0; p < n; ++p) start[keys[p] + 1]++;
    for (int32_t k = 0; k < nkeys; ++k) start[k + 1] += start[k];
    for (int64_t p = 0; p < n; ++p) {
        int32_t k = keys[p];
        perm[start[k] + cursor[k]++] = p;
    }
    free(cursor);
}

int orc_step(const orc_config* c, const int64_t* off,
             double* x, double* y, double* ux, double* uy, double* uz, const double* w,
             double* E, double* B, orc_ledger* led,
             double* J_out, double* M_out, double* Etheta_out)
{
    int64_t nn = (int64_t)c->nx * c->ny;
    double dV = c->dx * c->dy;
    double* J = (double*)malloc(sizeof(double) * 3 * nn);
    double* M = (double*)malloc(sizeof(double) * 81 * nn);
    double* b = (double*)malloc(sizeof(double) * 3 * nn);
    double* Et = (double*)malloc(sizeof(double) * 3 * nn);
    double* E0 = (double*)malloc(sizeof(double) * 3 * nn);
    double* B0 = (double*)malloc(sizeof(double) * 3 * nn);
    double* Jbar = (double*)malloc(sizeof(double) * 3 * nn);
    double en0[3], en1[3], sums[4];
    orc_energies(c, off, ux, uy, uz, w, E, B, en0);
    memcpy(E0, E, sizeof(double) * 3 * nn);
    memcpy(B0, B, sizeof(double) * 3 * nn);

    orc_deposit(c, off, x, y, ux, uy, uz, w, B, E, J, M);       /* steps 1-5 */
    orc_rhs(c, E, B, J, b);                                      /* step 6 */
    memcpy(Et, E, sizeof(double) * 3 * nn);
    int iters = 0;
    double relres = 0.0;
    int st = orc_gmres(c, M, b, Et, &iters, &relres);
    orc_field_update(c, Et, E, B);                               /* steps 7-8 */
    orc_push(c, off, x, y, ux, uy, uz, w, Et, B0, E0, sums);     /* steps 9-10 */
    orc_energies(c, off, ux, uy, uz, w, E, B, en1);

    if (led) {
        orc_apply_M(c, M, Et, Jbar);
        for (int64_t k = 0; k < 3 * nn; ++k) Jbar[k] += J[k];
        double dE2 = 0.0, dB2 = 0.0;
        for (int64_t k = 0; k < 3 * nn; ++k) {
            dE2 += (E[k] - E0[k]) * (E[k] - E0[k]);
            dB2 += (B[k] - B0[k]) * (B[k] - B0[k]);
        }
        led->W_E0 = en0[0]; led->W_B0 = en0[1]; led->K0 = en0[2];
        led->W_E1 = en1[0]; led->W_B1 = en1[1]; led->K1 = en1[2];
        led->work_grid = c->dt * dV * dot(3 * nn, Jbar, Et);
        led->work_particles = sums[2];
        led->mismatch = sums[3];
        led->dissipation = (c->theta - 0.5) * dV * (dE2 + dB2);
        led->residual = (en1[0] + en1[1] + en1[2]) - (en0[0] + en0[1] + en0[2])
                        - led->mismatch + led->dissipation;
        led->gmres_iters = iters;
        led->gmres_relres = relres;
    }
    if (J_out) memcpy(J_out, J, sizeof(double) * 3 * nn);
    if (M_out) memcpy(M_out, M, sizeof(double) * 81 * nn);
    if (Etheta_out) memcpy(Etheta_out, Et, sizeof(double) * 3 * nn);
    free(J); free(M); free(b); free(Et); free(E0); free(B0); free(Jbar);
    return st;
}
