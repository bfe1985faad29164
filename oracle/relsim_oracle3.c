/*
 * relsim_oracle3.c -- the plain FP64 CPU oracle of one RelSIM step in 3D.
 *
 * TEST INFRASTRUCTURE ONLY (see relsim_oracle.h): the tests and the
 * benchmark's CPU-baseline leg are its only users; the CUDA library never
 * links or calls it.
 *
 * The same scheme as the 2D oracle (relsim_oracle.c, steps 1-10 of its
 * header: Sec. 2's explicit pusher, implicit field solve and mass-matrix
 * formulation), written out on a periodic nx x ny x nz grid with trilinear
 * (CIC) shape functions: a particle touches the 8 nodes of its cell, so its
 * mass-matrix contributions couple node pairs up to one cell apart in each
 * direction (27 neighbour offsets, the 27-node stencil), and B is gathered
 * from the 8 cell centres around it. The base scheme only (gbar = gamma(u^n)).
 *
 * Layout: node (i,j,k) at (i dx, j dy, k dz) and the cell centre at
 * (i+1/2, j+1/2, k+1/2) cells share the linear index (k*ny + j)*nx + i.
 * Fields are component-major F[c*nn + idx]. The mass matrix is stored for
 * all 27 offsets: M[((g*27 + o)*3 + r)*3 + s] with
 * o = (dk+1)*9 + (dj+1)*3 + (di+1) for node g + (di,dj,dk).
 *
 * Discrete curls (the 3D counterparts of the 2D oracle's): a derivative
 * node -> centre differences the cell's node values along its direction and
 * averages the 4 edges of the cell in that direction; centre -> node
 * differences the 8 centres around the node and averages likewise.
 */
#include "relsim_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

static int64_t wrap3(int64_t i, int64_t n)
{
    i %= n;
    return i < 0 ? i + n : i;
}

static int64_t nn3(const orc3_config* c) { return (int64_t)c->nx * c->ny * c->nz; }

static int64_t idx3(const orc3_config* c, int64_t i, int64_t j, int64_t k)
{
    return (wrap3(k, c->nz) * c->ny + wrap3(j, c->ny)) * c->nx + wrap3(i, c->nx);
}

static void locate3(double s, double d, int n, int64_t* i, double* f)
{
    double t = s / d;
    double fl = floor(t);
    *f = t - fl;
    *i = wrap3((int64_t)fl, n);
}

/* The 8 nodes of the cell holding the point, with their trilinear weights;
   node a = (a&1, (a>>1)&1, (a>>2)&1) relative to the cell's lower corner.
   cell[3] receives the cell's (i, j, k). */
static void weights3(const orc3_config* c, double x, double y, double z, double sx, int64_t cell[3],
                     int64_t g[8], double W[8])
{
    double f[3];
    locate3(x - sx * c->dx, c->dx, c->nx, &cell[0], &f[0]);
    locate3(y - sx * c->dy, c->dy, c->ny, &cell[1], &f[1]);
    locate3(z - sx * c->dz, c->dz, c->nz, &cell[2], &f[2]);
    for (int a = 0; a < 8; ++a) {
        int ax = a & 1, ay = (a >> 1) & 1, az = (a >> 2) & 1;
        g[a] = idx3(c, cell[0] + ax, cell[1] + ay, cell[2] + az);
        W[a] = (ax ? f[0] : 1.0 - f[0]) * (ay ? f[1] : 1.0 - f[1]) * (az ? f[2] : 1.0 - f[2]);
    }
}

void orc3_node_weights(const orc3_config* c, double x, double y, double z, int64_t g[8], double W[8])
{
    int64_t cell[3];
    weights3(c, x, y, z, 0.0, cell, g, W);
}

void orc3_gather_E(const orc3_config* c, const double* E, double x, double y, double z, double out[3])
{
    int64_t g[8], cell[3];
    double W[8];
    int64_t nn = nn3(c);
    weights3(c, x, y, z, 0.0, cell, g, W);
    for (int k = 0; k < 3; ++k) {
        out[k] = 0.0;
        for (int a = 0; a < 8; ++a) out[k] += W[a] * E[k * nn + g[a]];
    }
}

/* centres at (i+1/2, j+1/2, k+1/2): the same weights on the lattice shifted
   by half a cell */
void orc3_gather_B(const orc3_config* c, const double* B, double x, double y, double z, double out[3])
{
    int64_t g[8], cell[3];
    double W[8];
    int64_t nn = nn3(c);
    weights3(c, x, y, z, 0.5, cell, g, W);
    for (int k = 0; k < 3; ++k) {
        out[k] = 0.0;
        for (int a = 0; a < 8; ++a) out[k] += W[a] * B[k * nn + g[a]];
    }
}

static double gamma3(const double u[3]) { return sqrt(1.0 + u[0] * u[0] + u[1] * u[1] + u[2] * u[2]); }

static double gamma3_m1(const double u[3])
{
    double u2 = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    return u2 / (sqrt(1.0 + u2) + 1.0);
}

/* Steps 1-5: Jhat[3 nn] and M[27*9 nn] from x^{n+1/2}, u^n, B^n. Node a and
   node b of one cell sit (bx-ax, by-ay, bz-az) apart. */
void orc3_deposit(const orc3_config* c, const int64_t* off, const double* x, const double* y, const double* z,
                  const double* ux, const double* uy, const double* uz, const double* w, const double* B,
                  double* J, double* M)
{
    int64_t nn = nn3(c);
    double dV = c->dx * c->dy * c->dz;
    memset(J, 0, sizeof(double) * 3 * nn);
    memset(M, 0, sizeof(double) * 243 * nn);
    for (int s = 0; s < c->nspecies; ++s) {
        double q = c->q[s], m = c->m[s];
        double beta = q * c->dt / (2.0 * m);
        for (int64_t p = off[s]; p < off[s + 1]; ++p) {
            double Bp[3], alpha[9], u[3] = {ux[p], uy[p], uz[p]};
            orc3_gather_B(c, B, x[p], y[p], z[p], Bp);
            double gbar = gamma3(u);
            orc_alpha(beta, gbar, Bp, alpha);
            double vJ[3];
            for (int r = 0; r < 3; ++r) {
                vJ[r] = 0.0;
                for (int k = 0; k < 3; ++k) vJ[r] += alpha[r * 3 + k] * u[k];
                vJ[r] /= gbar;
            }
            int64_t g[8], cell[3];
            double W[8];
            weights3(c, x[p], y[p], z[p], 0.0, cell, g, W);
            double cJ = w[p] * q / dV;
            double cM = w[p] * q * beta / (gbar * dV);
            for (int a = 0; a < 8; ++a) {
                for (int k = 0; k < 3; ++k) J[k * nn + g[a]] += cJ * W[a] * vJ[k];
                for (int b = 0; b < 8; ++b) {
                    int di = (b & 1) - (a & 1), dj = ((b >> 1) & 1) - ((a >> 1) & 1);
                    int dk = ((b >> 2) & 1) - ((a >> 2) & 1);
                    int o = (dk + 1) * 9 + (dj + 1) * 3 + (di + 1);
                    double* blk = M + (g[a] * 27 + o) * 9;
                    for (int rs = 0; rs < 9; ++rs) blk[rs] += cM * W[a] * W[b] * alpha[rs];
                }
            }
        }
    }
}

/* node -> centre curl */
void orc3_curl_c(const orc3_config* c, const double* E, double* out)
{
    int64_t nn = nn3(c);
    for (int k = 0; k < c->nz; ++k)
        for (int j = 0; j < c->ny; ++j)
            for (int i = 0; i < c->nx; ++i) {
                double d[3][3];   /* d[axis][component]: derivative along axis */
                for (int comp = 0; comp < 3; ++comp) {
                    const double* f = E + comp * nn;
                    double sx = 0.0, sy = 0.0, sz = 0.0;
                    for (int e1 = 0; e1 < 2; ++e1)
                        for (int e2 = 0; e2 < 2; ++e2) {
                            sx += f[idx3(c, i + 1, j + e1, k + e2)] - f[idx3(c, i, j + e1, k + e2)];
                            sy += f[idx3(c, i + e1, j + 1, k + e2)] - f[idx3(c, i + e1, j, k + e2)];
                            sz += f[idx3(c, i + e1, j + e2, k + 1)] - f[idx3(c, i + e1, j + e2, k)];
                        }
                    d[0][comp] = sx / (4.0 * c->dx);
                    d[1][comp] = sy / (4.0 * c->dy);
                    d[2][comp] = sz / (4.0 * c->dz);
                }
                int64_t g = idx3(c, i, j, k);
                out[g] = d[1][2] - d[2][1];
                out[nn + g] = d[2][0] - d[0][2];
                out[2 * nn + g] = d[0][1] - d[1][0];
            }
}

/* centre -> node curl over the 8 centres (i-1..i, j-1..j, k-1..k) */
void orc3_curl_n(const orc3_config* c, const double* B, double* out)
{
    int64_t nn = nn3(c);
    for (int k = 0; k < c->nz; ++k)
        for (int j = 0; j < c->ny; ++j)
            for (int i = 0; i < c->nx; ++i) {
                double d[3][3];
                for (int comp = 0; comp < 3; ++comp) {
                    const double* f = B + comp * nn;
                    double sx = 0.0, sy = 0.0, sz = 0.0;
                    for (int e1 = -1; e1 <= 0; ++e1)
                        for (int e2 = -1; e2 <= 0; ++e2) {
                            sx += f[idx3(c, i, j + e1, k + e2)] - f[idx3(c, i - 1, j + e1, k + e2)];
                            sy += f[idx3(c, i + e1, j, k + e2)] - f[idx3(c, i + e1, j - 1, k + e2)];
                            sz += f[idx3(c, i + e1, j + e2, k)] - f[idx3(c, i + e1, j + e2, k - 1)];
                        }
                    d[0][comp] = sx / (4.0 * c->dx);
                    d[1][comp] = sy / (4.0 * c->dy);
                    d[2][comp] = sz / (4.0 * c->dz);
                }
                int64_t g = idx3(c, i, j, k);
                out[g] = d[1][2] - d[2][1];
                out[nn + g] = d[2][0] - d[0][2];
                out[2 * nn + g] = d[0][1] - d[1][0];
            }
}

/* (M v)_g = sum_o M[g][o] v_{g+o} */
void orc3_apply_M(const orc3_config* c, const double* M, const double* v, double* out)
{
    int64_t nn = nn3(c);
    for (int k = 0; k < c->nz; ++k)
        for (int j = 0; j < c->ny; ++j)
            for (int i = 0; i < c->nx; ++i) {
                int64_t g = idx3(c, i, j, k);
                double acc[3] = {0.0, 0.0, 0.0};
                for (int dk = -1; dk <= 1; ++dk)
                    for (int dj = -1; dj <= 1; ++dj)
                        for (int di = -1; di <= 1; ++di) {
                            int o = (dk + 1) * 9 + (dj + 1) * 3 + (di + 1);
                            int64_t h = idx3(c, i + di, j + dj, k + dk);
                            const double* blk = M + (g * 27 + o) * 9;
                            for (int r = 0; r < 3; ++r)
                                for (int s = 0; s < 3; ++s) acc[r] += blk[r * 3 + s] * v[s * nn + h];
                        }
                for (int r = 0; r < 3; ++r) out[r * nn + g] = acc[r];
            }
}

void orc3_apply_A(const orc3_config* c, const double* M, const double* v, double* out)
{
    int64_t nn = nn3(c);
    double* cc = (double*)malloc(sizeof(double) * 3 * nn);
    double* cn = (double*)malloc(sizeof(double) * 3 * nn);
    double* mv = (double*)malloc(sizeof(double) * 3 * nn);
    double td = c->theta * c->dt;
    orc3_curl_c(c, v, cc);
    orc3_curl_n(c, cc, cn);
    orc3_apply_M(c, M, v, mv);
    for (int64_t k = 0; k < 3 * nn; ++k) out[k] = v[k] + td * td * cn[k] + td * mv[k];
    free(cc);
    free(cn);
    free(mv);
}

void orc3_rhs(const orc3_config* c, const double* E, const double* B, const double* J, double* b)
{
    int64_t nn = nn3(c);
    double td = c->theta * c->dt;
    double* cn = (double*)malloc(sizeof(double) * 3 * nn);
    orc3_curl_n(c, B, cn);
    for (int64_t k = 0; k < 3 * nn; ++k) b[k] = E[k] + td * cn[k] - td * J[k];
    free(cn);
}

static double dot3(int64_t n, const double* a, const double* b)
{
    double s = 0.0;
    for (int64_t k = 0; k < n; ++k) s += a[k] * b[k];
    return s;
}

/* Restarted GMRES(m), modified Gram-Schmidt, Givens rotations (the textbook
   algorithm, as in the 2D oracle), on the 3D operator. */
int orc3_gmres(const orc3_config* c, const double* M, const double* b, double* x, int* iters, double* relres)
{
    int64_t n = 3 * nn3(c);
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
    double bnorm = sqrt(dot3(n, b, b));
    if (bnorm == 0.0) {
        memset(x, 0, sizeof(double) * n);
        *iters = 0;
        *relres = 0.0;
        status = 0;
        goto done;
    }
    for (;;) {
        orc3_apply_A(c, M, x, w);
        for (int64_t k = 0; k < n; ++k) r[k] = b[k] - w[k];
        double beta = sqrt(dot3(n, r, r));
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
            orc3_apply_A(c, M, V + (int64_t)j * n, w);
            for (int i = 0; i <= j; ++i) {
                double* vi = V + (int64_t)i * n;
                double h = dot3(n, w, vi);
                H[i * m + j] = h;
                for (int64_t k = 0; k < n; ++k) w[k] -= h * vi[k];
            }
            double hn = sqrt(dot3(n, w, w));
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

void orc3_field_update(const orc3_config* c, const double* Etheta, double* E, double* B)
{
    int64_t nn = nn3(c);
    double th = c->theta;
    double* cc = (double*)malloc(sizeof(double) * 3 * nn);
    orc3_curl_c(c, Etheta, cc);
    for (int64_t k = 0; k < 3 * nn; ++k) {
        E[k] = (Etheta[k] - (1.0 - th) * E[k]) / th;
        B[k] = B[k] - c->dt * cc[k];
    }
    free(cc);
}

static double wrap_pos3(double s, double L)
{
    double t = s - L * floor(s / L);
    if (t >= L) t = 0.0;
    if (t < 0.0) t = 0.0;
    return t;
}

/* Steps 9 and 10 and the ledger's particle sums {K0, K1, work, mismatch}. */
void orc3_push(const orc3_config* c, const int64_t* off, double* x, double* y, double* z, double* ux, double* uy,
               double* uz, const double* w, const double* Etheta, const double* B, double sums[4])
{
    double L[3] = {c->nx * c->dx, c->ny * c->dy, c->nz * c->dz};
    for (int k = 0; k < 4; ++k) sums[k] = 0.0;
    for (int s = 0; s < c->nspecies; ++s) {
        double q = c->q[s], m = c->m[s];
        double beta = q * c->dt / (2.0 * m);
        for (int64_t p = off[s]; p < off[s + 1]; ++p) {
            double Ep[3], Bp[3], alpha[9];
            double u0[3] = {ux[p], uy[p], uz[p]};
            orc3_gather_E(c, Etheta, x[p], y[p], z[p], Ep);
            orc3_gather_B(c, B, x[p], y[p], z[p], Bp);
            double gbar = gamma3(u0);
            orc_alpha(beta, gbar, Bp, alpha);
            double wv[3], ub[3], u1[3];
            for (int k = 0; k < 3; ++k) wv[k] = u0[k] + beta * Ep[k];
            for (int r = 0; r < 3; ++r) {
                ub[r] = 0.0;
                for (int k = 0; k < 3; ++k) ub[r] += alpha[r * 3 + k] * wv[k];
            }
            for (int k = 0; k < 3; ++k) u1[k] = 2.0 * ub[k] - u0[k];
            double g1 = gamma3(u1);
            double ue = ub[0] * Ep[0] + ub[1] * Ep[1] + ub[2] * Ep[2];
            double du = 0.0;
            for (int k = 0; k < 3; ++k) du += (u0[k] - u1[k]) * (u0[k] + u1[k]);
            double g01 = du / (gbar + g1);
            sums[0] += w[p] * m * gamma3_m1(u0);
            sums[1] += w[p] * m * gamma3_m1(u1);
            sums[2] += c->dt * w[p] * q * ue / gbar;
            sums[3] += c->dt * w[p] * q * ue * g01 / (gbar * (gbar + g1));
            ux[p] = u1[0];
            uy[p] = u1[1];
            uz[p] = u1[2];
            x[p] = wrap_pos3(x[p] + c->dt * u1[0] / g1, L[0]);
            y[p] = wrap_pos3(y[p] + c->dt * u1[1] / g1, L[1]);
            z[p] = wrap_pos3(z[p] + c->dt * u1[2] / g1, L[2]);
        }
    }
}

void orc3_energies(const orc3_config* c, const int64_t* off, const double* ux, const double* uy, const double* uz,
                   const double* w, const double* E, const double* B, double out[3])
{
    int64_t nn = nn3(c);
    double dV = c->dx * c->dy * c->dz;
    out[0] = 0.5 * dV * dot3(3 * nn, E, E);
    out[1] = 0.5 * dV * dot3(3 * nn, B, B);
    out[2] = 0.0;
    for (int s = 0; s < c->nspecies; ++s)
        for (int64_t p = off[s]; p < off[s + 1]; ++p) {
            double u[3] = {ux[p], uy[p], uz[p]};
            out[2] += w[p] * c->m[s] * gamma3_m1(u);
        }
}

void orc3_cell_keys(const orc3_config* c, int64_t n, const double* x, const double* y, const double* z,
                    int32_t* keys)
{
    for (int64_t p = 0; p < n; ++p) {
        int64_t i, j, k;
        double f;
        locate3(x[p], c->dx, c->nx, &i, &f);
        locate3(y[p], c->dy, c->ny, &j, &f);
        locate3(z[p], c->dz, c->nz, &k, &f);
        keys[p] = (int32_t)((k * c->ny + j) * c->nx + i);
    }
}

int orc3_step(const orc3_config* c, const int64_t* off, double* x, double* y, double* z, double* ux, double* uy,
              double* uz, const double* w, double* E, double* B, orc_ledger* led, double* J_out, double* M_out,
              double* Etheta_out)
{
    int64_t nn = nn3(c);
    double dV = c->dx * c->dy * c->dz;
    double* J = (double*)malloc(sizeof(double) * 3 * nn);
    double* M = (double*)malloc(sizeof(double) * 243 * nn);
    double* b = (double*)malloc(sizeof(double) * 3 * nn);
    double* Et = (double*)malloc(sizeof(double) * 3 * nn);
    double* E0 = (double*)malloc(sizeof(double) * 3 * nn);
    double* B0 = (double*)malloc(sizeof(double) * 3 * nn);
    double* Jbar = (double*)malloc(sizeof(double) * 3 * nn);
    double en0[3], en1[3], sums[4];
    orc3_energies(c, off, ux, uy, uz, w, E, B, en0);
    memcpy(E0, E, sizeof(double) * 3 * nn);
    memcpy(B0, B, sizeof(double) * 3 * nn);

    orc3_deposit(c, off, x, y, z, ux, uy, uz, w, B, J, M);       /* steps 1-5 */
    orc3_rhs(c, E, B, J, b);                                      /* step 6 */
    memcpy(Et, E, sizeof(double) * 3 * nn);
    int iters = 0;
    double relres = 0.0;
    int st = orc3_gmres(c, M, b, Et, &iters, &relres);
    orc3_field_update(c, Et, E, B);                               /* steps 7-8 */
    orc3_push(c, off, x, y, z, ux, uy, uz, w, Et, B0, sums);      /* steps 9-10 */
    orc3_energies(c, off, ux, uy, uz, w, E, B, en1);

    if (led) {
        orc3_apply_M(c, M, Et, Jbar);
        for (int64_t k = 0; k < 3 * nn; ++k) Jbar[k] += J[k];
        double dE2 = 0.0, dB2 = 0.0;
        for (int64_t k = 0; k < 3 * nn; ++k) {
            dE2 += (E[k] - E0[k]) * (E[k] - E0[k]);
            dB2 += (B[k] - B0[k]) * (B[k] - B0[k]);
        }
        led->W_E0 = en0[0]; led->W_B0 = en0[1]; led->K0 = en0[2];
        led->W_E1 = en1[0]; led->W_B1 = en1[1]; led->K1 = en1[2];
        led->work_grid = c->dt * dV * dot3(3 * nn, Jbar, Et);
        led->work_particles = sums[2];
        led->mismatch = sums[3];
        led->dissipation = (c->theta - 0.5) * dV * (dE2 + dB2);
        led->residual = (en1[0] + en1[1] + en1[2]) - (en0[0] + en0[1] + en0[2]) - led->mismatch + led->dissipation;
        led->gmres_iters = iters;
        led->gmres_relres = relres;
    }
    if (J_out) memcpy(J_out, J, sizeof(double) * 3 * nn);
    if (M_out) memcpy(M_out, M, sizeof(double) * 243 * nn);
    if (Etheta_out) memcpy(Etheta_out, Et, sizeof(double) * 3 * nn);
    free(J); free(M); free(b); free(Et); free(E0); free(B0); free(Jbar);
    return st;
}
