/*
 * relsim_oracle.h -- declarations of the plain FP64 CPU oracle.
 *
 * TEST INFRASTRUCTURE ONLY. This oracle is a slow, loop-by-loop restatement
 * of one step of the relativistic semi-implicit particle-in-cell method
 * (RelSIM, Sec. 2 "Methods and Simulation Setup": explicit particle pusher,
 * implicit field solve through a mass-matrix formulation). Only the tests,
 * the smoke check and the benchmark's CPU-baseline leg may build, load or run
 * it. It shares no code, header, table or helper with the CUDA library.
 *
 * Units: rationalised, c = 1. Grid: periodic nx x ny, node (i,j) at
 * (i dx, j dy) carries E, J and the mass matrix; cell centre (i+1/2, j+1/2)
 * carries B. Node and cell (i,j) both have linear index j*nx + i.
 * Field arrays are component-major: F[k*ncell + idx], k = x, y, z.
 * Particles of all species are concatenated; species s owns the index range
 * [off[s], off[s+1]). Positions are absolute, in [0, nx dx) x [0, ny dy).
 * The mass matrix is stored for all nine neighbour offsets:
 * M[((g*9 + o)*3 + r)*3 + s] with o = (dj+1)*3 + (di+1) for node g+(di,dj);
 * block (r,s) maps component s of E at node g+o to component r of J at g.
 */
#ifndef RELSIM_ORACLE_H
#define RELSIM_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
    int nx, ny;
    double dx, dy, dt, theta;
    int nspecies;
    double q[4], m[4];
    double gmres_tol;
    int gmres_restart, gmres_maxit;
    int gamma_pred;   /* 0: gbar = gamma(u^n); 1: gbar = gamma(u^n + beta E^n(x)) */
} orc_config;

typedef struct {
    /* energies before (0) and after (1) the step */
    double W_E0, W_B0, K0, W_E1, W_B1, K1;
    /* dt dV sum_g Jbar_g . E_g^{n+theta} (field side of the work)        */
    double work_grid;
    /* dt sum_p w q (ubar/gbar) . E_p    (particle side of the same work) */
    double work_particles;
    /* dt sum_p w q ubar.E_p [2/(g0+g1) - 1/gbar]  (relativistic mismatch) */
    double mismatch;
    /* (theta - 1/2) dV (sum |E1-E0|^2 + sum |B1-B0|^2)  (theta-scheme loss) */
    double dissipation;
    /* (W1 + K1) - (W0 + K0) - mismatch + dissipation: zero up to the solve
       residual and round-off */
    double residual;
    int gmres_iters;
    double gmres_relres;
} orc_ledger;

int    orc_version(void);

/* shape functions and gathers */
void   orc_node_weights(const orc_config* c, double x, double y, int64_t g[4], double W[4]);
void   orc_gather_E(const orc_config* c, const double* E, double x, double y, double out[3]);
void   orc_gather_B(const orc_config* c, const double* B, double x, double y, double out[3]);
void   orc_alpha(double beta, double gbar, const double Bp[3], double alpha[9]);

/* deposit of predicted current Jhat[3*ncell] and mass matrix M[ncell*81];
   E (E^n) is read only with gamma_pred */
void   orc_deposit(const orc_config* c, const int64_t* off,
                   const double* x, const double* y,
                   const double* ux, const double* uy, const double* uz,
                   const double* w, const double* B, const double* E, double* J, double* M);

/* discrete curls and the implicit operator */
void   orc_curl_c(const orc_config* c, const double* E, double* out);
void   orc_curl_n(const orc_config* c, const double* B, double* out);
void   orc_apply_M(const orc_config* c, const double* M, const double* v, double* out);
void   orc_apply_A(const orc_config* c, const double* M, const double* v, double* out);
void   orc_rhs(const orc_config* c, const double* E, const double* B, const double* J, double* b);
int    orc_gmres(const orc_config* c, const double* M, const double* b, double* x,
                 int* iters, double* relres);
void   orc_field_update(const orc_config* c, const double* Etheta, double* E, double* B);

/* explicit push; sums[4] = {K0, K1, work_particles, mismatch}; E (E^n) is
   read only with gamma_pred */
void   orc_push(const orc_config* c, const int64_t* off,
                double* x, double* y, double* ux, double* uy, double* uz,
                const double* w, const double* Etheta, const double* B, const double* E,
                double sums[4]);

/* energies of a state: out[0] = W_E, out[1] = W_B, out[2] = K */
void   orc_energies(const orc_config* c, const int64_t* off, const double* ux,
                    const double* uy, const double* uz, const double* w,
                    const double* E, const double* B, double out[3]);

/* stable counting sort: keys in [0, nkeys); perm[k] = index of the k-th
   element in sorted order; start[nkeys+1] = bucket starts */
void   orc_cell_keys(const orc_config* c, int64_t n, const double* x, const double* y,
                     int32_t* keys);
void   orc_stable_sort(int64_t n, const int32_t* keys, int32_t nkeys, int64_t* perm,
                       int64_t* start);

/* one full step; J, M, Etheta may be NULL (else receive the step's values) */
int    orc_step(const orc_config* c, const int64_t* off,
                double* x, double* y, double* ux, double* uy, double* uz, const double* w,
                double* E, double* B, orc_ledger* led,
                double* J_out, double* M_out, double* Etheta_out);

/* ---- 2D with quadratic (TSC) shapes (relsim_oracle_q.c): a particle
   touches 3 x 3 nodes; M for all 25 offsets, M[((g*25 + o)*3 + r)*3 + s]
   with o = (dj+2)*5 + (di+2). Curls, rhs, field update, energies: the 2D
   functions above. Base scheme. */
void   orcq_node_weights(const orc_config* c, double x, double y, int64_t g[9], double W[9]);
void   orcq_gather_E(const orc_config* c, const double* E, double x, double y, double out[3]);
void   orcq_gather_B(const orc_config* c, const double* B, double x, double y, double out[3]);
void   orcq_deposit(const orc_config* c, const int64_t* off, const double* x, const double* y,
                    const double* ux, const double* uy, const double* uz, const double* w, const double* B,
                    double* J, double* M);
void   orcq_apply_M(const orc_config* c, const double* M, const double* v, double* out);
void   orcq_apply_A(const orc_config* c, const double* M, const double* v, double* out);
int    orcq_gmres(const orc_config* c, const double* M, const double* b, double* x, int* iters,
                  double* relres);
void   orcq_push(const orc_config* c, const int64_t* off, double* x, double* y, double* ux, double* uy,
                 double* uz, const double* w, const double* Etheta, const double* B, double sums[4]);
int    orcq_step(const orc_config* c, const int64_t* off, double* x, double* y, double* ux, double* uy,
                 double* uz, const double* w, double* E, double* B, orc_ledger* led, double* J_out,
                 double* M_out, double* Etheta_out);

/* ---- 3D (relsim_oracle3.c): periodic nx x ny x nz, trilinear shapes, the
   base scheme. Node and cell (i,j,k) have linear index (k*ny + j)*nx + i;
   M[((g*27 + o)*3 + r)*3 + s] with o = (dk+1)*9 + (dj+1)*3 + (di+1). */
typedef struct {
    int nx, ny, nz;
    double dx, dy, dz, dt, theta;
    int nspecies;
    double q[4], m[4];
    double gmres_tol;
    int gmres_restart, gmres_maxit;
} orc3_config;

void   orc3_node_weights(const orc3_config* c, double x, double y, double z, int64_t g[8], double W[8]);
void   orc3_gather_E(const orc3_config* c, const double* E, double x, double y, double z, double out[3]);
void   orc3_gather_B(const orc3_config* c, const double* B, double x, double y, double z, double out[3]);
void   orc3_deposit(const orc3_config* c, const int64_t* off, const double* x, const double* y, const double* z,
                    const double* ux, const double* uy, const double* uz, const double* w, const double* B,
                    double* J, double* M);
void   orc3_curl_c(const orc3_config* c, const double* E, double* out);
void   orc3_curl_n(const orc3_config* c, const double* B, double* out);
void   orc3_apply_M(const orc3_config* c, const double* M, const double* v, double* out);
void   orc3_apply_A(const orc3_config* c, const double* M, const double* v, double* out);
void   orc3_rhs(const orc3_config* c, const double* E, const double* B, const double* J, double* b);
int    orc3_gmres(const orc3_config* c, const double* M, const double* b, double* x, int* iters,
                  double* relres);
void   orc3_field_update(const orc3_config* c, const double* Etheta, double* E, double* B);
void   orc3_push(const orc3_config* c, const int64_t* off, double* x, double* y, double* z, double* ux,
                 double* uy, double* uz, const double* w, const double* Etheta, const double* B, double sums[4]);
void   orc3_energies(const orc3_config* c, const int64_t* off, const double* ux, const double* uy,
                     const double* uz, const double* w, const double* E, const double* B, double out[3]);
void   orc3_cell_keys(const orc3_config* c, int64_t n, const double* x, const double* y, const double* z,
                      int32_t* keys);
int    orc3_step(const orc3_config* c, const int64_t* off, double* x, double* y, double* z, double* ux,
                 double* uy, double* uz, const double* w, double* E, double* B, orc_ledger* led,
                 double* J_out, double* M_out, double* Etheta_out);

#ifdef __cplusplus
}
#endif
#endif
