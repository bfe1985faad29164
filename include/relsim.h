/*
 * relsim.h -- C ABI of the GB300 (sm_103a) RelSIM hot-path library.
 *
 * One time step of the relativistic semi-implicit particle-in-cell method
 * used in the paper (Sec. 2, "Methods and Simulation Setup": the particle
 * pusher is explicit, only the field solver is implicit, and the field
 * solver uses a mass-matrix formulation). A step is three calls, in order:
 *
 *   relsim_build_mass_matrix   gather B^n at x^{n+1/2}, build each
 *                              particle's rotation matrix alpha, deposit the
 *                              predicted current Jhat and the 3x3 mass
 *                              matrix blocks M_{g,g'} on the grid nodes
 *   relsim_field_solve         solve the implicit field equation for
 *                              E^{n+theta} (matrix-free GMRES), then advance
 *                              E^{n+1} and B^{n+1}
 *   relsim_push                push u^{n+1}, x^{n+3/2} with E^{n+theta} and
 *                              B^n, and re-sort the particles by cell
 *
 * followed, when wanted, by relsim_energy_ledger. relsim_step does all
 * four. The discrete equations (the paper cites them and does not print
 * them; these are the readings this library implements, rationalised
 * units with c = 1):
 *
 *   gbar  = sqrt(1 + |u^n|^2),  beta = q dt / (2 m),  a = beta B^n(x)/gbar
 *   alpha = (I - [a]x + a a^T)/(1 + |a|^2)
 *   Jhat_g = sum_p w q W_g(x) alpha u^n / gbar / dV
 *   M_gg'  = sum_p w q beta / gbar W_g(x) W_g'(x) alpha / dV
 *   (I + (theta dt)^2 curl_n curl_c + theta dt M) E^{n+theta}
 *        = E^n + theta dt curl_n B^n - theta dt Jhat
 *   E^{n+1} = (E^{n+theta} - (1 - theta) E^n)/theta
 *   B^{n+1} = B^n - dt curl_c E^{n+theta}
 *   ubar = alpha (u^n + beta E^{n+theta}(x)),  u^{n+1} = 2 ubar - u^n
 *   x^{n+3/2} = x^{n+1/2} + dt u^{n+1}/sqrt(1 + |u^{n+1}|^2)   (periodic)
 *
 * Grid: 2D, periodic, nx x ny. Node (i,j) sits at (i dx, j dy) and carries
 * E, Jhat and M; the cell centre (i+1/2, j+1/2) carries B. Node and cell
 * (i,j) both have the linear index j*nx + i. W is the linear (cloud-in-cell)
 * shape function. Requires nx, ny >= 3.
 *
 * Conventions for every entry point:
 * - Return value: RELSIM_OK (0) or a negative RELSIM_ERR_* code. Nothing
 *   aborts; relsim_last_error() returns a message owned by the context
 *   (valid until the next call on it).
 * - All work is enqueued on the CUDA stream given to relsim_init (0 means
 *   the legacy default stream). Calls that return data to the host
 *   (RELSIM_HOST outputs, relsim_field_solve's residual, the ledger)
 *   synchronise that stream; the others return without waiting.
 * - Buffers are owned by the caller. The library copies inputs (it never
 *   keeps a caller pointer) and owns its device buffers until
 *   relsim_destroy. "where" says whether a caller pointer is host memory
 *   (RELSIM_HOST) or device memory of the context's GPU (RELSIM_DEVICE).
 * - Field arrays are FP64, component-major: F[k*ncell + idx], k = x, y, z,
 *   ncell = nx*ny. Particle arrays are FP64: positions x[2n] interleaved
 *   (x_p, y_p) absolute in [0, nx dx) x [0, ny dy), momenta u[3n]
 *   interleaved (ux, uy, uz) with u = gamma v, weights w[n].
 * - Internally the FP32 form stores a position as cell index + FP32 offset
 *   and computes particles, fields and mass matrices in FP32, keeping FP64
 *   for the GMRES Krylov basis, its orthogonalisation and residual, and for
 *   the energy-ledger reductions. The FP64 form computes everything in FP64.
 */
#ifndef RELSIM_H
#define RELSIM_H

#include <stdint.h>

/* the library exports these entry points and nothing else */
#if defined(__GNUC__)
#define RELSIM_API __attribute__((visibility("default")))
#else
#define RELSIM_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

#define RELSIM_OK 0
#define RELSIM_ERR_INVALID_ARG (-1)   /* bad pointer, size, species or config   */
#define RELSIM_ERR_BAD_STATE (-2)     /* calls out of order (build/solve/push)  */
#define RELSIM_ERR_CUDA (-3)          /* a CUDA runtime error; see the message  */
#define RELSIM_ERR_OOM (-4)           /* device allocation failed               */
#define RELSIM_ERR_NOT_CONVERGED (-5) /* GMRES hit gmres_maxit; state advanced  */
#define RELSIM_ERR_NONFINITE (-6)     /* NaN/Inf found in inputs or results     */
#define RELSIM_ERR_TIMEOUT (-7)       /* a bounded device wait gave up          */
#define RELSIM_ERR_INTERNAL (-8)      /* an internal consistency check failed   */

#define RELSIM_HOST 0
#define RELSIM_DEVICE 1

typedef struct relsim_ctx relsim_ctx;  /* opaque, owned by the library */

typedef struct {
    int dim;               /* 2, or 3 for the 3D form (see below)              */
    int nx, ny, nz;        /* cells per direction (nz ignored in 2D)           */
    double dx, dy, dz;     /* cell sizes                                       */
    double dt;             /* time step                                        */
    double theta_implicit; /* theta in (0, 1]; 0.5 conserves energy            */
    int precision;         /* 32 (FP32 form) or 64 (FP64 form)                 */
    int nspecies;          /* 1..4                                             */
    double q[4], m[4];     /* charge and mass per species (m > 0)              */
    double gmres_tol;      /* relative residual target; 0 -> 1e-6 (FP32 form)
                              or 1e-10 (FP64 form)                             */
    int gmres_restart;     /* Krylov dimension per cycle; 0 -> 30 (max 100)    */
    int gmres_maxit;       /* total Arnoldi steps per solve; 0 -> 500          */
    int track_ids;         /* nonzero: carry an int32 id per particle (its load
                              index) through every sort, for tracking           */
    uint64_t seed;         /* reserved                                         */
    int gamma_pred;        /* 0: gbar = gamma(u^n) in alpha and M; 1: gbar =
                              gamma(u^n + beta E^n(x)), the Lorentz factor of
                              the predicted half-step momentum (E^n standing
                              in for E^{n+theta}), which shrinks the
                              relativistic energy error of a step          */
    int shape;             /* particle shape: 0 or 1 linear (CIC); 2 quadratic
                              (TSC, 2D base scheme only): 3 x 3 nodes per
                              particle, node pairs up to two cells apart, the
                              mass matrix stored for 13 offsets per node
                              ((0,0), (1,0), (2,0), (di,1) and (di,2) for
                              di = -2..2: ncell x 117); the re-sort is a
                              counting sort, as in 3D                     */
    int gmres_fp64;        /* the GMRES vectors (Krylov basis, iterate, right-
                              hand side) of the FP32 form of the 2D scheme
                              with linear shapes: 0 double-float pairs (two
                              FP32 numbers per value, about 48 significant
                              bits, arithmetic on the FP32 pipe: GB300's FP64
                              pipe issues at about 1/64 of the FP32 rate);
                              1 FP64. Other forms always use FP64 vectors  */
} relsim_config;

typedef struct {
    /* energies of the current state (after the last push or load) */
    double W_E, W_B, K, total;   /* 1/2 dV sum|E|^2, 1/2 dV sum|B|^2,
                                    sum w m (gamma - 1), their sum            */
    double K_species[4];
    /* terms of the last completed step (zero before the first step) */
    double W_E0, W_B0, K0;       /* energies at the start of that step          */
    double dW_E, dW_B, dK;       /* changes over the step, summed per element   */
    double work_grid;            /* dt dV sum_g (Jhat + M E^{n+theta}).E^{n+theta} */
    double work_particles;       /* dt sum_p w q (ubar/gbar).E^{n+theta}(x_p)    */
    double mismatch;             /* dt sum_p w q ubar.E [2/(g0+g1) - 1/gbar]     */
    double dissipation;          /* (theta - 1/2) dV (sum|dE|^2 + sum|dB|^2)     */
    double residual;             /* dW_E + dW_B + dK - mismatch + dissipation:
                                    zero up to the solve tolerance and round-off */
    int gmres_iters;
    int gmres_restarts;
    double gmres_relres;         /* true ||b - A E^{n+theta}|| / ||b||           */
    int64_t step;                /* completed steps since the last load          */
    int64_t n_particles;
} relsim_energy;

/* Create a context for one simulation on the current CUDA device.
   Paper: no counterpart (the context holds the state of the step of Sec. 2,
   "Methods and Simulation Setup"; the configuration's fields are that
   step's parameters).
   cfg: see relsim_config. cuda_stream: a cudaStream_t (or 0). On success
   *out receives the context. Errors: INVALID_ARG (bad config), CUDA, OOM.
   Allocates the grid arrays (fields, Jhat, M, GMRES basis) up front. */
RELSIM_API int relsim_init(const relsim_config* cfg, void* cuda_stream, relsim_ctx** out);

/* Free every device buffer of the context and the context itself (no
   counterpart in the paper). Safe on NULL. Synchronises the context's stream first. */
RELSIM_API void relsim_destroy(relsim_ctx* ctx);

/* Message of the last error on this context ("" if none; no counterpart in
   the paper). Owned by ctx. */
RELSIM_API const char* relsim_last_error(const relsim_ctx* ctx);

/* The 3D form (dim = 3, nx, ny, nz >= 3): the same step on a periodic
   nx x ny x nz grid with trilinear shape functions (27-node stencil). Node
   and cell (i,j,k) have linear index (k*ny + j)*nx + i, ncell = nx*ny*nz;
   positions carry three coordinates (x[3n], (x, y, z) interleaved); the
   stored mass matrix keeps 14 of the 27 offsets per node, in this order:
   (0,0,0), (1,0,0), (-1,1,0), (0,1,0), (1,1,0), then (di,dj,1) for
   dj = -1..1 (outer) and di = -1..1 (inner), i.e. ncell x 126 values (the
   2D form: (0,0), (1,0), (-1,1), (0,1), (1,1), ncell x 45). The 3D form
   covers the base scheme; its push allows any move length and re-sorts by a
   counting sort that does not keep the order within a cell. The adjoints
   cover the 2D form (INVALID_ARG in 3D).

   Load (replace) the particles of one species (paper: Sec. 2, the
   particles of the explicit pusher, each with a position, a momentum
   u = gamma v and a weight; the loaded state is the initial Harris
   equilibrium of Sec. 2, Eqs. 3-6, or any state): n particles, positions x[2n]
   (x[3n] in 3D),
   momenta u[3n], weights w[n], all FP64 (layout above). Positions outside
   the box are wrapped periodically. The library converts to its internal
   form and sorts the particles by cell (stable: equal cells keep the input
   order). Ids (if tracked) are the input indices 0..n-1. n = 0 empties the
   species. Errors: INVALID_ARG (species out of range, n < 0 or > 2^31-1,
   NULL arrays with n > 0), NONFINITE (NaN/Inf in the input), OOM, CUDA.
   Resets the step state: the next call must be relsim_build_mass_matrix. */
RELSIM_API int relsim_load_particles(relsim_ctx* ctx, int species, int64_t n, const double* x,
                          const double* u, const double* w, int where);

/* Set E^n on nodes and B^n on cell centres (each 3*ncell FP64, layout above;
   paper: the fields of Sec. 2, e.g. the Harris B_x profile of Eq. 4).
   Either pointer may be NULL to keep that field. Resets the step state.
   Errors: INVALID_ARG, NONFINITE, CUDA. */
RELSIM_API int relsim_set_fields(relsim_ctx* ctx, const double* E, const double* B, int where);

/* Copy the current E and B (after a solve: E^{n+1}, B^{n+1}) out as FP64
   (state access; no counterpart in the paper).
   Either pointer may be NULL. Errors: INVALID_ARG, CUDA. */
RELSIM_API int relsim_get_fields(relsim_ctx* ctx, double* E, double* B, int where);

/* Number of particles of a species (state access; no counterpart in the
   paper). */
RELSIM_API int relsim_num_particles(relsim_ctx* ctx, int species, int64_t* n);

/* (State access; no counterpart in the paper.) Copy the particles of a
   species out, in the library's current order
   (sorted by cell, stable), as FP64 x[2n] (x[3n] in 3D), u[3n], w[n] and, if ids are
   tracked, id[n] (each pointer may be NULL to skip it). Positions are
   absolute. Errors: INVALID_ARG (species out of range, id requested but not
   tracked), CUDA. */
RELSIM_API int relsim_get_particles(relsim_ctx* ctx, int species, double* x, double* u, double* w,
                         int32_t* id, int where);

/* (State access; no counterpart in the paper.) The particles of a species
   in the library's own form (the state it steps,
   read out and loaded back bit for bit: a checkpoint, or a state that moves
   between host and device every step at half the bytes of the FP64 record
   in the FP32 form). The species is sorted by cell; cell c (index
   (k*ny + j)*nx + i) holds particles start[c] .. start[c+1]-1. Per particle:
   the offsets within its cell off[D*n] (component k of particle p at
   off[k*n + p]: fx, fy and in 3D fz, each in [0, 1)), the momenta u[3n]
   (component k at u[k*n + p]) and the weight w[n]. The element type of off,
   u and w is the context's precision: float for precision 32, double for
   64. start has ncell + 1 int32 entries; id[n] (optional) the carried ids.

   relsim_get_particles_native copies the species out (each pointer may be
   NULL to skip it). Errors: INVALID_ARG (species, id without tracking),
   BAD_STATE (the species was never loaded), CUDA.

   relsim_load_particles_native replaces the species by n particles in this
   form (no conversion, no sort). It checks on the device: start[0] = 0,
   start[ncell] = n and start never decreasing, every offset in [0, 1), u and
   w finite, ids in [0, n); with ids tracked and id NULL the ids are
   0..n-1. Errors: INVALID_ARG (species, n, NULL arrays with n > 0, a NULL
   start table, id without tracking, a check above that fails), NONFINITE,
   OOM, CUDA; after a failed check the species is empty. Resets the step
   state like relsim_load_particles. */
RELSIM_API int relsim_get_particles_native(relsim_ctx* ctx, int species, int32_t* start, void* off, void* u,
                                           void* w, int32_t* id, int where);
RELSIM_API int relsim_load_particles_native(relsim_ctx* ctx, int species, int64_t n, const int32_t* start,
                                            const void* off, const void* u, const void* w, const int32_t* id,
                                            int where);

/* (State access; no counterpart in the paper.) Start index of each cell's
   particles of a species in the current order:
   start[ncell+1], start[ncell] = n. Errors: INVALID_ARG, CUDA. */
RELSIM_API int relsim_get_cell_start(relsim_ctx* ctx, int species, int64_t* start, int where);

/* Step part 1 (paper: Sec. 2, "Methods and Simulation Setup": the field
   solver's mass-matrix formulation, with each particle's relativistic
   rotation through its Lorentz factor; the equations are the header's
   gbar, a, alpha, Jhat and M lines): gather B^n, form alpha per particle,
   deposit Jhat and M.
   Allowed after load/set_fields or a push. Errors: BAD_STATE, CUDA. */
RELSIM_API int relsim_build_mass_matrix(relsim_ctx* ctx);

/* (State access; no counterpart in the paper.) The deposited Jhat (3*ncell,
   component-major) and M (Sec. 2's mass matrices), stored for the five
   neighbour offsets o in {(0,0), (1,0), (-1,1), (0,1), (1,1)} as
   M[(g*5 + k)*9 + r*3 + s] = block (r,s) of M_{g, g+o_k}; the other four
   offsets follow from M_{g+o,g} = M_{g,g+o}. In 3D the 14 stored offsets
   listed with the 3D form: M[(g*14 + k)*9 + r*3 + s]. FP64 out. Either
   pointer may be NULL. Errors: BAD_STATE (nothing built), INVALID_ARG,
   CUDA. */
RELSIM_API int relsim_get_mass_matrix(relsim_ctx* ctx, double* M, double* J, int where);

/* (Test access; no counterpart in the paper.) Replace the built Jhat and M
   by caller values (same layouts as
   relsim_get_mass_matrix), e.g. to drive the field solve on its own.
   Leaves the context in the built state. Errors: INVALID_ARG, CUDA. */
RELSIM_API int relsim_set_mass_matrix(relsim_ctx* ctx, const double* M, const double* J, int where);

/* Step part 2 (paper: Sec. 2, "the method is implicit only in the field
   solver"; the equations are the header's implicit-system, E^{n+1} and
   B^{n+1} lines; the paper names no linear solver, GMRES is this library's
   choice): GMRES solve for E^{n+theta}, then E^{n+1}, B^{n+1}.
   *iters (may be NULL) receives the Arnoldi steps, *rel_residual (may be
   NULL) the true relative residual. Synchronises the stream. The restart
   and Arnoldi decisions (Givens rotations, stop tests, the triangular
   solve) are taken on the device; here the host only reads them to know
   when to stop enqueueing iterations. A cycle whose new basis vector loses
   orthogonality (|w - V h|^2 < 1e-4 |w|^2) ends without it and restarts
   from the true residual. Errors: BAD_STATE (not built),
   NOT_CONVERGED (gmres_maxit reached; the fields are still advanced with
   the best iterate), NONFINITE, CUDA. */
RELSIM_API int relsim_field_solve(relsim_ctx* ctx, int* iters, double* rel_residual);

/* Adjoint of the field part of the solved step (the paper computes no
   gradients: this is the chain rule through its Sec. 2 step), with the
   particles held fixed (the implicit field solve of Sec. 2 is the step's only global
   coupling; this is the piece a differentiable window chains with the
   adjoints of the push and the deposit). The forward map is linear in
   (E^n, B^n, Jhat):
     b = E^n + theta dt curl_n B^n - theta dt Jhat,  A E^{n+theta} = b,
     E^{n+1} = (E^{n+theta} - (1-theta) E^n)/theta,
     B^{n+1} = B^n - dt curl_c E^{n+theta}.
   Given gE1 = dL/dE^{n+1} and gB1 = dL/dB^{n+1} (3*ncell FP64 each, field
   layout), it solves A^T lambda = gE1/theta - dt curl_c^T gB1 by GMRES
   (the same device-controlled loop, transposed operator; gmres_tol and
   gmres_maxit of the context) and returns dL/dE^n = lambda - (1-theta)/theta
   gE1, dL/dB^n = gB1 + theta dt curl_n^T lambda, dL/dJhat = -theta dt lambda
   (3*ncell each) and dL/dM for the stored mass-matrix blocks (ncell x 45 in
   relsim_get_mass_matrix's layout; a block serves both node pairs (g, g+o)
   and (g+o, g)): -theta dt (lambda_g E_{g+o}^T + [o != 0] lambda_{g+o}
   E_g^T), E = E^{n+theta}. gEt (may be NULL) is a further dL/dE^{n+theta}
   added to the right-hand side, e.g. the pushes' (relsim_push_adjoint), to
   chain the adjoints of one step. Any output may be NULL. Call it between
   relsim_field_solve and relsim_push (BAD_STATE otherwise). *iters and
   *rel_residual (may be NULL) report the adjoint solve. Synchronises the
   stream. Errors: INVALID_ARG, BAD_STATE, NOT_CONVERGED (outputs still
   written), NONFINITE, OOM, CUDA. */
RELSIM_API int relsim_field_adjoint(relsim_ctx* ctx, const double* gE1, const double* gB1, const double* gEt,
                                    double* gE0, double* gB0, double* gJ, double* gM, int* iters,
                                    double* rel_residual, int where);

/* Adjoint of the deposit of one species (no counterpart in the paper: the
   chain rule through Sec. 2's mass-matrix deposit; base scheme, gbar =
   gamma(u^n)):
   the deposit Jhat_g += (w q/dV) W_g(x) alpha u/gbar and M_{gg'} += (w q
   beta/dV) W_g W_g' alpha/gbar, alpha from B^n(x). Given gJ = dL/dJhat
   (3*ncell) and gM = dL/dM for the stored blocks (ncell x 45, the layout of
   relsim_get_mass_matrix and relsim_field_adjoint's output), it returns per
   particle gu0 = dL/du^n (3n, interleaved), gx0 = dL/dx^{n+1/2} (2n,
   interleaved) and, if gw0 is not NULL, gw0 = dL/dw (n; Jhat and M are
   linear in the weight, so this is the particle's contribution to
   <gJ, Jhat> + <gM, M> per unit weight), in the current order, and
   overwrites gB = dL/dB^n (centre field, 3*ncell) with this species'
   contribution. Per particle from the stored values, in the form's
   precision. Call it after relsim_build_mass_matrix and before
   relsim_push. Synchronises the stream. Errors: INVALID_ARG (including a
   gamma_pred context: relsim_step_adjoint covers that reading), BAD_STATE,
   OOM, CUDA.
   One step's adjoint chains the three: relsim_push_adjoint per species
   (giving dL/dE^{n+theta} and part of dL/dB^n), relsim_field_adjoint with
   gEt = their sum (giving dL/dE^n, the field part of dL/dB^n, dL/dJhat,
   dL/dM), relsim_deposit_adjoint per species; dL/du^n and dL/dx^{n+1/2} are
   the sums of the push's and the deposit's, dL/dB^n of all three. */
RELSIM_API int relsim_deposit_adjoint(relsim_ctx* ctx, int species, const double* gJ, const double* gM,
                                      double* gu0, double* gx0, double* gB, double* gw0, int where);

/* Adjoint of the push of one species with the fields held fixed (no
   counterpart in the paper: the chain rule through the explicit pusher of
   Sec. 2; base scheme, gbar = gamma(u^n)). For the
   solved step's push u^{n+1} = 2 alpha (u^n + beta E^{n+theta}(x)) - u^n,
   x^{n+3/2} = x + dt u^{n+1}/gamma^{n+1}, with alpha from B^n(x): given
   gu1 = dL/du^{n+1} (3n, interleaved (ux, uy, uz)) and gx1 =
   dL/dx^{n+3/2} (2n, interleaved (x, y)) for the species' n particles in
   their current order (the order relsim_get_particles returns before the
   push), it returns gu0 = dL/du^n (3n), gx0 = dL/dx^{n+1/2} (2n), and
   overwrites gE = dL/dE^{n+theta} (node field, 3*ncell) and gB = dL/dB^n
   (centre field, 3*ncell) with this species' contribution (sum the species
   yourself). The push is replayed per particle in FP64 from the stored
   values; the gathers' transposes are scatters with the same weights.
   Call it between relsim_field_solve and relsim_push. Synchronises the
   stream. Errors: INVALID_ARG (including a gamma_pred context), BAD_STATE,
   OOM, CUDA. */
RELSIM_API int relsim_push_adjoint(relsim_ctx* ctx, int species, const double* gu1, const double* gx1,
                                   double* gu0, double* gx0, double* gE, double* gB, int where);

/* One whole step's adjoint on device memory, in place (no counterpart in
   the paper, which computes no gradients; either reading of gbar): the
   chain rule through the step of Sec. 2 (deposit of the
   mass matrices and the predicted current, implicit field solve, push).
   From the state the context holds (loaded or pushed, not yet built) it
   builds the mass matrix and solves the step forward, then runs the pushes'
   adjoints (relsim_push_adjoint), the field adjoint with the pushes'
   dL/dE^{n+theta} (relsim_field_adjoint) and the deposits' adjoints
   (relsim_deposit_adjoint), and adds up every path. Arguments, all DEVICE
   memory (FP64):
     gE, gB   3*ncell each, field layout: on entry dL/dE^{n+1} (nodes) and
              dL/dB^{n+1} (cell centres), on return dL/dE^n and dL/dB^n;
     gu[s]    3 n_s, interleaved (ux, uy, uz), and
     gx[s]    2 n_s, interleaved (x, y), one pair per species s (arrays of
              nspecies host pointers to device arrays): indexed by the
              particle's id (track_ids), on entry dL/du^{n+1} and
              dL/dx^{n+3/2}, on return dL/du^n and dL/dx^{n+1/2};
     gw[s]    n_s per species (gw, or any gw[s], may be NULL), indexed by
              id: the step's dL/dw is added (the weights do not change
              from step to step, so a window sums the steps' terms).
   Ids must be a permutation of 0 .. n_s - 1 (as a load assigns them, or
   after relsim_relabel_particles with a permutation); with repeated ids the
   gradients of the colliding particles are undefined (every access stays in
   bounds). Indexing by id makes the call independent of the order the
   push's re-sort leaves, so a window of steps chains calls without
   reordering anything. The context is left solved (relsim_push advances
   it). *iters, *rel_residual (may be NULL): the adjoint solve. Device
   scratch of 10 max_s(n_s) + 7*3*ncell + 45*ncell doubles is kept by the
   context. In a gamma_pred context the chain also runs through the
   predicted Lorentz factor gamma(u^n + beta E^n(x)) of the deposit and the
   push: its dL/dE^n joins the field adjoint's in gE, its dL/du^n and
   dL/dx^{n+1/2} the particles'. Synchronises the stream. Errors:
   INVALID_ARG (a null array, track_ids off), BAD_STATE (not a loaded or pushed
   state), NOT_CONVERGED (the forward or the adjoint solve; outputs still
   written), NONFINITE, OOM, CUDA. */
RELSIM_API int relsim_step_adjoint(relsim_ctx* ctx, double* gE, double* gB, double* const* gu, double* const* gx,
                                   double* const* gw, int* iters, double* rel_residual);

/* (State access; no counterpart in the paper.) Relabel a species'
   particles (track_ids): each particle carrying id j
   gets ids[j] (n_s int32, host or device per where). Right after a load
   the ids are the input indices, so this gives the particle loaded from
   index i the label ids[i] (e.g. to keep the labels of a state saved with
   relsim_get_particles). Every carried id and every ids[j] must lie in
   [0, n_s): checked before anything changes. Synchronises the stream.
   Errors: INVALID_ARG (species, where, ids not tracked, null ids, a value
   out of range), CUDA. */
RELSIM_API int relsim_relabel_particles(relsim_ctx* ctx, int species, const int32_t* ids, int where);

/* E^{n+theta} of the last solve (Sec. 2's implicit field; 3*ncell FP64;
   state access). Errors: BAD_STATE, CUDA. */
RELSIM_API int relsim_get_E_theta(relsim_ctx* ctx, double* E, int where);

/* (Test access.) Apply the implicit operator of Sec. 2's field solve,
   A = I + (theta dt)^2 curl_n curl_c + theta dt M
   of the built mass matrix to v (3*ncell FP64, device or host per where),
   writing out (same layout). Errors: BAD_STATE, INVALID_ARG, CUDA. */
RELSIM_API int relsim_apply_operator(relsim_ctx* ctx, const double* v, double* out, int where);

/* Step part 3 (paper: Sec. 2, "the particle pusher is explicit"; the
   equations are the header's ubar, u^{n+1} and x^{n+3/2} lines; the re-sort
   by cell is this library's layout, the paper is silent on it): push
   velocities and positions of every species with
   E^{n+theta} and B^n, then sort each species by its new cells. Also
   accumulates the particle terms of the energy ledger. Allowed after a
   solve. Errors: BAD_STATE, CUDA. */
RELSIM_API int relsim_push(relsim_ctx* ctx);

/* Energy ledger of the current state and of the last step (FP64 struct,
   caller-owned). Paper: Sec. 2's energy claim (the mass-matrix field solve
   conserves energy exactly, to machine precision, in the non-relativistic
   limit, and reduces the relativistic energy error) and Table 1's column of
   the energy error |E - E0|/E0: W_E + W_B + K is the total energy, and
   `residual` closes the step's discrete identity while `mismatch` is the
   scheme's own relativistic energy error. Synchronises the stream. Errors: INVALID_ARG, NONFINITE
   (NaN/Inf in an energy), CUDA. */
RELSIM_API int relsim_energy_ledger(relsim_ctx* ctx, relsim_energy* out);

/* One full step of Sec. 2's method (build, solve, push; the three calls
   above); fills *ledger if it is non-NULL.
   Returns the first error of its parts (NOT_CONVERGED still completes the
   step). The first step after a load runs its parts from the host; later
   steps (when profiling is off and, in the 2D form with linear shapes, no
   particle can cross more than one cell per step; always in the 3D form and
   with quadratic shapes) run as one CUDA graph captured on first use for the current
   buffer layout: the solve's restart and Arnoldi loops are conditional while
   nodes whose conditions the device sets, so the step needs one launch and
   one synchronisation. Both routes run the same kernels in the same order.
   If capturing fails the context keeps stepping from the host (see
   relsim_graph_info). A NONFINITE solve in a graph step is reported after
   the whole step ran (the state is then invalid, as on the host route). */
RELSIM_API int relsim_step(relsim_ctx* ctx, relsim_energy* ledger);

/* (Runtime state; no counterpart in the paper.) Whether steps run as
   graphs: *graph_steps (may be NULL) = steps run as a
   graph so far; *disabled = 1 if a capture failed and *why (owned by the
   context) says why. Errors: INVALID_ARG. */
RELSIM_API int relsim_graph_info(const relsim_ctx* ctx, int64_t* graph_steps, int* disabled, const char** why);

/* Particle energy spectrum of a species (diagnostic; the paper's spectra,
   Sec. 3.2 "Nonlinear reconnection and spectra" and its spectrum figures,
   are weighted particle distributions over the Lorentz factor or the proper
   speed u/c). variable 0 bins x = gamma - 1 = |u|^2/(gamma + 1), variable 1
   bins x = |u|. edges: nbins + 1 strictly ascending finite FP64 bin edges in
   HOST memory (1 <= nbins <= 4096), e.g. logarithmic. Outputs (each may be
   NULL, host or device per where) have nbins + 2 entries: [0] below
   edges[0], [b] for edges[b-1] <= x < edges[b] (b = 1..nbins), [nbins+1] at
   or above edges[nbins]; weight = sum of the particles' weights (FP64),
   count = number of particles. x is computed in the form's precision (FP32
   or FP64) with correctly rounded operations and no fused multiply-add, and
   the bin decision is exact against the FP64 edges, so counts are
   reproducible bit for bit. Synchronises the stream for host outputs.
   Errors: INVALID_ARG (species, variable, nbins, edges not ascending or not
   finite), OOM, CUDA. */
RELSIM_API int relsim_energy_spectrum(relsim_ctx* ctx, int species, int variable, int nbins,
                                      const double* edges, double* weight, int64_t* count, int where);

/* Energy in the Fourier modes along x of one component of B (diagnostic;
   the linear-tearing measurement of Sec. 3.1 and Fig. 1 follows the B_y
   energy, its low-pass part and single modes, whose exponential growth gives
   the tearing rate). For m = 0 .. nmodes-1, with F_{m,j} the DFT along x of
   row j of the cell-centre component B_c,
     F_{m,j} = sum_i B_c(i, j) exp(-2 pi sqrt(-1) m i / nx),
     energy[m] = (1/2) dV (c_m / nx) sum_j |F_{m,j}|^2,
   c_m = 1 for m = 0 and m = nx/2, else 2, so that the energies of
   m = 0 .. nx/2 add up to (1/2) sum B_c^2 dV (Parseval). Mode m has the
   wavenumber k = 2 pi m / L_x, L_x = nx dx. B is the current B (B^{n+1}
   after a push). component: 0, 1, 2 (x, y, z); 1 <= nmodes <= nx/2 + 1.
   energy: nmodes FP64 values, host or device per where. With where =
   RELSIM_DEVICE nothing waits (the result is enqueued on the stream);
   with RELSIM_HOST the stream is synchronised. The sums along x run in the
   form's precision from exact integer phases, the rest in FP64 in a fixed
   order: repeated calls give identical results. Errors: INVALID_ARG, OOM,
   CUDA. */
RELSIM_API int relsim_field_modes(relsim_ctx* ctx, int component, int nmodes, double* energy, int where);

/* The energy of one Fourier mode m of a B component (as relsim_field_modes:
   Sec. 3.1's tearing diagnostic, the loss of a differentiable window) and
   its gradient in the field: *energy = W_m, and gB (3*ncell FP64, field
   layout) = dW_m/dB: zero outside `component`, and there
     dW_m/dB_c(i, j) = dV (c_m/nx) (Re F_{m,j} cos(2 pi m i/nx)
                                     - Im F_{m,j} sin(2 pi m i/nx)),
   F_{m,j} = sum_i B_c(i, j) exp(-2 pi sqrt(-1) m i/nx). 0 <= mode <= nx/2.
   Both outputs host or device per where (device: enqueued, nothing waits;
   host: synchronises). Errors: INVALID_ARG, OOM, CUDA. */
RELSIM_API int relsim_field_mode_gradient(relsim_ctx* ctx, int component, int mode, double* energy, double* gB,
                                          int where);

/* Exponential growth rate of a positive series s[k] sampled at equal
   steps dt (host code, no context): the least-squares slope of log s[k]
   against k dt over every run of `window` consecutive samples
   (2 <= window <= n), and the largest of them with the index of its first
   sample. Runs containing a non-positive or non-finite sample are skipped.
   For a mode energy the field amplitude grows at half this rate (Sec. 3.1:
   the tearing rate as the best-fit slope of a mode's energy over its linear
   phase). Errors: INVALID_ARG (bad sizes, NULL, dt <= 0, or no admissible
   run). */
RELSIM_API int relsim_growth_fit(const double* s, int n, double dt, int window, double* rate, int* first);

/* Per-mode growth rates and the tearing dispersion fit (host code, no
   context). Sec. 3.1 measures the growth of each Fourier mode of B_y as a
   best fit over the linear phase and compares the rates with the
   dispersion f(k) = ka (1 - k^2 a^2) of Sec. 2, whose peak lies at
   ka = 1/sqrt(3) and whose unstable range ends at ka = 1 (Fig. 1 b, d).
   modes: nsamples x nmodes energies, row-major by sample (the layout
   relsim_batch_run writes for one instance), sampled every dt. For mode m
   = 1 .. nmodes-1, rates[m] = half the least-squares slope of log
   modes[k][m] against k dt over samples first .. first+window-1 (the
   field amplitude's growth rate), or NaN when a sample there is not
   positive and finite; rates[0] (the mean field) is NaN. Mode m has
   x_m = k_m a = 2 pi m a / Lx. The fit: rate(x) = A x b (1 - x^2 b^2) by
   least squares over the modes with finite rates, A closed-form for each
   b, b minimising the residual over [0.2, 4] (a grid of step 1e-3, then a
   golden-section search of the best grid cell to 1e-12); *A and *b receive
   the fit, the fitted curve peaks at x = 1/(sqrt(3) b) and changes sign at
   x = 1/b. Errors: INVALID_ARG (NULL pointers, nsamples < 2, nmodes < 3,
   window < 2, first out of range, dt, Lx or a not positive and finite, or
   fewer than two finite rates). */
RELSIM_API int relsim_dispersion_fit(const double* modes, int nsamples, int nmodes, double dt, int first,
                                     int window, double Lx, double a, double* rates, double* A, double* b);

/* ---- batched independent instances (the paper has no counterpart: a
   parameter scan of independent tearing runs, e.g. over L_x, the sheet
   half-thickness and sigma, each instance a context of its own) ----
   relsim_batch_create takes `count` contexts that hold a loaded state
   (particles and fields) and `nworkers` host threads (1 <= nworkers <= 256).
   The batch does not own the contexts: destroy them after the batch. Give
   each context its own CUDA stream so instances overlap on the GPU.
   Errors: INVALID_ARG, OOM. */
typedef struct relsim_batch relsim_batch;
RELSIM_API int relsim_batch_create(relsim_ctx* const* ctxs, int count, int nworkers, relsim_batch** out);

/* Advance every instance nsteps full steps (relsim_step without the
   ledger; the independent tearing runs of a scan such as Sec. 3.1's). The workers take instances largest first (by particle count) and
   each runs its instance through all steps before taking the next; no two
   threads touch one context. After every step of instance b the energies of
   modes 0 .. nmodes-1 of B's component `component` (as relsim_field_modes)
   go to modes[(b nsteps + s) nmodes + m] (host; pass NULL or nmodes = 0
   to skip) and the step's GMRES iteration count to iters[b nsteps + s]
   (host, may be NULL). status[b] (host, required) receives RELSIM_OK, the
   first error of instance b (its later steps are skipped), or
   RELSIM_ERR_NOT_CONVERGED if a solve hit gmres_maxit (the steps go on).
   Returns RELSIM_OK when every status is OK, otherwise the first non-OK
   status in instance order. Errors of the call itself: INVALID_ARG, OOM,
   CUDA. */
RELSIM_API int relsim_batch_run(relsim_batch* b, int nsteps, int component, int nmodes, double* modes,
                                int* status, int* iters);

/* Shared launches over the batch's instances (off by default). With on = 1,
   relsim_batch_run splits the instances into `groups` groups of about equal
   particle count (groups <= 0: one group) and steps each group through ONE
   graph per step in which one deposit launch, one push launch and one
   re-sort launch per species cover the particles of all its instances (each
   instance's row units numbered after the previous instance's), while each
   instance's field solve, field update and sort tables run as parallel
   branches of the same graph; the groups run on streams of their own, so one
   group's solves overlap another's particle kernels. This is
   the batched form of the data-parallel step over independent instances
   (Sec. 3.1's scan of tearing runs: many small grids that one instance
   alone cannot fill the GPU with). It applies when every instance is of the
   2D form with linear shapes and one-cell moves, shares the precision,
   species count and reading of the Lorentz factor, has every species
   loaded, and all instances have taken the same number of steps in the run
   so far; otherwise relsim_batch_run falls back to per-instance graphs or
   host-driven steps. deposit_blocks and push_blocks set the shared launches'
   grids (<= 0: 2 and 16 blocks per SM). Results equal the per-instance
   steps' up to the order of floating-point sums (the deposit's and the
   ledger's atomics). Errors: INVALID_ARG. */
RELSIM_API int relsim_batch_set_shared(relsim_batch* b, int on, int groups, int deposit_blocks, int push_blocks);

/* How the last relsim_batch_run advanced the instances after their first
   step (no counterpart in the paper): 0 host-driven workers, 1 per-instance
   step graphs, 2 shared launches (relsim_batch_set_shared); -1 before any
   run. */
RELSIM_API int relsim_batch_last_path(const relsim_batch* b);

/* Free the batch (not its contexts; no counterpart in the paper). NULL is
   a no-op. */
RELSIM_API void relsim_batch_destroy(relsim_batch* b);

/* ---- launch-shape autotuner (no counterpart in the paper) ----
   Times candidate launch shapes of the two heaviest particle kernels on the
   loaded state and keeps the fastest for this context: the deposit's block
   count (it strides over row units of 32 cells: 1, 2, 3, 4 blocks per SM in
   the 2D form with linear shapes; 2, 4, 8, 16 in 3D and with quadratic
   shapes) and the push's grid (at most 4, 8, 16, 32 blocks per SM), and, in
   the 2D form with linear shapes, a compile-time shape of the implicit
   operator (the 3D and quadratic operators have one): its tile height
   (32-node-wide tiles of 8 or 4 rows in the FP32 form, 4 or 2 in FP64; an
   Arnoldi-mode application with 8 dot products on the deposited mass
   matrix). Each candidate runs once untimed and three times timed (CUDA events;
   the least counts). Call it on a loaded state before a build (the trials
   overwrite only what the next step recomputes); later steps use the
   choice (captured step graphs are recaptured). out (may be NULL) receives
   the candidates, their times and the choice. Synchronises the stream.
   Errors: INVALID_ARG, BAD_STATE, OOM, CUDA. */
typedef struct {
    int ncand;
    int deposit_blocks[8];
    float deposit_ms[8];
    int push_blocks[8];
    float push_ms[8];
    int deposit_choice, push_choice;   /* indices into the candidates */
    int op_nrows;                      /* tile heights tried for the 2D operator */
    int op_rows[4];                    /* rows per operator tile (32 nodes wide)  */
    float op_ms[4];                    /* an Arnoldi-mode application, 8 dots    */
    int op_choice;
} relsim_tuning;
RELSIM_API int relsim_autotune(relsim_ctx* ctx, relsim_tuning* out);

/* Set the launch shapes the autotuner chooses (e.g. one instance's tuning
   applied to others of the same size): the deposit's block count and the
   push's grid cap (0: the defaults; the deposit two blocks per SM in the 2D
   form with linear shapes, at most 8 in 3D and with quadratic shapes; the
   push at most 16) and the 2D
   operator's tile rows (0 or the form's default: 8 in FP32, 4 in FP64; or
   the alternative: 4 in FP32, 2 in FP64). Results do not depend on the
   shapes beyond rounding (launch shapes have no counterpart in the paper).
   Errors: INVALID_ARG. */
RELSIM_API int relsim_set_launch_shapes(relsim_ctx* ctx, int deposit_blocks, int push_blocks, int op_rows);

/* Library version (major*10000 + minor*100 + patch; no counterpart in the
   paper). */
RELSIM_API int relsim_version(void);

/* ---- profiling (the paper has no counterpart; a measurement aid) ----
   When enabled, the library records a CUDA event pair on its stream around
   each group of kernel launches below and accumulates the elapsed device
   time per group. Slots: */
#define RELSIM_PROF_DEPOSIT 0      /* zero M/Jhat + the deposit kernel          */
#define RELSIM_PROF_PUSH 1         /* push; each old cell written back grouped
                                      by move direction; ledger sums          */
#define RELSIM_PROF_SORT_TABLES 2  /* new-cell counts and their scan           */
#define RELSIM_PROF_PERMUTE 3      /* the pushed particles into new-cell order */
#define RELSIM_PROF_GMRES_APPLY 4  /* operator applications in GMRES           */
#define RELSIM_PROF_GMRES_ORTHO 5  /* Gram-Schmidt, norms, basis updates       */
#define RELSIM_PROF_FIELD_UPDATE 6 /* E^{n+1}, B^{n+1}, field ledger terms     */
#define RELSIM_PROF_RHS 7          /* right-hand side of the field equation    */
#define RELSIM_PROF_LOAD 8         /* load conversion + radix sort + gather    */
#define RELSIM_PROF_GENERAL_SORT 9 /* long-move push path (radix sort)         */
#define RELSIM_PROF_NSLOTS 10

typedef struct {
    double ms[16];           /* accumulated device time per slot            */
    int64_t groups[16];      /* timed launch groups per slot                */
    int64_t kernels[16];     /* kernel launches per slot                    */
} relsim_profile;

/* Turn event timing on (nonzero) or off (a measurement aid with no
   counterpart in the paper). Errors: INVALID_ARG, CUDA. */
RELSIM_API int relsim_profile_enable(relsim_ctx* ctx, int on);

/* Read the accumulated times (synchronises the stream; no counterpart in
   the paper); reset != 0 clears them afterwards. Errors: INVALID_ARG,
   CUDA. */
RELSIM_API int relsim_profile_read(relsim_ctx* ctx, relsim_profile* out, int reset);

/* Total kernel launches made by this library in this process (all
   contexts), for counting the kernels of a timed region (no counterpart in
   the paper). */
RELSIM_API int64_t relsim_kernel_launches(void);

/* ---- allocation-free kinetic energy (the paper has no counterpart) ----
   For callers that cannot allocate device memory where they need this
   number: a diagnostics hook inside a time loop whose device memory is all
   reserved up front by its own pool, or code running where cudaMalloc /
   cudaFree would synchronise the device or is not allowed.

   *out (one device double) = sum_p w[p] m (gamma_p - 1) over n particles,
   gamma_p = sqrt(1 + |u_p|^2), u[3n] interleaved (ux, uy, uz) and w[n] FP64
   in device memory; the same sum the energy ledger reports per species. No
   context is needed and nothing is allocated: the per-block partial sums
   go to one fixed 32 KB device array inside the library, which every GPU
   that loads the library holds until the process exits. The work is
   enqueued on cuda_stream (0: the legacy default stream) and the call
   returns without waiting.

   The first call on a device looks up that array's device address
   (cudaGetSymbolAddress) with the device current; make that first call
   before any stream capture. The address is kept for the life of the
   process: after cudaDeviceReset on that device it no longer points at the
   array, so do not call this entry point on a device that was reset. All
   calls share the array and each overwrites
   the partials it uses, so nothing needs clearing, but calls that overlap
   on the GPU (on different streams, or from several threads) race on it and
   must be serialised by the caller. The result is written by the second of
   two kernels, in a fixed order, so repeated calls give identical sums.

   Errors: INVALID_ARG (n < 0, NULL out, or NULL arrays with n > 0),
   TOO_LARGE (n > RELSIM_NOALLOC_MAX_PARTICLES: split the particles and add
   the results), CUDA (launch failure or no current device). */
#define RELSIM_ERR_TOO_LARGE (-9)
#define RELSIM_NOALLOC_MAX_PARTICLES 33554432   /* 4096 blocks x 8192 particles */
RELSIM_API int relsim_kinetic_energy_noalloc(const double* u, const double* w, int64_t n, double m,
                                  double* out, void* cuda_stream);

#ifdef __cplusplus
}
#endif

#endif /* RELSIM_H */
