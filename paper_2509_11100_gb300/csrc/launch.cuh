// launch.cuh -- host-side launchers of the RelSIM kernels (internal).
//
// Every launcher enqueues on the given stream and returns the launch status
// (cudaGetLastError); none synchronises.
#pragma once

#include "common.cuh"

namespace relsim {

// process-wide count of kernel launches made by this library
void count_launches(int n);

// One buffer of a species' particles in the internal form: position as cell
// (implicit: the particles are stored sorted by cell, cell c owning
// [start[c], start[c+1])) plus offsets fx, fy in [0,1); momenta u = gamma v;
// weight w; optional int32 id.
template <typename T>
struct PArrays {
    T* fx;
    T* fy;
    T* ux;
    T* uy;
    T* uz;
    T* w;
    int32_t* id;   // may be null
};

// Per-species constants of the deposit and the push.
struct SpeciesConst {
    double q, m;
};

template <typename T>
struct DepositSpecies {
    int nsp;
    const T* fx[kMaxSpecies];
    const T* fy[kMaxSpecies];
    const T* ux[kMaxSpecies];
    const T* uy[kMaxSpecies];
    const T* uz[kMaxSpecies];
    const T* w[kMaxSpecies];
    const int32_t* start[kMaxSpecies];
    T beta[kMaxSpecies];   // q dt / (2 m)
    T cJ[kMaxSpecies];     // q / dV
    T cM[kMaxSpecies];     // q beta / dV
};

// One instance's species in a shared launch over several instances (the
// push and the re-sort of the batched 2D form with linear shapes): its
// arrays, fields, grid and constants, its ledger slots (dK, work, mismatch,
// K1, added to atomically) and the first unit of the instance in the
// launch's numbering (ascending across the descriptors).
template <typename T>
struct PushDesc {
    PArrays<T> src, dst;
    const int32_t* start;       // cell starts of src (the push's input)
    const int32_t* start_new;   // the new cell starts (the re-sort's)
    int32_t* n9;
    int32_t* off9;
    const T* Eth;
    const T* B;
    const T* En;
    GridP g;
    T beta, dt_dx, dt_dy, qdt, m;
    double* led;
    int* err;
    int unit0;
};

// One instance in a shared deposit launch: its species' particles (as the
// single-instance deposit takes them), B, E^n (the predicted-gamma form),
// its mass matrix and current, grid, and first unit.
template <typename T>
struct DepDesc {
    DepositSpecies<T> ds;
    const T* B;
    const T* En;
    T* M;
    T* J;
    GridP g;
    int unit0;
};

// shared launches over several instances (descs in device memory, unit0
// ascending; all instances of the 2D form with linear shapes and one-cell
// moves, the same precision, species count and reading of gbar)
template <typename T>
cudaError_t deposit_batch(const DepDesc<T>* descs, int ninst, int total_units, bool pred, int* err, cudaStream_t st,
                          int blocks);
template <typename T>
cudaError_t push_sort_batch(const PushDesc<T>* descs, int ninst, int total_units, bool pred, int blocks,
                            cudaStream_t st);   // ledger sums added to each descriptor's led
template <typename T>
cudaError_t permute_batch(const PushDesc<T>* descs, int ninst, int total_units, cudaStream_t st);

// ----- sort.cu -----
// exclusive scan of n int32 values (n <= 4096*16384); out may alias in;
// *total (device) receives the sum if non-null. tmp: scan_tmp_size(n) ints.
size_t scan_tmp_ints(int64_t n);
cudaError_t scan_exclusive_i32(const int32_t* in, int32_t* out, int64_t n, int32_t* total,
                               int32_t* tmp, cudaStream_t st);
// stable LSD radix sort of (key, val) pairs, keys in [0, 2^key_bits).
// Ping-pongs between (k0,v0) and (k1,v1); *result_in_1 tells where it ended.
size_t radix_tmp_ints(int64_t n);
cudaError_t radix_sort_pairs(int32_t* k0, int32_t* v0, int32_t* k1, int32_t* v1, int64_t n,
                             int key_bits, int32_t* tmp, bool* result_in_1, cudaStream_t st);
// counts[k] = #keys equal to k (counts zeroed inside)
cudaError_t histogram_keys(const int32_t* keys, int64_t n, int32_t* counts, int nkeys,
                           cudaStream_t st);
// new-cell counts of the neighbour-move sort
cudaError_t move_counts(const int32_t* n9, int32_t* count_new, GridP g, cudaStream_t st);
// zero `bytes` (a multiple of 4) from p (16-byte aligned) with a kernel
cudaError_t zero_fill(void* p, size_t bytes, cudaStream_t st);
cudaError_t iota_i32(int32_t* a, int64_t n, cudaStream_t st);

// ----- d3.cu (the 3D form) -----
struct GmDyn;
template <typename T>
struct FzArrays {
    const T* fz[kMaxSpecies];
};
template <typename T>
cudaError_t load_convert3(const double* x, const double* u, const double* w, int64_t n, GridP g, PArrays<T> out,
                          T* ofz, int32_t* key, int32_t* val, int* bad, cudaStream_t st);
template <typename T>
cudaError_t gather_particles3(const int32_t* perm, PArrays<T> src, const T* sfz, PArrays<T> dst, T* dfz, int64_t n,
                              bool ids_from_perm, cudaStream_t st);
template <typename T>
cudaError_t export_particles3(PArrays<T> p, const T* fz, const int32_t* start, GridP g, double* x, double* u,
                              double* w, int32_t* id, cudaStream_t st);
template <typename T>
cudaError_t deposit3(const DepositSpecies<T>& ds, const FzArrays<T>& fz, const T* B, T* M, T* J, GridP g,
                     cudaStream_t st, int blocks = 0);   // blocks 0: at most 8 per SM
int op_blocks3(GridP g);
template <typename T, int MODE, bool TR>
cudaError_t launch_op3(const T* M, const double* in, double sc, const double* b, double* out, double* vj,
                       const double* V, int64_t ldv, int nv, GridP g, double* partial, cudaStream_t st,
                       const GmDyn* dyn);
template <typename T>
cudaError_t rhs3(const T* E, const T* B, const T* J, double* b, GridP g, cudaStream_t st);
template <typename T>
cudaError_t field_update3(const double* x, const T* M, const T* J, T* Eth, T* E, const T* B0, T* B1, GridP g,
                          double* partial, int nblocks, cudaStream_t st);
int push_blocks3(GridP g, int cap = 0);   // cap 0: 16 blocks per SM
// rank/count null: keys only; else rank[p] = slot among the new cell's particles (count zeroed first)
template <typename T>
cudaError_t push3(PArrays<T> src, const T* sfz, PArrays<T> dst, T* dfz, const int32_t* start, int32_t* key,
                  int32_t* rank, int32_t* count, const T* Eth, const T* B, GridP g, SpeciesConst sc, double* lsum,
                  int nblocks, cudaStream_t st);
template <typename T>
cudaError_t place3(PArrays<T> src, const T* sfz, PArrays<T> dst, T* dfz, const int32_t* key, const int32_t* rank,
                   const int32_t* start, int64_t n, cudaStream_t st);

// ----- quad.cu (2D, quadratic shapes) -----
template <typename T>
cudaError_t deposit_q(const DepositSpecies<T>& ds, const T* B, T* M, T* J, GridP g, cudaStream_t st,
                      int blocks = 0);   // blocks 0: at most 8 per SM
int op_blocks_q(GridP g);
template <typename T, int MODE, bool TR>
cudaError_t launch_op_q(const T* M, const double* in, double sc, const double* b, double* out, double* vj,
                        const double* V, int64_t ldv, int nv, GridP g, double* partial, cudaStream_t st,
                        const GmDyn* dyn);
template <typename T>
cudaError_t field_update_q(const double* x, const T* M, const T* J, T* Eth, T* E, const T* B0, T* B1, GridP g,
                           double* partial, int nblocks, cudaStream_t st);
int push_blocks_q(GridP g, int cap = 0);   // cap 0: 16 blocks per SM
template <typename T>
cudaError_t push_q(PArrays<T> src, PArrays<T> dst, const int32_t* start, int32_t* key, int32_t* rank,
                   int32_t* count, const T* Eth, const T* B, GridP g, SpeciesConst sc, double* lsum, int nblocks,
                   cudaStream_t st);

// ----- native.cu -----
// bits of *bad (accumulated): 1 non-finite u or w, 2 an offset outside [0, 1),
// 4 a start table that does not run from 0 to n without decreasing, 8 an id
// outside [0, n) (p.id may be null; fz null in 2D)
template <typename T>
cudaError_t check_native(const int32_t* start, int ncell, PArrays<T> p, const T* fz, int64_t n, int* bad,
                         cudaStream_t st);
// id[i] = i
cudaError_t iota_ids(int32_t* id, int64_t n, cudaStream_t st);

// ----- adjoint.cu -----
// lu[i] = gu[id[i]], lx[i] = gx[id[i]] (FP64, 3 and 2 interleaved components)
cudaError_t gather_grad(const int32_t* id, const double* gu, const double* gx, double* lu, double* lx, int64_t n,
                        cudaStream_t st);
// gu[id[i]] = lu[i], gx[id[i]] = lx[i] (or += with add)
cudaError_t scatter_grad(const int32_t* id, const double* lu, const double* lx, double* gu, double* gx, int64_t n,
                         bool add, cudaStream_t st);
// gw[id[i]] += lw[i]
cudaError_t scatter_add_w(const int32_t* id, const double* lw, double* gw, int64_t n, cudaStream_t st);
// bit 0 of *bad if id[i] or ids[i] is outside [0, n) (flag accumulates)
cudaError_t check_ids(const int32_t* id, const int32_t* ids, int64_t n, int* bad, cudaStream_t st);
// id[i] = ids[id[i]]
cudaError_t relabel_ids(int32_t* id, const int32_t* ids, int64_t n, cudaStream_t st);
// out = a + b (FP64)
cudaError_t add_fields(const double* a, const double* b, double* out, int64_t n, cudaStream_t st);

// ----- particles.cu -----
// bit 2 of *flag if keys[0..n) is not non-decreasing (flag accumulates)
cudaError_t keys_unsorted(const int32_t* keys, int64_t n, int* flag, cudaStream_t st);
template <typename T>
cudaError_t load_convert(const double* x, const double* u, const double* w, int64_t n, GridP g,
                         PArrays<T> out, int32_t* key, int32_t* val, int* bad, cudaStream_t st);
template <typename T>
cudaError_t gather_particles(const int32_t* perm, PArrays<T> src, PArrays<T> dst, int64_t n,
                             bool ids_from_perm, cudaStream_t st);
template <typename T>
cudaError_t export_particles(PArrays<T> p, const int32_t* start, GridP g, double* x, double* u,
                             double* w, int32_t* id, cudaStream_t st);
template <typename T>
cudaError_t deposit(const DepositSpecies<T>& sp, const T* B, const T* En, T* M, T* J, GridP g, int* err,
                    cudaStream_t st, int max_blocks = 0);   // En = E^n for the predicted-gamma variant, else
                                                            // null; max_blocks 0: two per SM
// push with the cell-local sort: each old cell's pushed particles are written
// back over the cell's own index range in dst grouped by move direction d;
// n9[c][d] and off9[c][d] receive the count and the start of each run; the
// particle ledger sums (K0, dK, work, mismatch, K1) go to lsum (per block).
template <typename T>
cudaError_t push_sort(PArrays<T> src, PArrays<T> dst, const int32_t* start, int32_t* n9, int32_t* off9,
                      const T* Eth, const T* B, const T* En, GridP g, SpeciesConst sc, double* lsum_partial,
                      int lsum_blocks, int* err, cudaStream_t st);   // err: reserved for a bounded wait
// general path (moves longer than one cell): pushed particles to the same
// index of dst, their new cell to key; ledger sums as above
template <typename T>
cudaError_t push_general(PArrays<T> src, PArrays<T> dst, const int32_t* start, int32_t* key, const T* Eth,
                         const T* B, const T* En, GridP g, SpeciesConst sc, double* lsum_partial, int lsum_blocks,
                         cudaStream_t st);
// adjoint of the deposit: per particle dL/du^n, dL/dx^{n+1/2} and (gw0 not
// null) dL/dw from dL/dJhat (3 ncell) and dL/dM (ncell x 45, stored
// blocks); dL/dB^n added into gB (FP64 atomics). En not null: the
// predicted gbar = gamma(u^n + beta E^n(x)) with E^n = En, and dL/dE^n
// added into gEn.
template <typename T>
cudaError_t deposit_adjoint(PArrays<T> src, const int32_t* start, const double* gJ, const double* gM, double* gu0,
                            double* gx0, double* gw0, double* gB, const T* B, GridP g, SpeciesConst sc,
                            cudaStream_t st, const T* En = nullptr, double* gEn = nullptr);
// adjoint of the push with the fields fixed: per particle dL/du^n,
// dL/dx^{n+1/2} from dL/du^{n+1}, dL/dx^{n+3/2} (FP64, interleaved, current
// order); dL/dE^{n+theta}, dL/dB^n added into gE, gB (FP64 atomics); En not
// null: the predicted gbar, dL/dE^n added into gEn
template <typename T>
cudaError_t push_adjoint(PArrays<T> src, const int32_t* start, const double* gu1, const double* gx1, double* gu0,
                         double* gx0, double* gE, double* gB, const T* Eth, const T* B, GridP g, SpeciesConst sc,
                         cudaStream_t st, const T* En = nullptr, double* gEn = nullptr);
// the stable new-cell order from the runs of push_sort (err bit 1 if the
// runs and the new cell starts disagree)
template <typename T>
cudaError_t permute(PArrays<T> src, PArrays<T> dst, const int32_t* start_new, const int32_t* n9,
                    const int32_t* off9, GridP g, int* err, cudaStream_t st);
int push_grid_blocks(GridP g, int precision, int cap = 0);
int row_units(GridP g);   // the row units (up to 32 cells of one row) of the 2D particle passes   // cap: most blocks (0: 152 x 16)
// weighted and counted histogram of gamma - 1 (variable 0) or |u| (1) over
// nbins bins between ascending edges (nbins + 1, rounded up to T), plus the
// bins below and above them: wsum/cnt[nbins + 2], accumulated (zero them)
template <typename T>
cudaError_t spectrum(PArrays<T> p, int64_t n, int variable, const T* edges, int nbins, double* wsum,
                     unsigned long long* cnt, cudaStream_t st);
template <typename T>
cudaError_t kinetic_energy(PArrays<T> p, int64_t n, double m, double* partial, int nblocks,
                           cudaStream_t st);

// ----- fields.cu -----
template <typename T>
cudaError_t fields_from_double(const double* in, T* out, int64_t n, int* bad, cudaStream_t st);
template <typename T>
cudaError_t fields_to_double(const T* in, double* out, int64_t n, cudaStream_t st);
// a field into a GMRES vector (FP64, or double-float pairs when df)
template <typename T>
cudaError_t fields_to_vec(const T* in, double* out, int64_t n, int df, cudaStream_t st);
// FP64 <-> GMRES vector (a copy when df = 0; in and out may then coincide)
cudaError_t vec_from_double(const double* in, double* out, int64_t n, int df, cudaStream_t st);
cudaError_t vec_to_double(const double* in, double* out, int64_t n, int df, cudaStream_t st);
template <typename T>
cudaError_t rhs(const T* E, const T* B, const T* J, double* b, GridP g, cudaStream_t st);
// The implicit operator A = I + B, B = (theta dt)^2 curl_n curl_c + theta dt M,
// on shared-memory tiles; err gets bit 2 if a staging wait gave up.
// out = A v:
template <typename T>
cudaError_t apply_A(const T* M, const double* v, double* out, GridP g, int* err, cudaStream_t st,
                    bool tr = false);   // tr: A^T (every mass-matrix block transposed)
// r = b - A x and per-tile partials of |r|^2 (op_blocks(g) of them):
template <typename T>
cudaError_t op_residual(const T* M, const double* x, const double* b, double* r, GridP g, double* partial,
                        int* err, cudaStream_t st, bool tr = false);
// one Arnoldi step on B: v_j = sc u is written to vj (if not null), w = B v_j,
// and per tile the j+2 partials <w, V_q> (q < j), <w, v_j>, <w, w> (row
// stride j+2):
template <typename T>
cudaError_t op_arnoldi(const T* M, const double* u, double sc, double* vj, double* w, const double* V,
                       int64_t ldv, int j, GridP g, double* partial, int* err, cudaStream_t st);
int op_blocks(GridP g, int precision);
template <typename T>
cudaError_t field_update(const double* x, const T* M, const T* J, T* Eth, T* E, const T* B0,
                         T* B1, GridP g, double* partial, int nblocks, cudaStream_t st);
template <typename T>
cudaError_t field_energy(const T* E, const T* B, GridP g, double* partial, int nblocks,
                         cudaStream_t st);
template <typename T>
cudaError_t mass_to_double(const T* M, const T* J, double* Md, double* Jd, GridP g,
                           cudaStream_t st);
template <typename T>
cudaError_t mass_from_double(const double* Md, const double* Jd, T* M, T* J, GridP g, int* bad,
                             cudaStream_t st);
int field_grid_blocks(GridP g);

// GMRES vector kernels: FP64 vectors, or double-float ones when df (the
// sums and dot products then come out in FP64 per block)
cudaError_t gm_dots(const double* V, int64_t ldv, int k, const double* w, int64_t n,
                    double* partial, int nblocks, cudaStream_t st, int df);     // k dots + w.w
cudaError_t gm_update(double* w, const double* V, int64_t ldv, int k, const double* h,
                      int64_t n, double* partial, int nblocks, cudaStream_t st, int df);  // w -= V h; |w|^2
cudaError_t gm_scale(double* dst, const double* src, double s, int64_t n, cudaStream_t st, int df);
// vout = (w - V h)/hn with hn^2 = hw[k] - |h|^2, h = hw[0..k-1]
cudaError_t gm_update_scale(const double* w, const double* V, int64_t ldv, int k, const double* hw,
                            double* vout, int64_t n, cudaStream_t st, int df);
cudaError_t gm_sub(double* r, const double* b, const double* Ax, int64_t n, double* partial,
                   int nblocks, cudaStream_t st, int df);                      // r = b - Ax; |r|^2
cudaError_t gm_combine(double* x, const double* V, int64_t ldv, int k, const double* y,
                       int64_t n, cudaStream_t st, int df);                    // x += V y
cudaError_t gm_combine_dev(double* x, const double* V, int64_t ldv, const int* k, const double* y,
                           int64_t n, cudaStream_t st, int df);                // x += V y, k read on the device
cudaError_t reduce_partials(const double* partial, int nblocks, int nsums, double* out,
                            cudaStream_t st);
int gm_blocks(int64_t n);

// adjoint of the field part of a step (FP64; gEt and lambda are GMRES
// vectors, double-float when g.df): gEt = gE1/theta - dt curl_n gB1 (+ gEx);
// after A^T lambda = gEt: gE0, gB0, gJ (each may be null) and the gradient of
// the stored mass-matrix blocks (ncell x 45)
cudaError_t adjoint_pre(const double* gE1, const double* gB1, const double* gEx, double* gEt, GridP g,
                        cudaStream_t st);   // gEx (may be null): a further dL/dE^{n+theta} term
cudaError_t adjoint_post(const double* gE1, const double* gB1, const double* lam, double* gE0, double* gB0,
                         double* gJ, GridP g, cudaStream_t st);
template <typename T>
cudaError_t adjoint_mass(const double* lam, const T* Et, double* gM, GridP g, cudaStream_t st);

// ----- device-side GMRES control (gmres.cu) -----
// Launch arguments of the next Arnoldi iteration, written by the device (the
// cycle start or the previous iteration's tail) and read by the iteration's
// kernels, so that no host decision sits between two iterations.
struct GmDyn {
    const double* in;   // v_j unscaled: r for j = 0, V_j after
    double* vj;         // where v_j = s in is written (V_0 for j = 0), or null
    double* out;        // w_j = B v_j
    double* ds;         // the j + 2 sums <w,V_0..V_{j-1}>, <w,v_j>, <w,w>
    double s;           // 1/beta for j = 0, else 1
    int nv;             // j
    int live;           // 0: the iteration is not to run (its kernels return)
};
// The solve's control state on the device. The head (up to H) is what the
// host reads back after a solve.
struct GmState {
    GmDyn dyn;
    double bnorm, beta, relres;
    int total, restarts, kdim, run, inner, status, zero, pad;
    double cs[kMaxRestart], sn[kMaxRestart], gv[kMaxRestart + 1], y[kMaxRestart];
    double H[(kMaxRestart + 1) * kMaxRestart];
};
enum { kGmOk = 0, kGmNotConverged = 1, kGmNonfinite = 2 };
// The fixed pointers the control kernels build launch arguments from.
struct GmPtrs {
    double* r;       // residual / first Krylov vector (also w of odd j)
    double* w0;      // w of even j
    double* V;       // Krylov basis, ldv apart
    double* ds0;     // sums of even j
    double* ds1;     // sums of odd j
    int64_t ldv;
};
struct GmParams {
    double tol;
    int m, maxit;
};
// a graph loop condition the control kernels set (has = 0: host-driven)
struct GmCond {
    unsigned long long h;
    int has;
};
// bnorm from |b|^2 = sums[0]; resets the counters
cudaError_t gm_begin(GmState* st, const double* sums, cudaStream_t s);
// x = 0 when b = 0 (the exact solution); no-op otherwise
cudaError_t gm_zero_x(const GmState* st, double* x, int64_t n, cudaStream_t s);
// after r = b - A x, |r|^2 = sums[0]: converged / out of iterations / start
// a cycle (launch arguments of iteration 0); sets the cycle condition
cudaError_t gm_cycle(GmState* st, const double* sums, GmPtrs p, GmParams q, GmCond cond, cudaStream_t s);
// sets the Arnoldi-loop condition to the state's "run"
cudaError_t gm_arm(const GmState* st, GmCond cond, cudaStream_t s);
// after iteration j's sums: Hessenberg column, Givens rotation, residual
// estimate, stop test, launch arguments of iteration j + 1; sets the
// Arnoldi-loop condition
cudaError_t gm_tail(GmState* st, GmPtrs p, GmParams q, GmCond cond, cudaStream_t s);
// y from the triangular system of the finished cycle; x += V y
cudaError_t gm_finish_cycle(GmState* st, double* x, const double* V, int64_t ldv, int64_t n, int m,
                            cudaStream_t s, int df);
// Arnoldi iteration kernels reading their arguments from dyn
template <typename T>
cudaError_t op_arnoldi_dyn(const T* M, const GmDyn* dyn, const double* V, int64_t ldv, GridP g,
                           double* partial, int* err, cudaStream_t st, bool tr = false);
cudaError_t reduce_partials_dyn(const double* partial, int nblocks, const GmDyn* dyn, int maxsums,
                                cudaStream_t st);
cudaError_t gm_update_scale_dyn(const GmDyn* dyn, const double* V, int64_t ldv, int64_t n, cudaStream_t st,
                                int df);

// ----- diag.cu -----
// tw[2 (m nx + i) + {0, 1}] = cos, sin of 2 pi ((m i) mod nx) / nx, m < nmodes
template <typename T>
cudaError_t mode_twiddles(T* tw, int nx, int nmodes, cudaStream_t st);
// out[m] = (1/2) dV (c_m / nx) sum_j |sum_i Bc(i,j) e^{-2 pi i m i/nx}|^2 for
// m < nmodes (Bc: one component, ny rows of nx); rows: nmodes * ny doubles
template <typename T>
cudaError_t field_modes(const T* Bc, const T* tw, int nx, int ny, int nmodes, double dV, double* rows,
                        double* out, cudaStream_t st);
// *energy = the mode-m energy as above and g[j nx + i] = its derivative in
// Bc(i, j) (FP64); rows: ny doubles; tw must hold mode m
template <typename T>
cudaError_t mode_gradient(const T* Bc, const T* tw, int nx, int ny, int m, double dV, double* rows,
                          double* energy, double* g, cudaStream_t st);

}  // namespace relsim

// ----- capi.cu: what the batch runner needs of a context -----
struct relsim_ctx;
namespace relsim {
cudaStream_t ctx_stream(const relsim_ctx* c);
int ctx_last_iters(const relsim_ctx* c);
int64_t ctx_particles(const relsim_ctx* c);
// graph steps enqueued without waiting: prepare captures both buffer layouts
// (1: ready; 0: this context steps from the host); enqueue launches one
// step and copies its solve outcome (head_bytes) to the pinned host buffer
// head; outcome reads one such head after the stream was synchronised
size_t ctx_graph_head_bytes();
int ctx_graph_prepare(relsim_ctx* c);
int ctx_graph_enqueue(relsim_ctx* c, void* head);
int ctx_graph_outcome(relsim_ctx* c, const void* head, int* iters);
}  // namespace relsim

// shared launches over the instances of a batch (capi.cu): create returns 1
// and *out when every instance qualifies (then both layouts are captured),
// 0 when one does not, or a negative error; enqueue launches one step of all
// instances on the shared stream and copies each instance's solve outcome
// to heads + i head_stride; outcome reads instance i's after the stream was
// synchronised (first: count the shared kernels once per step)
struct relsim_shared;
namespace relsim {
int shared_create(relsim_ctx* const* ctxs, int count, int dep_blocks, int push_blocks, relsim_shared** out);
void shared_destroy(relsim_shared* sb);
cudaStream_t shared_stream(const relsim_shared* sb);
int shared_enqueue(relsim_shared* sb, unsigned char* heads, size_t head_stride);
// the shared graphs still fit these instances (same contexts and grids, no
// reload, retune or lone step since the capture)
bool shared_valid(const relsim_shared* sb, relsim_ctx* const* ctxs, int count, int dep_blocks, int push_blocks);
int shared_outcome(relsim_shared* sb, int i, const void* head, int* iters, bool first);
}  // namespace relsim
