// capi.cu -- the C ABI declared in include/relsim.h: context, device
// buffers, particle load and export, and the step orchestration (deposit,
// restarted GMRES with an FP64 Krylov basis, field update, push + sort).
#include <atomic>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <limits>
#include <new>
#include <string>
#include <vector>

#include "launch.cuh"
#include "relsim.h"

namespace relsim {
static std::atomic<long long> g_launches{0};
void count_launches(int n) { g_launches.fetch_add(n, std::memory_order_relaxed); }
}  // namespace relsim

using namespace relsim;

namespace {

enum State { kEmpty = 0, kReady = 1, kBuilt = 2, kSolved = 3 };

constexpr int kLedgerField = 6;    // dW_E, dW_B, dissipation, W_E1, W_B1, work_grid
constexpr int kLedgerSpecies = 5;  // K0, dK, work, mismatch, K1
constexpr int kLedgerLen = kLedgerField + kLedgerSpecies * kMaxSpecies + 2;   // + W_E0, W_B0

struct Species {
    int64_t n = 0, cap = 0;
    void* a[2][6] = {};   // fx, fy, ux, uy, uz, w of buffer 0 and 1
    int32_t* id[2] = {nullptr, nullptr};
    int cur = 0;
    int32_t* start = nullptr;
    int32_t* start_alt = nullptr;
};

// CUDA-event timing of launch groups (enabled on demand)
struct Prof {
    bool on = false;
    std::vector<cudaEvent_t> pool;
    size_t used = 0;
    struct Rec {
        int slot;
        size_t e0, e1;
        long long kernels;
    };
    std::vector<Rec> recs;
    double ms[16] = {};
    long long groups[16] = {};
    long long kernels[16] = {};
    int open_slot = -1;
    size_t open_ev = 0;
    long long open_k = 0;
};

}  // namespace

struct relsim_ctx {
    relsim_config cfg;
    cudaStream_t st = 0;
    int prec = 32;
    size_t esz = 4;
    GridP g;
    bool fast_sort = true;
    int key_bits = 1;
    Species sp[kMaxSpecies];
    void* E = nullptr;
    void* Eth = nullptr;
    void* B[2] = {nullptr, nullptr};
    int bcur = 0;
    void* J = nullptr;
    void* M = nullptr;
    int32_t* n9 = nullptr;
    int32_t* off9 = nullptr;
    int32_t* count_new = nullptr;
    int32_t* scan_tmp = nullptr;
    size_t scan_tmp_n = 0;
    // radix scratch (grown on demand)
    int32_t* rk[2] = {nullptr, nullptr};
    int32_t* rv[2] = {nullptr, nullptr};
    int32_t* rtmp = nullptr;
    int64_t rcap = 0;
    // GMRES
    int mrest = 30;
    int64_t nvec = 0;
    double* V = nullptr;
    double* gw = nullptr;
    double* gw2 = nullptr;
    double* gx = nullptr;
    double* gb = nullptr;
    double* partial = nullptr;
    int64_t partial_cap = 0;
    double* dsum = nullptr;    // small device results (>= 2*(kMaxRestart+2))
    double* dled = nullptr;    // ledger sums, kLedgerLen
    double* hpin = nullptr;    // pinned host, 4*(kMaxRestart+2)
    int* dflag = nullptr;
    int* hflag = nullptr;
    cudaEvent_t gev[2] = {nullptr, nullptr};   // read-back events of the pipelined Arnoldi loop
    int* dpush = nullptr;     // set by the push if its two passes ever disagree
    int* hpush = nullptr;
    // spectrum diagnostic (grown on demand)
    double* spec_w = nullptr;
    unsigned long long* spec_c = nullptr;
    void* spec_e = nullptr;
    int spec_cap = 0;   // bins
    // field-mode diagnostic: twiddles for modes < mode_tw_m, row sums
    void* mode_tw = nullptr;
    int mode_tw_m = 0;
    double* mode_rows = nullptr;
    int64_t mode_rows_cap = 0;   // doubles
    // staging for host <-> device copies
    double* stage = nullptr;
    int64_t stage_cap = 0;   // doubles
    int state = kEmpty;
    bool have_step = false;
    int64_t step = 0;
    int last_iters = 0, last_restarts = 0;
    double last_relres = 0.0;
    Prof prof;
    std::string err;
};

namespace {

int fail(relsim_ctx* c, int code, const char* fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    if (c) c->err = buf;
    return code;
}

int check_push(relsim_ctx* c);

#define CK(call)                                                                             \
    do {                                                                                     \
        cudaError_t e_ = (call);                                                             \
        if (e_ != cudaSuccess)                                                               \
            return fail(c, RELSIM_ERR_CUDA, "%s: %s", #call, cudaGetErrorString(e_));        \
    } while (0)

int prof_flush(relsim_ctx* c)
{
    Prof& P = c->prof;
    if (P.recs.empty()) return RELSIM_OK;
    CK(cudaStreamSynchronize(c->st));
    for (const Prof::Rec& r : P.recs) {
        float ms = 0.f;
        CK(cudaEventElapsedTime(&ms, P.pool[r.e0], P.pool[r.e1]));
        P.ms[r.slot] += ms;
        P.groups[r.slot] += 1;
        P.kernels[r.slot] += r.kernels;
    }
    P.recs.clear();
    P.used = 0;
    return RELSIM_OK;
}

// open a timed group on the context's stream (no-op when profiling is off)
int prof_begin(relsim_ctx* c, int slot)
{
    Prof& P = c->prof;
    if (!P.on) return RELSIM_OK;
    if (P.used + 2 > P.pool.size()) {
        int r = prof_flush(c);
        if (r != RELSIM_OK) return r;
    }
    P.open_slot = slot;
    P.open_ev = P.used++;
    P.open_k = g_launches.load(std::memory_order_relaxed);
    CK(cudaEventRecord(P.pool[P.open_ev], c->st));
    return RELSIM_OK;
}

int prof_end(relsim_ctx* c)
{
    Prof& P = c->prof;
    if (!P.on || P.open_slot < 0) return RELSIM_OK;
    size_t e1 = P.used++;
    CK(cudaEventRecord(P.pool[e1], c->st));
    P.recs.push_back({P.open_slot, P.open_ev, e1,
                      g_launches.load(std::memory_order_relaxed) - P.open_k});
    P.open_slot = -1;
    return RELSIM_OK;
}

#define PROF_BEGIN(slot) TRY(prof_begin(c, slot))
#define PROF_END() TRY(prof_end(c))

template <class P>
int dalloc(relsim_ctx* c, P** p, size_t bytes)
{
    *p = nullptr;
    if (bytes == 0) bytes = 16;
    cudaError_t e = cudaMalloc((void**)p, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        return fail(c, e == cudaErrorMemoryAllocation ? RELSIM_ERR_OOM : RELSIM_ERR_CUDA,
                    "cudaMalloc(%zu bytes): %s", bytes, cudaGetErrorString(e));
    }
    return RELSIM_OK;
}

template <class P>
void dfree(P*& p)
{
    if (p) cudaFree((void*)p);
    p = nullptr;
}

#define TRY(x)                     \
    do {                           \
        int r_ = (x);              \
        if (r_ != RELSIM_OK) return r_; \
    } while (0)

template <typename T>
PArrays<T> arrays(Species& s, int buf)
{
    PArrays<T> p;
    p.fx = (T*)s.a[buf][0];
    p.fy = (T*)s.a[buf][1];
    p.ux = (T*)s.a[buf][2];
    p.uy = (T*)s.a[buf][3];
    p.uz = (T*)s.a[buf][4];
    p.w = (T*)s.a[buf][5];
    p.id = s.id[buf];
    return p;
}

int ensure_stage(relsim_ctx* c, int64_t ndoubles)
{
    if (ndoubles <= c->stage_cap) return RELSIM_OK;
    dfree(c->stage);
    c->stage_cap = 0;
    TRY(dalloc(c, &c->stage, sizeof(double) * (size_t)ndoubles));
    c->stage_cap = ndoubles;
    return RELSIM_OK;
}

int ensure_radix(relsim_ctx* c, int64_t n)
{
    if (n <= c->rcap) return RELSIM_OK;
    for (int b = 0; b < 2; ++b) {
        dfree(c->rk[b]);
        dfree(c->rv[b]);
    }
    dfree(c->rtmp);
    c->rcap = 0;
    for (int b = 0; b < 2; ++b) {
        TRY(dalloc(c, &c->rk[b], sizeof(int32_t) * (size_t)n));
        TRY(dalloc(c, &c->rv[b], sizeof(int32_t) * (size_t)n));
    }
    size_t t = radix_tmp_ints(n);
    size_t s2 = scan_tmp_ints(n);
    TRY(dalloc(c, &c->rtmp, sizeof(int32_t) * (t > s2 ? t : s2)));
    c->rcap = n;
    return RELSIM_OK;
}

int ensure_partial(relsim_ctx* c, int64_t n)
{
    if (n <= c->partial_cap) return RELSIM_OK;
    dfree(c->partial);
    c->partial_cap = 0;
    TRY(dalloc(c, &c->partial, sizeof(double) * (size_t)n));
    c->partial_cap = n;
    return RELSIM_OK;
}

int ensure_species(relsim_ctx* c, int s, int64_t n)
{
    Species& sp = c->sp[s];
    if (!sp.start) {
        TRY(dalloc(c, &sp.start, sizeof(int32_t) * (size_t)(c->g.ncell + 1)));
        TRY(dalloc(c, &sp.start_alt, sizeof(int32_t) * (size_t)(c->g.ncell + 1)));
    }
    if (n <= sp.cap) return RELSIM_OK;
    for (int b = 0; b < 2; ++b) {
        for (int k = 0; k < 6; ++k) dfree(sp.a[b][k]);
        dfree(sp.id[b]);
    }
    sp.cap = 0;
    for (int b = 0; b < 2; ++b) {
        for (int k = 0; k < 6; ++k) TRY(dalloc(c, &sp.a[b][k], c->esz * (size_t)(n + 8)));
        if (c->cfg.track_ids) TRY(dalloc(c, &sp.id[b], sizeof(int32_t) * (size_t)n));
    }
    sp.cap = n;
    return RELSIM_OK;
}

// copy a caller array to the device (or use it in place). Page-locked host
// memory that is mapped into the device's address space is read in place by
// the consuming kernel, over the host link, with no staging copy; the caller
// synchronises before returning, so no caller pointer outlives the call.
int stage_in(relsim_ctx* c, const double* src, int64_t count, int where, const double** dev,
             int64_t stage_off)
{
    if (where == RELSIM_DEVICE) {
        *dev = src;
        return RELSIM_OK;
    }
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, src) == cudaSuccess && at.type == cudaMemoryTypeHost && at.devicePointer) {
        *dev = (const double*)at.devicePointer;
        return RELSIM_OK;
    }
    (void)cudaGetLastError();   // an unregistered pointer is not an error here
    CK(cudaMemcpyAsync(c->stage + stage_off, src, sizeof(double) * (size_t)count,
                       cudaMemcpyHostToDevice, c->st));
    *dev = c->stage + stage_off;
    return RELSIM_OK;
}

int check_flag(relsim_ctx* c, const char* what)
{
    CK(cudaMemcpyAsync(c->hflag, c->dflag, sizeof(int), cudaMemcpyDeviceToHost, c->st));
    CK(cudaStreamSynchronize(c->st));
    if (*c->hflag) return fail(c, RELSIM_ERR_NONFINITE, "non-finite value in %s", what);
    return RELSIM_OK;
}

template <typename T>
int load_impl(relsim_ctx* c, int s, int64_t n, const double* x, const double* u, const double* w,
              int where)
{
    Species& sp = c->sp[s];
    TRY(ensure_species(c, s, n));
    sp.n = n;
    sp.cur = 0;
    if (n == 0) {
        CK(cudaMemsetAsync(sp.start, 0, sizeof(int32_t) * (size_t)(c->g.ncell + 1), c->st));
    } else {
        const double *dx, *du, *dw;
        if (where == RELSIM_HOST) TRY(ensure_stage(c, 6 * n));
        TRY(stage_in(c, x, 2 * n, where, &dx, 0));
        TRY(stage_in(c, u, 3 * n, where, &du, 2 * n));
        TRY(stage_in(c, w, n, where, &dw, 5 * n));
        TRY(ensure_radix(c, n));
        CK(cudaMemsetAsync(c->dflag, 0, sizeof(int), c->st));
        PROF_BEGIN(RELSIM_PROF_LOAD);
        PArrays<T> tmp = arrays<T>(sp, 1), dst = arrays<T>(sp, 0);
        CK(load_convert<T>(dx, du, dw, n, c->g, tmp, c->rk[0], c->rv[0], c->dflag, c->st));
        CK(keys_unsorted(c->rk[0], n, c->dflag, c->st));
        PROF_END();
        CK(cudaMemcpyAsync(c->hflag, c->dflag, sizeof(int), cudaMemcpyDeviceToHost, c->st));
        CK(cudaStreamSynchronize(c->st));
        if (*c->hflag & 1) return fail(c, RELSIM_ERR_NONFINITE, "non-finite value in particles");
        PROF_BEGIN(RELSIM_PROF_LOAD);
        const int32_t* keys = c->rk[0];
        if (*c->hflag & 2) {
            // the stable sort by cell, then the particles gathered in that order
            bool in1 = false;
            CK(radix_sort_pairs(c->rk[0], c->rv[0], c->rk[1], c->rv[1], n, c->key_bits, c->rtmp, &in1,
                                c->st));
            keys = c->rk[in1 ? 1 : 0];
            const int32_t* perm = c->rv[in1 ? 1 : 0];
            CK(gather_particles<T>(perm, tmp, dst, n, true, c->st));
        } else {
            // already in cell order (e.g. state read back from this library):
            // the identity is the stable sort, and the converted buffer stays
            sp.cur = 1;
            if (tmp.id)
                CK(cudaMemcpyAsync(tmp.id, c->rv[0], sizeof(int32_t) * (size_t)n, cudaMemcpyDeviceToDevice, c->st));
        }
        CK(histogram_keys(keys, n, c->count_new, c->g.ncell, c->st));
        CK(scan_exclusive_i32(c->count_new, sp.start, c->g.ncell, sp.start + c->g.ncell, c->scan_tmp,
                              c->st));
        PROF_END();
    }
    // kinetic energy of the loaded species -> ledger slot K1
    const int nb = 152 * 4;
    TRY(ensure_partial(c, nb));
    CK(cudaMemsetAsync(c->dled + kLedgerField + kLedgerSpecies * s, 0, sizeof(double) * kLedgerSpecies,
                       c->st));
    if (n > 0) {
        CK(kinetic_energy<T>(arrays<T>(sp, sp.cur), n, c->cfg.m[s], c->partial, nb, c->st));
        CK(reduce_partials(c->partial, nb, 1, c->dled + kLedgerField + kLedgerSpecies * s + 4, c->st));
    }
    return RELSIM_OK;
}

template <typename T>
int field_energy_now(relsim_ctx* c)
{
    const int nb = 152 * 4;
    TRY(ensure_partial(c, 2 * nb));
    CK(field_energy<T>((const T*)c->E, (const T*)c->B[c->bcur], c->g, c->partial, nb, c->st));
    CK(reduce_partials(c->partial, nb, 2, c->dled + 3, c->st));
    return RELSIM_OK;
}

template <typename T>
int set_fields_impl(relsim_ctx* c, const double* E, const double* B, int where)
{
    const int64_t n = 3 * (int64_t)c->g.ncell;
    if (where == RELSIM_HOST) TRY(ensure_stage(c, 2 * n));
    CK(cudaMemsetAsync(c->dflag, 0, sizeof(int), c->st));
    if (E) {
        const double* d;
        TRY(stage_in(c, E, n, where, &d, 0));
        CK(fields_from_double<T>(d, (T*)c->E, n, c->dflag, c->st));
    }
    if (B) {
        const double* d;
        TRY(stage_in(c, B, n, where, &d, n));
        CK(fields_from_double<T>(d, (T*)c->B[c->bcur], n, c->dflag, c->st));
    }
    TRY(check_flag(c, "fields"));
    return field_energy_now<T>(c);
}

int copy_out(relsim_ctx* c, double* dst, const double* dev, int64_t count, int where)
{
    if (where == RELSIM_DEVICE) {
        if (dst != dev)
            CK(cudaMemcpyAsync(dst, dev, sizeof(double) * (size_t)count, cudaMemcpyDeviceToDevice, c->st));
        return RELSIM_OK;
    }
    CK(cudaMemcpyAsync(dst, dev, sizeof(double) * (size_t)count, cudaMemcpyDeviceToHost, c->st));
    CK(cudaStreamSynchronize(c->st));
    return RELSIM_OK;
}

template <typename T>
int get_fields_impl(relsim_ctx* c, double* E, double* B, int where)
{
    const int64_t n = 3 * (int64_t)c->g.ncell;
    const int bnow = c->state == kSolved ? 1 - c->bcur : c->bcur;
    for (int f = 0; f < 2; ++f) {
        double* out = f == 0 ? E : B;
        if (!out) continue;
        const T* src = (const T*)(f == 0 ? c->E : c->B[bnow]);
        double* dst = out;
        if (where == RELSIM_HOST) {
            TRY(ensure_stage(c, n));
            dst = c->stage;
        }
        CK(fields_to_double<T>(src, dst, n, c->st));
        TRY(copy_out(c, out, dst, n, where));
    }
    return RELSIM_OK;
}

template <typename T>
int get_particles_impl(relsim_ctx* c, int s, double* x, double* u, double* w, int32_t* id, int where)
{
    Species& sp = c->sp[s];
    const int64_t n = sp.n;
    if (n == 0) return RELSIM_OK;
    PArrays<T> pa = arrays<T>(sp, sp.cur);
    if (where == RELSIM_DEVICE) {
        CK(export_particles<T>(pa, sp.start, c->g, x, u, w, id, c->st));
        return RELSIM_OK;
    }
    TRY(ensure_stage(c, 6 * n + (n + 1) / 2));
    double* dx = x ? c->stage : nullptr;
    double* du = u ? c->stage + 2 * n : nullptr;
    double* dw = w ? c->stage + 5 * n : nullptr;
    int32_t* did = id ? (int32_t*)(c->stage + 6 * n) : nullptr;
    CK(export_particles<T>(pa, sp.start, c->g, dx, du, dw, did, c->st));
    if (x) CK(cudaMemcpyAsync(x, dx, sizeof(double) * 2 * n, cudaMemcpyDeviceToHost, c->st));
    if (u) CK(cudaMemcpyAsync(u, du, sizeof(double) * 3 * n, cudaMemcpyDeviceToHost, c->st));
    if (w) CK(cudaMemcpyAsync(w, dw, sizeof(double) * n, cudaMemcpyDeviceToHost, c->st));
    if (id) CK(cudaMemcpyAsync(id, did, sizeof(int32_t) * n, cudaMemcpyDeviceToHost, c->st));
    CK(cudaStreamSynchronize(c->st));
    return RELSIM_OK;
}

template <typename T>
int build_impl(relsim_ctx* c)
{
    const int nc = c->g.ncell;
    PROF_BEGIN(RELSIM_PROF_DEPOSIT);
    CK(cudaMemsetAsync(c->M, 0, c->esz * (size_t)nc * kMBlock, c->st));
    CK(cudaMemsetAsync(c->J, 0, c->esz * 3 * (size_t)nc, c->st));
    DepositSpecies<T> ds;
    memset(&ds, 0, sizeof(ds));
    ds.nsp = c->cfg.nspecies;
    for (int s = 0; s < ds.nsp; ++s) {
        Species& sp = c->sp[s];
        PArrays<T> pa = arrays<T>(sp, sp.cur);
        ds.fx[s] = pa.fx;
        ds.fy[s] = pa.fy;
        ds.ux[s] = pa.ux;
        ds.uy[s] = pa.uy;
        ds.uz[s] = pa.uz;
        ds.w[s] = pa.w;
        ds.start[s] = sp.start;
        const double beta = c->cfg.q[s] * c->g.dt / (2.0 * c->cfg.m[s]);
        ds.beta[s] = (T)beta;
        ds.cJ[s] = (T)(c->cfg.q[s] / c->g.dV);
        ds.cM[s] = (T)(c->cfg.q[s] * beta / c->g.dV);
    }
    CK(deposit<T>(ds, (const T*)c->B[c->bcur], (T*)c->M, (T*)c->J, c->g, c->dpush, c->st));
    PROF_END();
    return RELSIM_OK;
}

// read back count reduced values (and the kernels' error flags) after a sync
int readback(relsim_ctx* c, const double* dev, int count, double* host)
{
    CK(cudaMemcpyAsync(host, dev, sizeof(double) * (size_t)count, cudaMemcpyDeviceToHost, c->st));
    CK(cudaMemcpyAsync(c->hpush, c->dpush, sizeof(int), cudaMemcpyDeviceToHost, c->st));
    CK(cudaStreamSynchronize(c->st));
    return RELSIM_OK;
}

template <typename T>
int solve_impl(relsim_ctx* c, int* iters_out, double* relres_out)
{
    // Restarted GMRES on A = I + B. The Arnoldi process runs on B (the same
    // Krylov space: A V_k = V_k + B V_k, so the Hessenberg matrix of A is that
    // of B plus the identity). Working on B avoids the cancellation of
    // orthogonalising A v ~ v against v, and keeps the identity exact in FP64.
    const int64_t n = c->nvec;
    const int64_t ldv = n;
    const int m = c->mrest;
    const int nb = gm_blocks(n);
    const int nbo = op_blocks(c->g, c->prec);
    TRY(ensure_partial(c, (int64_t)(nb > nbo ? nb : nbo) * (m + 2)));
    const double tol = c->cfg.gmres_tol;
    const int maxit = c->cfg.gmres_maxit;
    double* hp = c->hpin;                      // readback area
    double* yp = c->hpin + 2 * (kMaxRestart + 2);   // y upload area
    double* dy = c->dsum + 2 * (kMaxRestart + 2);
    double H[(kMaxRestart + 1) * kMaxRestart];
    double cs[kMaxRestart], sn[kMaxRestart], gv[kMaxRestart + 1], y[kMaxRestart];
    double* gw[2] = {c->gw, c->gw2};

    PROF_BEGIN(RELSIM_PROF_RHS);
    CK(rhs<T>((const T*)c->E, (const T*)c->B[c->bcur], (const T*)c->J, c->gb, c->g, c->st));
    CK(fields_to_double<T>((const T*)c->E, c->gx, n, c->st));
    PROF_END();
    CK(gm_dots(c->V, ldv, 0, c->gb, n, c->partial, nb, c->st));
    CK(reduce_partials(c->partial, nb, 1, c->dsum, c->st));
    TRY(readback(c, c->dsum, 1, hp));
    TRY(check_push(c));
    const double bnorm = std::sqrt(hp[0]);
    if (!std::isfinite(bnorm)) return fail(c, RELSIM_ERR_NONFINITE, "non-finite right-hand side");
    int total = 0, restarts = 0, status = RELSIM_OK;
    double relres = 0.0;
    if (bnorm == 0.0) {
        CK(cudaMemsetAsync(c->gx, 0, sizeof(double) * (size_t)n, c->st));
    } else {
        for (;;) {
            // r = b - A x (unnormalised first Krylov vector) and |r|^2
            PROF_BEGIN(RELSIM_PROF_GMRES_APPLY);
            CK(op_residual<T>((const T*)c->M, c->gx, c->gb, gw[0], c->g, c->partial, c->dpush, c->st));
            CK(reduce_partials(c->partial, nbo, 1, c->dsum, c->st));
            PROF_END();
            TRY(readback(c, c->dsum, 1, hp));
            TRY(check_push(c));
            const double beta = std::sqrt(hp[0]);
            if (!std::isfinite(beta)) return fail(c, RELSIM_ERR_NONFINITE, "non-finite residual");
            relres = beta / bnorm;
            if (relres <= tol) break;
            if (total >= maxit) {
                status = fail(c, RELSIM_ERR_NOT_CONVERGED,
                              "GMRES reached %d iterations at relative residual %.3e", total, relres);
                break;
            }
            for (int k = 0; k <= m; ++k) gv[k] = 0.0;
            gv[0] = beta;
            int kdim = 0;
            // Iteration j: w_j = B v_j (v_0 = r/|r|, written to V_0 on the
            // way) with the dot products <w_j, V_i> (i <= j) and <w_j, w_j>,
            // then V_{j+1} = (w_j - V h)/hn, hn^2 = <w,w> - |h|^2 formed on
            // the device (classical Gram-Schmidt with the normalisation
            // fused). Nothing of it waits for the host, so iteration j+1 is
            // launched before the host reads iteration j's sums back; w, the
            // device sums and the host read-back alternate between two slots.
            double* ws[2] = {gw[1], gw[0]};   // gw[0] holds r until iteration 0 has read it
            double* dss[2] = {c->dsum, c->dsum + 3 * (kMaxRestart + 2)};
            double* hps[2] = {c->hpin, c->hpin + (kMaxRestart + 2)};
            auto launch_iter = [&](int j) -> int {
                double* w = ws[j % 2];
                double* ds = dss[j % 2];
                PROF_BEGIN(RELSIM_PROF_GMRES_APPLY);
                if (j == 0)
                    CK(op_arnoldi<T>((const T*)c->M, gw[0], 1.0 / beta, c->V, w, c->V, ldv, 0, c->g, c->partial,
                                     c->dpush, c->st));
                else
                    CK(op_arnoldi<T>((const T*)c->M, c->V + (int64_t)j * ldv, 1.0, nullptr, w, c->V, ldv, j, c->g,
                                     c->partial, c->dpush, c->st));
                PROF_END();
                PROF_BEGIN(RELSIM_PROF_GMRES_ORTHO);
                CK(reduce_partials(c->partial, nbo, j + 2, ds, c->st));
                CK(gm_update_scale(w, c->V, ldv, j + 1, ds, c->V + (int64_t)(j + 1) * ldv, n, c->st));
                PROF_END();
                CK(cudaMemcpyAsync(hps[j % 2], ds, sizeof(double) * (size_t)(j + 2), cudaMemcpyDeviceToHost, c->st));
                CK(cudaMemcpyAsync(c->hpush, c->dpush, sizeof(int), cudaMemcpyDeviceToHost, c->st));
                CK(cudaEventRecord(c->gev[j % 2], c->st));
                return RELSIM_OK;
            };
            TRY(launch_iter(0));
            for (int j = 0; j < m; ++j) {
                const bool more = j + 1 < m && total + 1 < maxit;   // could iteration j+1 run?
                // launch it ahead unless the residual's geometric trend says
                // iteration j converges (a launch ahead is then wasted work)
                // (|sin| of the previous rotation is the last reduction factor)
                const bool last = j >= 1 && std::fabs(gv[j]) * std::fabs(sn[j - 1]) <= tol * bnorm;
                const bool ahead = more && !last;
                if (ahead) TRY(launch_iter(j + 1));
                CK(cudaEventSynchronize(c->gev[j % 2]));
                TRY(check_push(c));
                const double* hj = hps[j % 2];
                const double ww = hj[j + 1];
                double hn2 = ww;
                for (int i = 0; i <= j; ++i) {
                    H[i * m + j] = hj[i];
                    hn2 -= hj[i] * hj[i];
                }
                if (!std::isfinite(hn2)) return fail(c, RELSIM_ERR_NONFINITE, "non-finite Arnoldi norm");
                if (hn2 < 1e-4 * ww) {
                    // |w - V h| < |w|/100: the norm above has lost digits.
                    // Drain the speculative iteration, orthogonalise w_j twice
                    // explicitly (CGS2), normalise it into V_{j+1}, and launch
                    // iteration j+1 again.
                    CK(cudaStreamSynchronize(c->st));
                    double* w = ws[j % 2];
                    double* scratch = dss[(j + 1) % 2];
                    PROF_BEGIN(RELSIM_PROF_GMRES_ORTHO);
                    CK(gm_update(w, c->V, ldv, j + 1, dss[j % 2], n, c->partial, nb, c->st));
                    CK(gm_dots(c->V, ldv, j + 1, w, n, c->partial, nb, c->st));
                    CK(reduce_partials(c->partial, nb, j + 2, scratch, c->st));
                    CK(gm_update(w, c->V, ldv, j + 1, scratch, n, c->partial, nb, c->st));
                    CK(reduce_partials(c->partial, nb, 1, scratch + kMaxRestart + 1, c->st));
                    PROF_END();
                    TRY(readback(c, scratch, kMaxRestart + 2, hp));
                    for (int i = 0; i <= j; ++i) H[i * m + j] += hp[i];
                    hn2 = hp[kMaxRestart + 1];
                    if (!std::isfinite(hn2)) return fail(c, RELSIM_ERR_NONFINITE, "non-finite Arnoldi norm");
                    if (hn2 > 0.0) {
                        PROF_BEGIN(RELSIM_PROF_GMRES_ORTHO);
                        CK(gm_scale(c->V + (int64_t)(j + 1) * ldv, w, 1.0 / std::sqrt(hn2), n, c->st));
                        PROF_END();
                    }
                    if (ahead) TRY(launch_iter(j + 1));
                }
                const double hn = std::sqrt(hn2 > 0.0 ? hn2 : 0.0);
                H[j * m + j] += 1.0;   // A = I + B
                H[(j + 1) * m + j] = hn;
                for (int i = 0; i < j; ++i) {
                    const double t = cs[i] * H[i * m + j] + sn[i] * H[(i + 1) * m + j];
                    H[(i + 1) * m + j] = -sn[i] * H[i * m + j] + cs[i] * H[(i + 1) * m + j];
                    H[i * m + j] = t;
                }
                const double a = H[j * m + j], b = H[(j + 1) * m + j];
                const double r = std::hypot(a, b);
                cs[j] = r == 0.0 ? 1.0 : a / r;
                sn[j] = r == 0.0 ? 0.0 : b / r;
                H[j * m + j] = r;
                H[(j + 1) * m + j] = 0.0;
                gv[j + 1] = -sn[j] * gv[j];
                gv[j] = cs[j] * gv[j];
                ++total;
                kdim = j + 1;
                // a speculative iteration j+1 still in flight only writes
                // V_{j+2}, its w and its sums: nothing the solution reads
                if (std::fabs(gv[j + 1]) <= tol * bnorm || total >= maxit || hn == 0.0) break;
                if (more && !ahead) TRY(launch_iter(j + 1));
            }
            for (int i = kdim - 1; i >= 0; --i) {
                double s = gv[i];
                for (int k = i + 1; k < kdim; ++k) s -= H[i * m + k] * y[k];
                y[i] = H[i * m + i] != 0.0 ? s / H[i * m + i] : 0.0;
            }
            for (int i = 0; i < kdim; ++i) yp[i] = y[i];
            CK(cudaMemcpyAsync(dy, yp, sizeof(double) * (size_t)kdim, cudaMemcpyHostToDevice, c->st));
            PROF_BEGIN(RELSIM_PROF_GMRES_ORTHO);
            CK(gm_combine(c->gx, c->V, ldv, kdim, dy, n, c->st));
            PROF_END();
            ++restarts;
        }
    }
    // field update and the field side of the ledger
    CK(cudaMemcpyAsync(c->dled + kLedgerLen - 2, c->dled + 3, 2 * sizeof(double),
                       cudaMemcpyDeviceToDevice, c->st));
    const int nbf = field_grid_blocks(c->g);
    TRY(ensure_partial(c, (int64_t)nbf * 6));
    PROF_BEGIN(RELSIM_PROF_FIELD_UPDATE);
    CK(field_update<T>(c->gx, (const T*)c->M, (const T*)c->J, (T*)c->Eth, (T*)c->E,
                       (const T*)c->B[c->bcur], (T*)c->B[1 - c->bcur], c->g, c->partial, nbf, c->st));
    CK(reduce_partials(c->partial, nbf, 6, c->dled, c->st));
    PROF_END();
    c->last_iters = total;
    c->last_restarts = restarts;
    c->last_relres = relres;
    if (iters_out) *iters_out = total;
    if (relres_out) *relres_out = relres;
    return status;
}

template <typename T>
int push_impl(relsim_ctx* c)
{
    const int nbp = push_grid_blocks(c->g, c->prec);
    TRY(ensure_partial(c, (int64_t)nbp * (kLedgerSpecies - 1)));
    for (int s = 0; s < c->cfg.nspecies; ++s) {
        Species& sp = c->sp[s];
        double* led = c->dled + kLedgerField + kLedgerSpecies * s;
        if (sp.n == 0) {
            CK(cudaMemsetAsync(led, 0, sizeof(double) * kLedgerSpecies, c->st));
            continue;
        }
        SpeciesConst sc{c->cfg.q[s], c->cfg.m[s]};
        PArrays<T> src = arrays<T>(sp, sp.cur), dst = arrays<T>(sp, 1 - sp.cur);
        const T* Eth = (const T*)c->Eth;
        const T* B = (const T*)c->B[c->bcur];
        if (c->fast_sort) {
            // push, each old cell written back grouped by move direction
            // into the other buffer; then the stable new-cell order back into
            // the current buffer
            PROF_BEGIN(RELSIM_PROF_PUSH);
            // K0 of this step is the kinetic energy the last push (or load) left
            CK(cudaMemcpyAsync(led, led + 4, sizeof(double), cudaMemcpyDeviceToDevice, c->st));
            CK(push_sort<T>(src, dst, sp.start, c->n9, c->off9, Eth, B, c->g, sc, c->partial, nbp, c->st));
            CK(reduce_partials(c->partial, nbp, kLedgerSpecies - 1, led + 1, c->st));
            PROF_END();
            PROF_BEGIN(RELSIM_PROF_SORT_TABLES);
            CK(move_counts(c->n9, c->count_new, c->g, c->st));
            CK(scan_exclusive_i32(c->count_new, sp.start_alt, c->g.ncell, sp.start_alt + c->g.ncell,
                                  c->scan_tmp, c->st));
            PROF_END();
            PROF_BEGIN(RELSIM_PROF_PERMUTE);
            CK(permute<T>(dst, src, sp.start_alt, c->n9, c->off9, c->g, c->dpush, c->st));
            PROF_END();
            int32_t* t = sp.start;
            sp.start = sp.start_alt;
            sp.start_alt = t;
        } else {
            // general path: push in place order with keys, radix sort, gather
            TRY(ensure_radix(c, sp.n));
            PROF_BEGIN(RELSIM_PROF_GENERAL_SORT);
            CK(cudaMemcpyAsync(led, led + 4, sizeof(double), cudaMemcpyDeviceToDevice, c->st));
            CK(push_general<T>(src, dst, sp.start, c->rk[0], Eth, B, c->g, sc, c->partial, nbp, c->st));
            CK(reduce_partials(c->partial, nbp, kLedgerSpecies - 1, led + 1, c->st));
            CK(iota_i32(c->rv[0], sp.n, c->st));
            bool in1 = false;
            CK(radix_sort_pairs(c->rk[0], c->rv[0], c->rk[1], c->rv[1], sp.n, c->key_bits, c->rtmp,
                                &in1, c->st));
            const int32_t* keys = c->rk[in1 ? 1 : 0];
            const int32_t* perm = c->rv[in1 ? 1 : 0];
            CK(gather_particles<T>(perm, dst, src, sp.n, false, c->st));
            CK(histogram_keys(keys, sp.n, c->count_new, c->g.ncell, c->st));
            CK(scan_exclusive_i32(c->count_new, sp.start, c->g.ncell, sp.start + c->g.ncell,
                                  c->scan_tmp, c->st));
            PROF_END();
        }
    }
    c->bcur = 1 - c->bcur;
    // read back lazily: checked after the next synchronising call
    CK(cudaMemcpyAsync(c->hpush, c->dpush, sizeof(int), cudaMemcpyDeviceToHost, c->st));
    return RELSIM_OK;
}

template <typename T>
int spectrum_impl(relsim_ctx* c, int s, int variable, int nbins, const double* edges, double* weight,
                  int64_t* count, int where)
{
    if (nbins > c->spec_cap) {
        dfree(c->spec_w);
        dfree(c->spec_c);
        dfree(c->spec_e);
        c->spec_cap = 0;
        TRY(dalloc(c, &c->spec_w, sizeof(double) * (size_t)(nbins + 2)));
        TRY(dalloc(c, &c->spec_c, sizeof(unsigned long long) * (size_t)(nbins + 2)));
        TRY(dalloc(c, &c->spec_e, sizeof(double) * (size_t)(nbins + 1)));
        c->spec_cap = nbins;
    }
    // the edges in T, rounded up: for x in T, x >= e holds exactly when x >= edge
    std::vector<T> et((size_t)nbins + 1);
    for (int b = 0; b <= nbins; ++b) {
        T v = (T)edges[b];
        if ((double)v < edges[b]) v = std::nextafter(v, std::numeric_limits<T>::infinity());
        et[(size_t)b] = v;
    }
    CK(cudaMemcpyAsync(c->spec_e, et.data(), sizeof(T) * et.size(), cudaMemcpyHostToDevice, c->st));
    CK(cudaMemsetAsync(c->spec_w, 0, sizeof(double) * (size_t)(nbins + 2), c->st));
    CK(cudaMemsetAsync(c->spec_c, 0, sizeof(unsigned long long) * (size_t)(nbins + 2), c->st));
    Species& sp = c->sp[s];
    CK(spectrum<T>(arrays<T>(sp, sp.cur), sp.n, variable, (const T*)c->spec_e, nbins, c->spec_w, c->spec_c, c->st));
    const cudaMemcpyKind kind = where == RELSIM_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
    if (weight) CK(cudaMemcpyAsync(weight, c->spec_w, sizeof(double) * (size_t)(nbins + 2), kind, c->st));
    if (count) CK(cudaMemcpyAsync(count, c->spec_c, sizeof(int64_t) * (size_t)(nbins + 2), kind, c->st));
    // the host copy of the edges must outlive the copy above
    CK(cudaStreamSynchronize(c->st));
    return RELSIM_OK;
}

template <typename T>
int modes_impl(relsim_ctx* c, int comp, int nmodes, double* energy, int where)
{
    const int nx = c->g.nx, ny = c->g.ny;
    if (nmodes > c->mode_tw_m) {
        dfree(c->mode_tw);
        c->mode_tw_m = 0;
        TRY(dalloc(c, &c->mode_tw, sizeof(T) * 2 * (size_t)nx * (size_t)nmodes));
        CK(mode_twiddles<T>((T*)c->mode_tw, nx, nmodes, c->st));
        c->mode_tw_m = nmodes;
    }
    const int64_t need = (int64_t)nmodes * (ny + 1);
    if (need > c->mode_rows_cap) {
        dfree(c->mode_rows);
        c->mode_rows_cap = 0;
        TRY(dalloc(c, &c->mode_rows, sizeof(double) * (size_t)need));
        c->mode_rows_cap = need;
    }
    const int bnow = c->state == kSolved ? 1 - c->bcur : c->bcur;
    const T* Bc = (const T*)c->B[bnow] + (int64_t)comp * c->g.ncell;
    double* out = where == RELSIM_DEVICE ? energy : c->mode_rows + (int64_t)nmodes * ny;
    CK(field_modes<T>(Bc, (const T*)c->mode_tw, nx, ny, nmodes, c->g.dV, c->mode_rows, out, c->st));
    if (where == RELSIM_HOST) {
        CK(cudaMemcpyAsync(energy, out, sizeof(double) * (size_t)nmodes, cudaMemcpyDeviceToHost, c->st));
        CK(cudaStreamSynchronize(c->st));
    }
    return RELSIM_OK;
}

int check_push(relsim_ctx* c)
{
    if (*c->hpush & 2)
        return fail(c, RELSIM_ERR_TIMEOUT, "a shared-memory staging wait gave up (deposit or operator)");
    if (*c->hpush)
        return fail(c, RELSIM_ERR_INTERNAL, "particle sort: the moves counted and the new cell starts disagreed");
    return RELSIM_OK;
}

int ledger_impl(relsim_ctx* c, relsim_energy* out)
{
    double h[kLedgerLen];
    TRY(readback(c, c->dled, kLedgerLen, h));
    TRY(check_push(c));
    memset(out, 0, sizeof(*out));
    out->W_E = h[3];
    out->W_B = h[4];
    double K = 0, K0 = 0, dK = 0, work = 0, mis = 0;
    for (int s = 0; s < c->cfg.nspecies; ++s) {
        const double* L = h + kLedgerField + kLedgerSpecies * s;
        out->K_species[s] = L[4];
        K += L[4];
        K0 += L[0];
        dK += L[1];
        work += L[2];
        mis += L[3];
    }
    out->K = K;
    out->total = out->W_E + out->W_B + K;
    if (c->have_step) {
        out->W_E0 = h[kLedgerLen - 2];
        out->W_B0 = h[kLedgerLen - 1];
        out->K0 = K0;
        out->dW_E = h[0];
        out->dW_B = h[1];
        out->dK = dK;
        out->dissipation = h[2];
        out->work_grid = h[5];
        out->work_particles = work;
        out->mismatch = mis;
        out->residual = out->dW_E + out->dW_B + out->dK - out->mismatch + out->dissipation;
        out->gmres_iters = c->last_iters;
        out->gmres_restarts = c->last_restarts;
        out->gmres_relres = c->last_relres;
    }
    out->step = c->step;
    int64_t np = 0;
    for (int s = 0; s < c->cfg.nspecies; ++s) np += c->sp[s].n;
    out->n_particles = np;
    for (int k = 0; k < kLedgerLen; ++k)
        if (!std::isfinite(h[k])) return fail(c, RELSIM_ERR_NONFINITE, "non-finite energy ledger");
    return RELSIM_OK;
}

int validate(const relsim_config* cfg, std::string* why)
{
    char b[256];
    if (cfg->dim != 2) { *why = "only dim = 2 is supported"; return 0; }
    if (cfg->nx < 3 || cfg->ny < 3) { *why = "nx and ny must be >= 3"; return 0; }
    if ((int64_t)cfg->nx * cfg->ny > (int64_t)1 << 28) { *why = "grid too large (nx*ny > 2^28)"; return 0; }
    if (!(cfg->dx > 0) || !(cfg->dy > 0) || !(cfg->dt > 0)) { *why = "dx, dy, dt must be > 0"; return 0; }
    if (!(cfg->theta_implicit > 0) || cfg->theta_implicit > 1) { *why = "theta_implicit must be in (0, 1]"; return 0; }
    if (cfg->precision != 32 && cfg->precision != 64) { *why = "precision must be 32 or 64"; return 0; }
    if (cfg->nspecies < 1 || cfg->nspecies > kMaxSpecies) { *why = "nspecies must be 1..4"; return 0; }
    for (int s = 0; s < cfg->nspecies; ++s)
        if (!(cfg->m[s] > 0) || !std::isfinite(cfg->q[s])) {
            snprintf(b, sizeof(b), "species %d needs m > 0 and a finite q", s);
            *why = b;
            return 0;
        }
    if (cfg->gmres_restart < 0 || cfg->gmres_restart > kMaxRestart) { *why = "gmres_restart must be 0..100"; return 0; }
    if (cfg->gmres_tol < 0 || cfg->gmres_maxit < 0) { *why = "gmres_tol and gmres_maxit must be >= 0"; return 0; }
    return 1;
}

}  // namespace

namespace relsim {
cudaStream_t ctx_stream(const relsim_ctx* c) { return c->st; }
int ctx_last_iters(const relsim_ctx* c) { return c->last_iters; }
int64_t ctx_particles(const relsim_ctx* c)
{
    int64_t n = 0;
    for (int s = 0; s < c->cfg.nspecies; ++s) n += c->sp[s].n;
    return n;
}
}  // namespace relsim

#define DISPATCH(fn, ...) (c->prec == 32 ? fn<float>(__VA_ARGS__) : fn<double>(__VA_ARGS__))

extern "C" {

int relsim_version(void) { return 100; }

const char* relsim_last_error(const relsim_ctx* c) { return c ? c->err.c_str() : "null context"; }

int relsim_init(const relsim_config* cfg, void* cuda_stream, relsim_ctx** out)
{
    if (!out || !cfg) return RELSIM_ERR_INVALID_ARG;
    *out = nullptr;
    std::string why;
    if (!validate(cfg, &why)) return RELSIM_ERR_INVALID_ARG;
    relsim_ctx* c = new (std::nothrow) relsim_ctx();
    if (!c) return RELSIM_ERR_OOM;
    c->cfg = *cfg;
    c->st = (cudaStream_t)cuda_stream;
    c->prec = cfg->precision;
    c->esz = cfg->precision == 32 ? 4 : 8;
    if (c->cfg.gmres_tol == 0.0) c->cfg.gmres_tol = cfg->precision == 32 ? 1e-6 : 1e-10;
    if (c->cfg.gmres_restart == 0) c->cfg.gmres_restart = 30;
    if (c->cfg.gmres_maxit == 0) c->cfg.gmres_maxit = 500;
    c->mrest = c->cfg.gmres_restart;
    c->g.nx = cfg->nx;
    c->g.ny = cfg->ny;
    c->g.ncell = cfg->nx * cfg->ny;
    c->g.dx = cfg->dx;
    c->g.dy = cfg->dy;
    c->g.dt = cfg->dt;
    c->g.theta = cfg->theta_implicit;
    c->g.dV = cfg->dx * cfg->dy;
    // one-cell moves per step: c dt <= min(dx, dy)
    c->fast_sort = cfg->dt <= cfg->dx && cfg->dt <= cfg->dy;
    c->key_bits = 1;
    while (((int64_t)1 << c->key_bits) < (int64_t)c->g.ncell) ++c->key_bits;
    const int64_t nc = c->g.ncell;
    c->nvec = 3 * nc;
    int r = RELSIM_OK;
#define A(x)                                  \
    do {                                      \
        r = (x);                              \
        if (r != RELSIM_OK) goto fail_init;   \
    } while (0)
    A(dalloc(c, &c->E, c->esz * 3 * nc));
    A(dalloc(c, &c->Eth, c->esz * 3 * nc));
    A(dalloc(c, &c->B[0], c->esz * 3 * nc));
    A(dalloc(c, &c->B[1], c->esz * 3 * nc));
    A(dalloc(c, &c->J, c->esz * 3 * nc));
    A(dalloc(c, &c->M, c->esz * kMBlock * nc));
    A(dalloc(c, &c->n9, sizeof(int32_t) * kNDir * nc));
    A(dalloc(c, &c->off9, sizeof(int32_t) * kNDir * nc));
    A(dalloc(c, &c->count_new, sizeof(int32_t) * (nc + 1)));
    c->scan_tmp_n = scan_tmp_ints(nc);
    A(dalloc(c, &c->scan_tmp, sizeof(int32_t) * c->scan_tmp_n));
    A(dalloc(c, &c->V, sizeof(double) * (size_t)(c->mrest + 1) * c->nvec));
    A(dalloc(c, &c->gw, sizeof(double) * c->nvec));
    A(dalloc(c, &c->gw2, sizeof(double) * c->nvec));
    A(dalloc(c, &c->gx, sizeof(double) * c->nvec));
    A(dalloc(c, &c->gb, sizeof(double) * c->nvec));
    A(dalloc(c, &c->dsum, sizeof(double) * 4 * (kMaxRestart + 2)));
    A(dalloc(c, &c->dled, sizeof(double) * kLedgerLen));
    A(dalloc(c, &c->dflag, sizeof(int)));
    A(dalloc(c, &c->dpush, sizeof(int)));
    if (cudaEventCreateWithFlags(&c->gev[0], cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->gev[1], cudaEventDisableTiming) != cudaSuccess) {
        cudaGetLastError();
        r = fail(c, RELSIM_ERR_CUDA, "cudaEventCreate failed");
        goto fail_init;
    }
    if (cudaMallocHost((void**)&c->hpin, sizeof(double) * 4 * (kMaxRestart + 2)) != cudaSuccess ||
        cudaMallocHost((void**)&c->hflag, sizeof(int)) != cudaSuccess ||
        cudaMallocHost((void**)&c->hpush, sizeof(int)) != cudaSuccess) {
        cudaGetLastError();
        r = fail(c, RELSIM_ERR_OOM, "cudaMallocHost failed");
        goto fail_init;
    }
    {
        cudaError_t e = cudaMemsetAsync(c->E, 0, c->esz * 3 * nc, c->st);
        if (e == cudaSuccess) e = cudaMemsetAsync(c->B[0], 0, c->esz * 3 * nc, c->st);
        if (e == cudaSuccess) e = cudaMemsetAsync(c->dled, 0, sizeof(double) * kLedgerLen, c->st);
        if (e == cudaSuccess) e = cudaMemsetAsync(c->dpush, 0, sizeof(int), c->st);
        *c->hpush = 0;
        if (e == cudaSuccess) e = cudaMemsetAsync(c->M, 0, c->esz * kMBlock * nc, c->st);
        if (e == cudaSuccess) e = cudaMemsetAsync(c->J, 0, c->esz * 3 * nc, c->st);
        if (e != cudaSuccess) {
            r = fail(c, RELSIM_ERR_CUDA, "init memset: %s", cudaGetErrorString(e));
            goto fail_init;
        }
        for (int s = 0; s < c->cfg.nspecies; ++s) {
            A(ensure_species(c, s, 0));
            e = cudaMemsetAsync(c->sp[s].start, 0, sizeof(int32_t) * (nc + 1), c->st);
            if (e != cudaSuccess) {
                r = fail(c, RELSIM_ERR_CUDA, "init memset: %s", cudaGetErrorString(e));
                goto fail_init;
            }
        }
    }
#undef A
    c->state = kReady;
    *out = c;
    return RELSIM_OK;
fail_init:
    relsim_destroy(c);
    return r;
}

void relsim_destroy(relsim_ctx* c)
{
    if (!c) return;
    cudaStreamSynchronize(c->st);
    for (int s = 0; s < kMaxSpecies; ++s) {
        Species& sp = c->sp[s];
        for (int b = 0; b < 2; ++b) {
            for (int k = 0; k < 6; ++k) dfree(sp.a[b][k]);
            dfree(sp.id[b]);
        }
        dfree(sp.start);
        dfree(sp.start_alt);
    }
    dfree(c->E); dfree(c->Eth); dfree(c->B[0]); dfree(c->B[1]); dfree(c->J); dfree(c->M);
    dfree(c->n9); dfree(c->off9); dfree(c->count_new); dfree(c->scan_tmp);
    for (int b = 0; b < 2; ++b) {
        dfree(c->rk[b]);
        dfree(c->rv[b]);
    }
    dfree(c->rtmp);
    dfree(c->V); dfree(c->gw); dfree(c->gw2); dfree(c->gx); dfree(c->gb); dfree(c->partial);
    dfree(c->dsum); dfree(c->dled); dfree(c->dflag); dfree(c->dpush); dfree(c->stage);
    dfree(c->spec_w); dfree(c->spec_c); dfree(c->spec_e);
    dfree(c->mode_tw); dfree(c->mode_rows);
    if (c->hpin) cudaFreeHost(c->hpin);
    if (c->hflag) cudaFreeHost(c->hflag);
    if (c->hpush) cudaFreeHost(c->hpush);
    for (cudaEvent_t e : c->prof.pool) cudaEventDestroy(e);
    for (cudaEvent_t e : c->gev)
        if (e) cudaEventDestroy(e);
    delete c;
}

int relsim_load_particles(relsim_ctx* c, int species, int64_t n, const double* x, const double* u,
                          const double* w, int where)
{
    if (!c) return RELSIM_ERR_INVALID_ARG;
    if (species < 0 || species >= c->cfg.nspecies)
        return fail(c, RELSIM_ERR_INVALID_ARG, "species %d out of range", species);
    if (n < 0 || n > 2147483647LL) return fail(c, RELSIM_ERR_INVALID_ARG, "bad particle count %lld", (long long)n);
    if (n > 0 && (!x || !u || !w)) return fail(c, RELSIM_ERR_INVALID_ARG, "null particle array");
    if (where != RELSIM_HOST && where != RELSIM_DEVICE) return fail(c, RELSIM_ERR_INVALID_ARG, "bad where");
    int r = DISPATCH(load_impl, c, species, n, x, u, w, where);
    if (r == RELSIM_OK) {
        c->state = kReady;
        c->have_step = false;
        c->step = 0;
    }
    return r;
}

int relsim_set_fields(relsim_ctx* c, const double* E, const double* B, int where)
{
    if (!c) return RELSIM_ERR_INVALID_ARG;
    if (where != RELSIM_HOST && where != RELSIM_DEVICE) return fail(c, RELSIM_ERR_INVALID_ARG, "bad where");
    if (c->state == kSolved) c->bcur = 1 - c->bcur;   // the solved fields become current
    int r = DISPATCH(set_fields_impl, c, E, B, where);
    if (r == RELSIM_OK) {
        c->state = kReady;
        c->have_step = false;
    }
    return r;
}

int relsim_get_fields(relsim_ctx* c, double* E, double* B, int where)
{
    if (!c) return RELSIM_ERR_INVALID_ARG;
    if (where != RELSIM_HOST && where != RELSIM_DEVICE) return fail(c, RELSIM_ERR_INVALID_ARG, "bad where");
    return DISPATCH(get_fields_impl, c, E, B, where);
}

int relsim_num_particles(relsim_ctx* c, int species, int64_t* n)
{
    if (!c || !n) return RELSIM_ERR_INVALID_ARG;
    if (species < 0 || species >= c->cfg.nspecies)
        return fail(c, RELSIM_ERR_INVALID_ARG, "species %d out of range", species);
    *n = c->sp[species].n;
    return RELSIM_OK;
}

int relsim_get_particles(relsim_ctx* c, int species, double* x, double* u, double* w, int32_t* id,
                         int where)
{
    if (!c) return RELSIM_ERR_INVALID_ARG;
    if (species < 0 || species >= c->cfg.nspecies)
        return fail(c, RELSIM_ERR_INVALID_ARG, "species %d out of range", species);
    if (id && !c->cfg.track_ids) return fail(c, RELSIM_ERR_INVALID_ARG, "ids are not tracked");
    if (where != RELSIM_HOST && where != RELSIM_DEVICE) return fail(c, RELSIM_ERR_INVALID_ARG, "bad where");
    return DISPATCH(get_particles_impl, c, species, x, u, w, id, where);
}

namespace {
__global__ void k_widen(const int32_t* in, int64_t* out, int64_t n)
{
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n;
         k += (int64_t)gridDim.x * blockDim.x)
        out[k] = in[k];
}
}  // namespace

int relsim_get_cell_start(relsim_ctx* c, int species, int64_t* start, int where)
{
    if (!c || !start) return RELSIM_ERR_INVALID_ARG;
    if (species < 0 || species >= c->cfg.nspecies)
        return fail(c, RELSIM_ERR_INVALID_ARG, "species %d out of range", species);
    const int64_t n = c->g.ncell + 1;
    int64_t* dst = start;
    if (where == RELSIM_HOST) {
        TRY(ensure_stage(c, n));
        dst = (int64_t*)c->stage;
    }
    count_launches(1);
    k_widen<<<(unsigned)((n + 255) / 256 < 4096 ? (n + 255) / 256 : 4096), 256, 0, c->st>>>(c->sp[species].start, dst, n);
    CK(cudaGetLastError());
    if (where == RELSIM_HOST) {
        CK(cudaMemcpyAsync(start, dst, sizeof(int64_t) * n, cudaMemcpyDeviceToHost, c->st));
        CK(cudaStreamSynchronize(c->st));
    }
    return RELSIM_OK;
}

int relsim_build_mass_matrix(relsim_ctx* c)
{
    if (!c) return RELSIM_ERR_INVALID_ARG;
    if (c->state != kReady) return fail(c, RELSIM_ERR_BAD_STATE, "build needs a pushed or freshly loaded state");
    int r = DISPATCH(build_impl, c);
    if (r == RELSIM_OK) c->state = kBuilt;
    return r;
}

int relsim_get_mass_matrix(relsim_ctx* c, double* M, double* J, int where)
{
    if (!c) return RELSIM_ERR_INVALID_ARG;
    if (c->state != kBuilt && c->state != kSolved) return fail(c, RELSIM_ERR_BAD_STATE, "no mass matrix built");
    if (where != RELSIM_HOST && where != RELSIM_DEVICE) return fail(c, RELSIM_ERR_INVALID_ARG, "bad where");
    const int64_t nm = (int64_t)c->g.ncell * kMBlock, nj = 3 * (int64_t)c->g.ncell;
    double *dM = M, *dJ = J;
    if (where == RELSIM_HOST) {
        TRY(ensure_stage(c, nm + nj));
        dM = M ? c->stage : nullptr;
        dJ = J ? c->stage + nm : nullptr;
    }
    if (c->prec == 32) CK(mass_to_double<float>((const float*)c->M, (const float*)c->J, dM, dJ, c->g, c->st));
    else CK(mass_to_double<double>((const double*)c->M, (const double*)c->J, dM, dJ, c->g, c->st));
    if (where == RELSIM_HOST) {
        if (M) TRY(copy_out(c, M, dM, nm, where));
        if (J) TRY(copy_out(c, J, dJ, nj, where));
    }
    return RELSIM_OK;
}

int relsim_set_mass_matrix(relsim_ctx* c, const double* M, const double* J, int where)
{
    if (!c || !M || !J) return RELSIM_ERR_INVALID_ARG;
    if (where != RELSIM_HOST && where != RELSIM_DEVICE) return fail(c, RELSIM_ERR_INVALID_ARG, "bad where");
    if (c->state == kEmpty) return fail(c, RELSIM_ERR_BAD_STATE, "context not initialised");
    if (c->state == kSolved) return fail(c, RELSIM_ERR_BAD_STATE, "push the solved step first");
    const int64_t nm = (int64_t)c->g.ncell * kMBlock, nj = 3 * (int64_t)c->g.ncell;
    const double *dM, *dJ;
    if (where == RELSIM_HOST) TRY(ensure_stage(c, nm + nj));
    TRY(stage_in(c, M, nm, where, &dM, 0));
    TRY(stage_in(c, J, nj, where, &dJ, nm));
    CK(cudaMemsetAsync(c->dflag, 0, sizeof(int), c->st));
    if (c->prec == 32) CK(mass_from_double<float>(dM, dJ, (float*)c->M, (float*)c->J, c->g, c->dflag, c->st));
    else CK(mass_from_double<double>(dM, dJ, (double*)c->M, (double*)c->J, c->g, c->dflag, c->st));
    TRY(check_flag(c, "mass matrix"));
    c->state = kBuilt;
    return RELSIM_OK;
}

int relsim_field_solve(relsim_ctx* c, int* iters, double* rel_residual)
{
    if (!c) return RELSIM_ERR_INVALID_ARG;
    if (c->state != kBuilt) return fail(c, RELSIM_ERR_BAD_STATE, "solve needs a built mass matrix");
    int r = DISPATCH(solve_impl, c, iters, rel_residual);
    if (r == RELSIM_OK || r == RELSIM_ERR_NOT_CONVERGED) c->state = kSolved;
    return r;
}

int relsim_get_E_theta(relsim_ctx* c, double* E, int where)
{
    if (!c || !E) return RELSIM_ERR_INVALID_ARG;
    if (c->state != kSolved && !(c->state == kReady && c->have_step))
        return fail(c, RELSIM_ERR_BAD_STATE, "no solve yet");
    const int64_t n = 3 * (int64_t)c->g.ncell;
    double* dst = E;
    if (where == RELSIM_HOST) {
        TRY(ensure_stage(c, n));
        dst = c->stage;
    }
    if (c->prec == 32) CK(fields_to_double<float>((const float*)c->Eth, dst, n, c->st));
    else CK(fields_to_double<double>((const double*)c->Eth, dst, n, c->st));
    return copy_out(c, E, dst, n, where);
}

int relsim_apply_operator(relsim_ctx* c, const double* v, double* out, int where)
{
    if (!c || !v || !out) return RELSIM_ERR_INVALID_ARG;
    if (c->state != kBuilt && c->state != kSolved) return fail(c, RELSIM_ERR_BAD_STATE, "no mass matrix built");
    const int64_t n = c->nvec;
    const double* dv;
    if (where == RELSIM_HOST) TRY(ensure_stage(c, n));
    TRY(stage_in(c, v, n, where, &dv, 0));
    // the GMRES work vector is free outside a solve
    if (c->prec == 32) CK(apply_A<float>((const float*)c->M, dv, c->gw, c->g, c->dpush, c->st));
    else CK(apply_A<double>((const double*)c->M, dv, c->gw, c->g, c->dpush, c->st));
    if (where == RELSIM_DEVICE) return copy_out(c, out, c->gw, n, where);
    CK(cudaMemcpyAsync(c->hpush, c->dpush, sizeof(int), cudaMemcpyDeviceToHost, c->st));
    TRY(copy_out(c, out, c->gw, n, where));
    return check_push(c);
}

int relsim_push(relsim_ctx* c)
{
    if (!c) return RELSIM_ERR_INVALID_ARG;
    if (c->state != kSolved) return fail(c, RELSIM_ERR_BAD_STATE, "push needs a field solve first");
    int r = DISPATCH(push_impl, c);
    if (r == RELSIM_OK) {
        c->state = kReady;
        c->have_step = true;
        ++c->step;
    }
    return r;
}

int relsim_energy_ledger(relsim_ctx* c, relsim_energy* out)
{
    if (!c || !out) return RELSIM_ERR_INVALID_ARG;
    return ledger_impl(c, out);
}

int relsim_profile_enable(relsim_ctx* c, int on)
{
    if (!c) return RELSIM_ERR_INVALID_ARG;
    if (on && c->prof.pool.empty()) {
        c->prof.pool.resize(4096);
        for (auto& e : c->prof.pool) CK(cudaEventCreate(&e));
    }
    if (!on) TRY(prof_flush(c));
    c->prof.on = on != 0;
    return RELSIM_OK;
}

int relsim_profile_read(relsim_ctx* c, relsim_profile* out, int reset)
{
    if (!c || !out) return RELSIM_ERR_INVALID_ARG;
    TRY(prof_flush(c));
    memset(out, 0, sizeof(*out));
    for (int k = 0; k < 16; ++k) {
        out->ms[k] = c->prof.ms[k];
        out->groups[k] = c->prof.groups[k];
        out->kernels[k] = c->prof.kernels[k];
    }
    if (reset) {
        memset(c->prof.ms, 0, sizeof(c->prof.ms));
        memset(c->prof.groups, 0, sizeof(c->prof.groups));
        memset(c->prof.kernels, 0, sizeof(c->prof.kernels));
    }
    return RELSIM_OK;
}

int relsim_energy_spectrum(relsim_ctx* c, int species, int variable, int nbins, const double* edges,
                           double* weight, int64_t* count, int where)
{
    if (!c) return RELSIM_ERR_INVALID_ARG;
    if (species < 0 || species >= c->cfg.nspecies)
        return fail(c, RELSIM_ERR_INVALID_ARG, "species %d out of range", species);
    if (variable != 0 && variable != 1) return fail(c, RELSIM_ERR_INVALID_ARG, "variable must be 0 or 1");
    if (nbins < 1 || nbins > 4096) return fail(c, RELSIM_ERR_INVALID_ARG, "nbins must be 1..4096");
    if (!edges) return fail(c, RELSIM_ERR_INVALID_ARG, "null edges");
    if (where != RELSIM_HOST && where != RELSIM_DEVICE) return fail(c, RELSIM_ERR_INVALID_ARG, "bad where");
    for (int b = 0; b <= nbins; ++b)
        if (!std::isfinite(edges[b]) || (b > 0 && !(edges[b] > edges[b - 1])))
            return fail(c, RELSIM_ERR_INVALID_ARG, "edges must be finite and strictly ascending");
    return DISPATCH(spectrum_impl, c, species, variable, nbins, edges, weight, count, where);
}

int64_t relsim_kernel_launches(void) { return (int64_t)g_launches.load(); }

int relsim_field_modes(relsim_ctx* c, int component, int nmodes, double* energy, int where)
{
    if (!c) return RELSIM_ERR_INVALID_ARG;
    if (component < 0 || component > 2) return fail(c, RELSIM_ERR_INVALID_ARG, "component %d out of range", component);
    if (nmodes < 1 || nmodes > c->g.nx / 2 + 1)
        return fail(c, RELSIM_ERR_INVALID_ARG, "nmodes %d outside [1, nx/2 + 1]", nmodes);
    if (!energy) return fail(c, RELSIM_ERR_INVALID_ARG, "null output");
    if (where != RELSIM_HOST && where != RELSIM_DEVICE) return fail(c, RELSIM_ERR_INVALID_ARG, "bad where");
    return DISPATCH(modes_impl, c, component, nmodes, energy, where);
}

int relsim_step(relsim_ctx* c, relsim_energy* ledger)
{
    if (!c) return RELSIM_ERR_INVALID_ARG;
    int r = relsim_build_mass_matrix(c);
    if (r != RELSIM_OK) return r;
    int first = RELSIM_OK;
    r = relsim_field_solve(c, nullptr, nullptr);
    if (r != RELSIM_OK && r != RELSIM_ERR_NOT_CONVERGED) return r;
    first = r;
    r = relsim_push(c);
    if (r != RELSIM_OK) return r;
    if (ledger) {
        r = relsim_energy_ledger(c, ledger);
        if (r != RELSIM_OK) return r;
    }
    return first;
}

}  // extern "C"
