// capi.cu -- the C ABI declared in include/relsim.h: context, device
// buffers, particle load and export, and the step orchestration (deposit,
// restarted GMRES with an FP64 Krylov basis, field update, push + sort).
#include <atomic>
#include <cmath>
#include <cstdarg>
#include <cstddef>
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
// while a step graph is captured, launches count into the graph's tally
static thread_local long long* t_capture_count = nullptr;
void count_launches(int n)
{
    if (t_capture_count) *t_capture_count += n;
    else g_launches.fetch_add(n, std::memory_order_relaxed);
}
}  // namespace relsim

using namespace relsim;

namespace {

enum State { kEmpty = 0, kReady = 1, kBuilt = 2, kSolved = 3 };

constexpr int kLedgerField = 6;    // dW_E, dW_B, dissipation, W_E1, W_B1, work_grid
constexpr int kLedgerSpecies = 5;  // K0, dK, work, mismatch, K1
constexpr int kLedgerLen = kLedgerField + kLedgerSpecies * kMaxSpecies + 2;   // + W_E0, W_B0

struct Species {
    int64_t n = 0, cap = 0;
    void* a[2][7] = {};   // fx, fy, ux, uy, uz, w (and fz in 3D) of buffer 0 and 1
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

// One step captured as a CUDA graph (deposit, the solve with its loops as
// conditional while nodes, field update, push and re-sort), valid for the
// buffer layout it was captured on.
struct StepGraph {
    cudaGraphExec_t exec = nullptr;
    uint64_t gen = 0;
    int bcur = -1;
    int32_t* start[kMaxSpecies] = {};
    long long k_static = 0, k_cycle = 0, k_iter = 0;   // kernels outside the loops, per cycle, per iteration
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
    void* En = nullptr;        // E^n kept for the push of the predicted-gamma variant
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
    cudaEvent_t gev[2] = {nullptr, nullptr};   // read-back events of the host-driven Arnoldi loop
    GmState* gms = nullptr;    // device-side GMRES control state
    GmState* ghead = nullptr;  // pinned host, two read-back slots (heads only)
    // step graphs (two layouts alternate from step to step)
    StepGraph sg[2];
    uint64_t gen = 1;          // bumped whenever a buffer or the loaded state changes
    bool graph_off = false;    // a capture failed: host-driven steps from then on
    std::string graph_why;     // why
    int dep_blocks = 0;        // launch shapes chosen by relsim_autotune (0: defaults)
    int push_cap = 0;
    int64_t graph_steps = 0;   // steps run as a graph
    bool capturing = false;
    cudaStream_t gst = nullptr;        // graph stream, joined to st by events
    cudaStream_t aux[2] = {nullptr, nullptr};   // capture streams of the loop bodies
    cudaEvent_t gjoin[2] = {nullptr, nullptr};
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
    double* adj = nullptr;   // scratch of the whole-step adjoint
    int64_t adj_cap = 0;     // doubles
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
int ledger_fill(relsim_ctx* c, const double* h, relsim_energy* out);

#define CK(call)                                                                             \
    do {                                                                                     \
        cudaError_t e_ = (call);                                                             \
        if (e_ != cudaSuccess)                                                               \
            return fail(c, RELSIM_ERR_CUDA, "%s: %s", #call, cudaGetErrorString(e_));        \
    } while (0)
// the same, reporting on context cx
#define CK_CTX(cx, call)                                                                     \
    do {                                                                                     \
        cudaError_t e_ = (call);                                                             \
        if (e_ != cudaSuccess)                                                               \
            return fail(cx, RELSIM_ERR_CUDA, "%s: %s", #call, cudaGetErrorString(e_));       \
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
    if (c->capturing) return fail(c, RELSIM_ERR_INTERNAL, "device allocation while a step graph is captured");
    ++c->gen;   // captured step graphs may hold the buffer this replaces
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

int ensure_adj(relsim_ctx* c, int64_t ndoubles)
{
    if (ndoubles <= c->adj_cap) return RELSIM_OK;
    dfree(c->adj);
    c->adj_cap = 0;
    TRY(dalloc(c, &c->adj, sizeof(double) * (size_t)ndoubles));
    c->adj_cap = ndoubles;
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
        for (int k = 0; k < 7; ++k) dfree(sp.a[b][k]);
        dfree(sp.id[b]);
    }
    sp.cap = 0;
    const int narr = c->g.dim == 3 ? 7 : 6;
    for (int b = 0; b < 2; ++b) {
        for (int k = 0; k < narr; ++k) TRY(dalloc(c, &sp.a[b][k], c->esz * (size_t)(n + 8)));
        // 8 elements of slack: bulk copies round a range out to 16 bytes
        if (c->cfg.track_ids) TRY(dalloc(c, &sp.id[b], sizeof(int32_t) * (size_t)(n + 8)));
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
        const int D = c->g.dim;   // x holds D coordinates per particle
        if (where == RELSIM_HOST) TRY(ensure_stage(c, (D + 4) * n));
        TRY(stage_in(c, x, D * n, where, &dx, 0));
        TRY(stage_in(c, u, 3 * n, where, &du, D * n));
        TRY(stage_in(c, w, n, where, &dw, (D + 3) * n));
        TRY(ensure_radix(c, n));
        CK(cudaMemsetAsync(c->dflag, 0, sizeof(int), c->st));
        PROF_BEGIN(RELSIM_PROF_LOAD);
        PArrays<T> tmp = arrays<T>(sp, 1), dst = arrays<T>(sp, 0);
        if (D == 3)
            CK(load_convert3<T>(dx, du, dw, n, c->g, tmp, (T*)sp.a[1][6], c->rk[0], c->rv[0], c->dflag, c->st));
        else
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
            if (D == 3)
                CK(gather_particles3<T>(perm, tmp, (const T*)sp.a[1][6], dst, (T*)sp.a[0][6], n, true, c->st));
            else
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
    const int D = c->g.dim;
    const T* fz = (const T*)sp.a[sp.cur][6];
    if (where == RELSIM_DEVICE) {
        if (D == 3) CK(export_particles3<T>(pa, fz, sp.start, c->g, x, u, w, id, c->st));
        else CK(export_particles<T>(pa, sp.start, c->g, x, u, w, id, c->st));
        return RELSIM_OK;
    }
    TRY(ensure_stage(c, (D + 4) * n + (n + 1) / 2));
    double* dx = x ? c->stage : nullptr;
    double* du = u ? c->stage + D * n : nullptr;
    double* dw = w ? c->stage + (D + 3) * n : nullptr;
    int32_t* did = id ? (int32_t*)(c->stage + (D + 4) * n) : nullptr;
    if (D == 3) CK(export_particles3<T>(pa, fz, sp.start, c->g, dx, du, dw, did, c->st));
    else CK(export_particles<T>(pa, sp.start, c->g, dx, du, dw, did, c->st));
    if (x) CK(cudaMemcpyAsync(x, dx, sizeof(double) * D * n, cudaMemcpyDeviceToHost, c->st));
    if (u) CK(cudaMemcpyAsync(u, du, sizeof(double) * 3 * n, cudaMemcpyDeviceToHost, c->st));
    if (w) CK(cudaMemcpyAsync(w, dw, sizeof(double) * n, cudaMemcpyDeviceToHost, c->st));
    if (id) CK(cudaMemcpyAsync(id, did, sizeof(int32_t) * n, cudaMemcpyDeviceToHost, c->st));
    CK(cudaStreamSynchronize(c->st));
    return RELSIM_OK;
}

// the species in the library's own form (cell start table; per particle the
// offsets within the cell, the momenta and the weight, one array per
// component): plain copies, then one device check of the invariants the
// kernels rely on. A failed check leaves the species empty.
template <typename T>
int load_native_impl(relsim_ctx* c, int s, int64_t n, const int32_t* start, const void* off, const void* u,
                     const void* w, const int32_t* id, int where)
{
    Species& sp = c->sp[s];
    TRY(ensure_species(c, s, n));
    const int D = c->g.dim;
    const int64_t nc1 = (int64_t)c->g.ncell + 1;
    const cudaMemcpyKind kind = where == RELSIM_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
    const size_t bytes = sizeof(T) * (size_t)n;
    const int slot[3] = {0, 1, 6};   // fx, fy, fz
    sp.n = n;
    sp.cur = 0;
    CK(cudaMemcpyAsync(sp.start, start, sizeof(int32_t) * (size_t)nc1, kind, c->st));
    if (n > 0) {
        const T* o = (const T*)off;
        const T* uu = (const T*)u;
        for (int k = 0; k < D; ++k) CK(cudaMemcpyAsync(sp.a[0][slot[k]], o + k * n, bytes, kind, c->st));
        for (int k = 0; k < 3; ++k) CK(cudaMemcpyAsync(sp.a[0][2 + k], uu + k * n, bytes, kind, c->st));
        CK(cudaMemcpyAsync(sp.a[0][5], w, bytes, kind, c->st));
        if (sp.id[0]) {
            if (id) CK(cudaMemcpyAsync(sp.id[0], id, sizeof(int32_t) * (size_t)n, kind, c->st));
            else CK(iota_ids(sp.id[0], n, c->st));
        }
    }
    CK(cudaMemsetAsync(c->dflag, 0, sizeof(int), c->st));
    PArrays<T> pa = arrays<T>(sp, 0);
    if (!id) pa.id = nullptr;   // 0..n-1 need no check
    PROF_BEGIN(RELSIM_PROF_LOAD);
    CK(check_native<T>(sp.start, c->g.ncell, pa, D == 3 ? (const T*)sp.a[0][6] : nullptr, n, c->dflag, c->st));
    PROF_END();
    CK(cudaMemcpyAsync(c->hflag, c->dflag, sizeof(int), cudaMemcpyDeviceToHost, c->st));
    CK(cudaStreamSynchronize(c->st));
    const int f = *c->hflag;
    if (f) {
        sp.n = 0;
        CK(cudaMemsetAsync(sp.start, 0, sizeof(int32_t) * (size_t)nc1, c->st));
        CK(cudaStreamSynchronize(c->st));
        if (f & 1) return fail(c, RELSIM_ERR_NONFINITE, "non-finite momentum or weight");
        if (f & 2) return fail(c, RELSIM_ERR_INVALID_ARG, "an offset outside [0, 1)");
        if (f & 4) return fail(c, RELSIM_ERR_INVALID_ARG, "the cell start table does not run from 0 to n");
        return fail(c, RELSIM_ERR_INVALID_ARG, "an id outside [0, n)");
    }
    // kinetic energy of the loaded species -> ledger slot K1
    const int nb = 152 * 4;
    TRY(ensure_partial(c, nb));
    CK(cudaMemsetAsync(c->dled + kLedgerField + kLedgerSpecies * s, 0, sizeof(double) * kLedgerSpecies,
                       c->st));
    if (n > 0) {
        CK(kinetic_energy<T>(arrays<T>(sp, 0), n, c->cfg.m[s], c->partial, nb, c->st));
        CK(reduce_partials(c->partial, nb, 1, c->dled + kLedgerField + kLedgerSpecies * s + 4, c->st));
    }
    return RELSIM_OK;
}

template <typename T>
int get_native_impl(relsim_ctx* c, int s, int32_t* start, void* off, void* u, void* w, int32_t* id, int where)
{
    Species& sp = c->sp[s];
    const int64_t n = sp.n;
    const int D = c->g.dim;
    const cudaMemcpyKind kind = where == RELSIM_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
    const size_t bytes = sizeof(T) * (size_t)n;
    const int slot[3] = {0, 1, 6};
    const int b = sp.cur;
    if (start) CK(cudaMemcpyAsync(start, sp.start, sizeof(int32_t) * (size_t)(c->g.ncell + 1), kind, c->st));
    if (n > 0) {
        if (off)
            for (int k = 0; k < D; ++k) CK(cudaMemcpyAsync((T*)off + k * n, sp.a[b][slot[k]], bytes, kind, c->st));
        if (u)
            for (int k = 0; k < 3; ++k) CK(cudaMemcpyAsync((T*)u + k * n, sp.a[b][2 + k], bytes, kind, c->st));
        if (w) CK(cudaMemcpyAsync(w, sp.a[b][5], bytes, kind, c->st));
        if (id) CK(cudaMemcpyAsync(id, sp.id[b], sizeof(int32_t) * (size_t)n, kind, c->st));
    }
    CK(cudaStreamSynchronize(c->st));
    return RELSIM_OK;
}

template <typename T>
DepositSpecies<T> deposit_args(relsim_ctx* c);

template <typename T>
int build_impl(relsim_ctx* c)
{
    const int nc = c->g.ncell;
    PROF_BEGIN(RELSIM_PROF_DEPOSIT);
    CK(zero_fill(c->M, c->esz * (size_t)nc * mblock_of(c->g), c->st));
    CK(zero_fill(c->J, c->esz * 3 * (size_t)nc, c->st));
    const DepositSpecies<T> ds = deposit_args<T>(c);
    if (c->g.shape == 2) {
        CK(deposit_q<T>(ds, (const T*)c->B[c->bcur], (T*)c->M, (T*)c->J, c->g, c->st, c->dep_blocks));
    } else if (c->g.dim == 3) {
        FzArrays<T> fz;
        memset(&fz, 0, sizeof(fz));
        for (int s = 0; s < c->cfg.nspecies; ++s) fz.fz[s] = (const T*)c->sp[s].a[c->sp[s].cur][6];
        CK(deposit3<T>(ds, fz, (const T*)c->B[c->bcur], (T*)c->M, (T*)c->J, c->g, c->st, c->dep_blocks));
    } else {
        CK(deposit<T>(ds, (const T*)c->B[c->bcur], c->En ? (const T*)c->E : nullptr, (T*)c->M, (T*)c->J, c->g,
                      c->dpush, c->st, c->dep_blocks));
    }
    PROF_END();
    return RELSIM_OK;
}

// the deposit's view of the current particles
template <typename T>
DepositSpecies<T> deposit_args(relsim_ctx* c)
{
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
    return ds;
}

// Launch shapes timed on the loaded state: the deposit's block count (it
// strides over the row units) and the push's grid cap (warps per unit). Each
// candidate runs once untimed and three times timed with CUDA events; the
// fastest (least of the three) is kept. The trials overwrite only what the
// next step recomputes (M, Jhat, the other particle buffer, the run tables,
// the partial sums); the push trials take E^n as their field (any finite
// field times the same work).
// the push's grid for a cap on its block count (0: the form's default)
int push_blocks_cap(const relsim_ctx* c, int cap)
{
    return c->g.dim == 3 ? push_blocks3(c->g, cap)
                         : (c->g.shape == 2 ? push_blocks_q(c->g, cap) : push_grid_blocks(c->g, c->prec, cap));
}

template <typename T>
int autotune_impl(relsim_ctx* c, relsim_tuning* out)
{
    int dev = 0, nsm = 152;
    CK(cudaGetDevice(&dev));
    CK(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    const int ncand = 4;
    const bool lin2 = c->g.dim == 2 && c->g.shape != 2;   // the 2D kernels with linear shapes
    int dep_c[ncand], push_c[ncand];
    for (int k = 0; k < ncand; ++k) {
        dep_c[k] = lin2 ? (k + 1) * nsm : (2 << k) * nsm;   // 1..4 blocks per SM; 3D, quadratic: 2, 4, 8, 16
        push_c[k] = (4 << k) * nsm;                         // 4, 8, 16, 32 per SM
    }
    TRY(ensure_partial(c, (int64_t)push_blocks_cap(c, push_c[ncand - 1]) * (kLedgerSpecies - 1)));
    relsim_tuning t;
    memset(&t, 0, sizeof(t));
    t.ncand = ncand;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    int r = RELSIM_OK;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        if (e0) cudaEventDestroy(e0);
        return fail(c, RELSIM_ERR_CUDA, "event creation failed");
    }
    const DepositSpecies<T> ds = deposit_args<T>(c);
    int big = 0;   // the push is timed on the species with the most particles
    for (int s = 1; s < c->cfg.nspecies; ++s)
        if (c->sp[s].n > c->sp[big].n) big = s;
    Species& sp = c->sp[big];
    const SpeciesConst sc{c->cfg.q[big], c->cfg.m[big]};
    if (!lin2 && sp.n > 0) TRY(ensure_radix(c, sp.n));
    auto timed = [&](auto launch, float* best) -> int {
        *best = 1e30f;
        for (int rep = 0; rep < 4; ++rep) {
            CK(cudaEventRecord(e0, c->st));
            TRY(launch());
            CK(cudaEventRecord(e1, c->st));
            CK(cudaEventSynchronize(e1));
            float ms = 0.f;
            CK(cudaEventElapsedTime(&ms, e0, e1));
            if (rep > 0 && ms < *best) *best = ms;
        }
        return RELSIM_OK;
    };
    for (int k = 0; k < ncand && r == RELSIM_OK; ++k) {
        t.deposit_blocks[k] = dep_c[k];
        r = timed(
            [&]() -> int {
                const T* B = (const T*)c->B[c->bcur];
                if (c->g.shape == 2) {
                    CK(deposit_q<T>(ds, B, (T*)c->M, (T*)c->J, c->g, c->st, dep_c[k]));
                } else if (c->g.dim == 3) {
                    FzArrays<T> fz;
                    memset(&fz, 0, sizeof(fz));
                    for (int s = 0; s < c->cfg.nspecies; ++s) fz.fz[s] = (const T*)c->sp[s].a[c->sp[s].cur][6];
                    CK(deposit3<T>(ds, fz, B, (T*)c->M, (T*)c->J, c->g, c->st, dep_c[k]));
                } else {
                    CK(deposit<T>(ds, B, c->En ? (const T*)c->E : nullptr, (T*)c->M, (T*)c->J, c->g, c->dpush,
                                  c->st, dep_c[k]));
                }
                return RELSIM_OK;
            },
            &t.deposit_ms[k]);
    }
    for (int k = 0; k < ncand && r == RELSIM_OK && sp.n > 0; ++k) {
        const int nbp = push_blocks_cap(c, push_c[k]);
        t.push_blocks[k] = nbp;
        // the push reads the current buffer and writes the other one (and,
        // in 3D and with quadratic shapes, each particle's new cell and slot)
        r = timed(
            [&]() -> int {
                PArrays<T> src = arrays<T>(sp, sp.cur), dst = arrays<T>(sp, 1 - sp.cur);
                const T* E = (const T*)c->E;
                const T* B = (const T*)c->B[c->bcur];
                if (!lin2)
                    CK(cudaMemsetAsync(c->count_new, 0, sizeof(int32_t) * (size_t)(c->g.ncell + 1), c->st));
                if (c->g.dim == 3)
                    CK(push3<T>(src, (T*)sp.a[sp.cur][6], dst, (T*)sp.a[1 - sp.cur][6], sp.start, c->rk[0], c->rv[0],
                                c->count_new, E, B, c->g, sc, c->partial, nbp, c->st));
                else if (c->g.shape == 2)
                    CK(push_q<T>(src, dst, sp.start, c->rk[0], c->rv[0], c->count_new, E, B, c->g, sc, c->partial,
                                 nbp, c->st));
                else
                    CK(push_sort<T>(src, dst, sp.start, c->n9, c->off9, E, B, c->En ? E : nullptr, c->g, sc,
                                    c->partial, nbp, c->dpush, c->st));
                return RELSIM_OK;
            },
            &t.push_ms[k]);
    }
    // the operator's tile height (a compile-time shape with two instances):
    // an Arnoldi-mode application with 8 dot products on the deposited M
    const int alt = c->prec == 32 ? 4 : 2;
    const int rows_c[2] = {0, alt};
    t.op_nrows = lin2 ? 2 : 0;   // the 3D and quadratic operators have one tile shape
    if (r == RELSIM_OK && lin2) {
        const int jdots = 8;
        int64_t most = 0;
        for (int k = 0; k < 2; ++k) {
            GridP gk = c->g;
            gk.op_y = rows_c[k];
            const int64_t nb = op_blocks(gk, c->prec);
            most = nb > most ? nb : most;
        }
        r = ensure_partial(c, most * (jdots + 2));
        if (r == RELSIM_OK && cudaMemsetAsync(c->V, 0, sizeof(double) * (size_t)(jdots + 1) * c->nvec, c->st) != cudaSuccess)
            r = fail(c, RELSIM_ERR_CUDA, "cudaMemsetAsync failed");
        if (r == RELSIM_OK && cudaMemsetAsync(c->gw, 0, sizeof(double) * (size_t)c->nvec, c->st) != cudaSuccess)
            r = fail(c, RELSIM_ERR_CUDA, "cudaMemsetAsync failed");
        for (int k = 0; k < 2 && r == RELSIM_OK; ++k) {
            GridP gk = c->g;
            gk.op_y = rows_c[k];
            t.op_rows[k] = rows_c[k] > 0 ? rows_c[k] : (c->prec == 32 ? 8 : 4);
            r = timed(
                [&]() -> int {
                    CK(op_arnoldi<T>((const T*)c->M, c->gw, 1.0, nullptr, c->gw2, c->V, c->nvec, jdots, gk, c->partial,
                                     c->dpush, c->st));
                    return RELSIM_OK;
                },
                &t.op_ms[k]);
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (r != RELSIM_OK) return r;
    t.op_choice = lin2 && t.op_ms[1] < t.op_ms[0] ? 1 : 0;
    c->g.op_y = rows_c[t.op_choice];
    int bd = 0, bp = 0;
    for (int k = 1; k < ncand; ++k) {
        if (t.deposit_ms[k] < t.deposit_ms[bd]) bd = k;
        if (t.push_ms[k] < t.push_ms[bp]) bp = k;
    }
    t.deposit_choice = bd;
    t.push_choice = bp;
    c->dep_blocks = dep_c[bd];
    c->push_cap = push_c[bp];
    ++c->gen;   // step graphs hold the old launch shapes
    TRY(check_push(c));
    if (out) *out = t;
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

// Restarted GMRES on A = I + B, controlled on the device (gmres.cu). The
// Arnoldi process runs on B (the same Krylov space: A V_k = V_k + B V_k, so
// the Hessenberg matrix of A is that of B plus the identity). Working on B
// avoids the cancellation of orthogonalising A v ~ v against v, and keeps the
// identity exact in FP64. The pieces below enqueue on a given stream; each
// takes the graph condition it sets (0 when driven from the host).
struct GmSetup {
    int64_t n, ldv;
    int m, nb, nbo;
    GmPtrs p;
    GmParams q;
};

GmSetup gm_setup(relsim_ctx* c)
{
    GmSetup s;
    s.n = c->nvec;
    s.ldv = s.n;
    s.m = c->mrest;
    s.nb = gm_blocks(s.n);
    s.nbo = op_blocks(c->g, c->prec);
    s.p.r = c->gw;
    s.p.w0 = c->gw2;
    s.p.V = c->V;
    s.p.ds0 = c->dsum;
    s.p.ds1 = c->dsum + 3 * (kMaxRestart + 2);
    s.p.ldv = s.ldv;
    s.q.tol = c->cfg.gmres_tol;
    s.q.m = s.m;
    s.q.maxit = c->cfg.gmres_maxit;
    return s;
}

// b, x = E^n, |b|, r = b - A x, |r|, start of the first cycle
template <typename T>
int solve_prologue(relsim_ctx* c, const GmSetup& S, cudaStream_t s, GmCond outer)
{
    PROF_BEGIN(RELSIM_PROF_RHS);
    CK(rhs<T>((const T*)c->E, (const T*)c->B[c->bcur], (const T*)c->J, c->gb, c->g, s));
    CK(fields_to_vec<T>((const T*)c->E, c->gx, S.n, c->g.df, s));
    PROF_END();
    PROF_BEGIN(RELSIM_PROF_GMRES_ORTHO);
    CK(gm_dots(c->V, S.ldv, 0, c->gb, S.n, c->partial, S.nb, s, c->g.df));
    CK(reduce_partials(c->partial, S.nb, 1, c->dsum, s));
    CK(gm_begin(c->gms, c->dsum, s));
    CK(gm_zero_x(c->gms, c->gx, S.n, s));
    PROF_END();
    PROF_BEGIN(RELSIM_PROF_GMRES_APPLY);
    CK(op_residual<T>((const T*)c->M, c->gx, c->gb, S.p.r, c->g, c->partial, c->dpush, s));
    CK(reduce_partials(c->partial, S.nbo, 1, c->dsum, s));
    CK(gm_cycle(c->gms, c->dsum, S.p, S.q, outer, s));
    PROF_END();
    return RELSIM_OK;
}

// one Arnoldi iteration with the arguments the device left in gms->dyn
template <typename T>
int arnoldi_body(relsim_ctx* c, const GmSetup& S, cudaStream_t s, GmCond inner, bool tr = false)
{
    PROF_BEGIN(RELSIM_PROF_GMRES_APPLY);
    CK(op_arnoldi_dyn<T>((const T*)c->M, &c->gms->dyn, c->V, S.ldv, c->g, c->partial, c->dpush, s, tr));
    PROF_END();
    PROF_BEGIN(RELSIM_PROF_GMRES_ORTHO);
    CK(reduce_partials_dyn(c->partial, S.nbo, &c->gms->dyn, S.m + 2, s));
    CK(gm_update_scale_dyn(&c->gms->dyn, c->V, S.ldv, S.n, s, c->g.df));
    CK(gm_tail(c->gms, S.p, S.q, inner, s));
    PROF_END();
    return RELSIM_OK;
}

// x += V y of the finished cycle, the true residual, next cycle or stop
template <typename T>
int cycle_end(relsim_ctx* c, const GmSetup& S, cudaStream_t s, GmCond outer, bool tr = false)
{
    PROF_BEGIN(RELSIM_PROF_GMRES_ORTHO);
    CK(gm_finish_cycle(c->gms, c->gx, c->V, S.ldv, S.n, S.m, s, c->g.df));
    PROF_END();
    PROF_BEGIN(RELSIM_PROF_GMRES_APPLY);
    CK(op_residual<T>((const T*)c->M, c->gx, c->gb, S.p.r, c->g, c->partial, c->dpush, s, tr));
    CK(reduce_partials(c->partial, S.nbo, 1, c->dsum, s));
    CK(gm_cycle(c->gms, c->dsum, S.p, S.q, outer, s));
    PROF_END();
    return RELSIM_OK;
}

// E^{n+1}, B^{n+1} and the field side of the ledger
template <typename T>
int solve_epilogue(relsim_ctx* c, cudaStream_t s)
{
    CK(cudaMemcpyAsync(c->dled + kLedgerLen - 2, c->dled + 3, 2 * sizeof(double), cudaMemcpyDeviceToDevice, s));
    // the predicted-gamma push needs E^n after E^{n+1} has replaced it
    if (c->En) CK(cudaMemcpyAsync(c->En, c->E, c->esz * 3 * (size_t)c->g.ncell, cudaMemcpyDeviceToDevice, s));
    const int nbf = field_grid_blocks(c->g);
    PROF_BEGIN(RELSIM_PROF_FIELD_UPDATE);
    CK(field_update<T>(c->gx, (const T*)c->M, (const T*)c->J, (T*)c->Eth, (T*)c->E, (const T*)c->B[c->bcur],
                       (T*)c->B[1 - c->bcur], c->g, c->partial, nbf, s));
    CK(reduce_partials(c->partial, nbf, 6, c->dled, s));
    PROF_END();
    return RELSIM_OK;
}

// buffers the solve needs, sized before anything is enqueued (a graph
// capture must not allocate)
int solve_reserve(relsim_ctx* c, const GmSetup& S)
{
    const int nbf = field_grid_blocks(c->g);
    int64_t need = (int64_t)(S.nb > S.nbo ? S.nb : S.nbo) * (S.m + 2);
    if ((int64_t)nbf * 6 > need) need = (int64_t)nbf * 6;
    return ensure_partial(c, need);
}

// the solve's outcome from the device state read back after it
int solve_outcome(relsim_ctx* c, const GmState* h, int* iters_out, double* relres_out)
{
    c->last_iters = h->total;
    c->last_restarts = h->restarts;
    c->last_relres = h->relres;
    if (iters_out) *iters_out = h->total;
    if (relres_out) *relres_out = h->relres;
    if (h->status == kGmNonfinite) return fail(c, RELSIM_ERR_NONFINITE, "non-finite value in the field solve");
    if (h->status == kGmNotConverged)
        return fail(c, RELSIM_ERR_NOT_CONVERGED, "GMRES reached %d iterations at relative residual %.3e", h->total,
                    h->relres);
    return RELSIM_OK;
}

constexpr size_t kGmHead = offsetof(GmState, cs);

// the control state's head into host slot k (and the kernels' error flags)
int head_async(relsim_ctx* c, int k)
{
    CK(cudaMemcpyAsync(c->ghead + k, c->gms, kGmHead, cudaMemcpyDeviceToHost, c->st));
    CK(cudaMemcpyAsync(c->hpush, c->dpush, sizeof(int), cudaMemcpyDeviceToHost, c->st));
    return RELSIM_OK;
}

// The solve driven from the host: the same kernels as the graph, with the
// host reading the device's decisions. Iteration j+1 is enqueued before
// iteration j's decision is read (it returns at once if j was the last).
// the restart and Arnoldi loops from the host, after a prologue enqueued
// the first cycle start (tr: the operator is A^T)
template <typename T>
int gm_drive(relsim_ctx* c, const GmSetup& S, bool tr)
{
    TRY(head_async(c, 0));
    CK(cudaStreamSynchronize(c->st));
    TRY(check_push(c));
    while (c->ghead[0].run) {
        int cur = 0;
        TRY(arnoldi_body<T>(c, S, c->st, GmCond{0, 0}, tr));
        TRY(head_async(c, cur));
        CK(cudaEventRecord(c->gev[cur], c->st));
        for (int guard = 0; guard <= S.m; ++guard) {
            TRY(arnoldi_body<T>(c, S, c->st, GmCond{0, 0}, tr));
            TRY(head_async(c, 1 - cur));
            CK(cudaEventRecord(c->gev[1 - cur], c->st));
            CK(cudaEventSynchronize(c->gev[cur]));
            TRY(check_push(c));
            if (!c->ghead[cur].inner) break;
            cur = 1 - cur;
        }
        TRY(cycle_end<T>(c, S, c->st, GmCond{0, 0}, tr));
        TRY(head_async(c, 0));
        CK(cudaStreamSynchronize(c->st));
        TRY(check_push(c));
    }
    return RELSIM_OK;
}

template <typename T>
int solve_impl(relsim_ctx* c, int* iters_out, double* relres_out)
{
    const GmSetup S = gm_setup(c);
    TRY(solve_reserve(c, S));
    TRY(solve_prologue<T>(c, S, c->st, GmCond{0, 0}));
    TRY(gm_drive<T>(c, S, false));
    const GmState h = c->ghead[0];
    if (h.status == kGmNonfinite) return solve_outcome(c, &h, iters_out, relres_out);
    TRY(solve_epilogue<T>(c, c->st));
    return solve_outcome(c, &h, iters_out, relres_out);
}

// the push's grid (its ledger partials are sized by it)
int push_blocks_for(const relsim_ctx* c) { return push_blocks_cap(c, c->push_cap); }

// steps that can run as a captured graph: the one-cell-move sort of the 2D
// linear form, and the counting-sort paths of the 3D form and the quadratic
// shapes (no host decision inside a step); the radix path of long moves is
// left host-driven
bool graph_path(const relsim_ctx* c) { return c->fast_sort || c->g.dim == 3 || c->g.shape == 2; }

// the host side of a push: the new cell starts and the new B become current
void push_commit(relsim_ctx* c)
{
    if (c->fast_sort)
        for (int s = 0; s < c->cfg.nspecies; ++s) {
            Species& sp = c->sp[s];
            if (sp.n == 0) continue;
            int32_t* t = sp.start;
            sp.start = sp.start_alt;
            sp.start_alt = t;
        }
    c->bcur = 1 - c->bcur;
}

// enqueue the push and the re-sort of every species (push_commit follows)
template <typename T>
int push_enqueue(relsim_ctx* c)
{
    const int nbp = push_blocks_for(c);
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
        if (c->g.dim == 3) {
            // 3D: push with each particle's new cell and its slot there
            // (warp-aggregated counts), then an unstable counting sort: the
            // cells' starts by a scan, each particle placed at start + slot.
            // The order within a cell is not kept (nothing in the 3D form
            // depends on it beyond rounding; ids follow the particles)
            TRY(ensure_radix(c, sp.n));
            T* sfz = (T*)sp.a[sp.cur][6];
            T* dfz = (T*)sp.a[1 - sp.cur][6];
            PROF_BEGIN(RELSIM_PROF_GENERAL_SORT);
            CK(cudaMemcpyAsync(led, led + 4, sizeof(double), cudaMemcpyDeviceToDevice, c->st));
            CK(cudaMemsetAsync(c->count_new, 0, sizeof(int32_t) * (size_t)(c->g.ncell + 1), c->st));
            CK(push3<T>(src, sfz, dst, dfz, sp.start, c->rk[0], c->rv[0], c->count_new, Eth, B, c->g, sc, c->partial,
                        nbp, c->st));
            CK(reduce_partials(c->partial, nbp, kLedgerSpecies - 1, led + 1, c->st));
            CK(scan_exclusive_i32(c->count_new, sp.start, c->g.ncell, sp.start + c->g.ncell, c->scan_tmp, c->st));
            CK(place3<T>(dst, dfz, src, sfz, c->rk[0], c->rv[0], sp.start, sp.n, c->st));
            PROF_END();
        } else if (c->g.shape == 2) {
            // quadratic shapes: the push with each particle's new cell and
            // slot, the unstable counting sort as in 3D
            TRY(ensure_radix(c, sp.n));
            PROF_BEGIN(RELSIM_PROF_GENERAL_SORT);
            CK(cudaMemcpyAsync(led, led + 4, sizeof(double), cudaMemcpyDeviceToDevice, c->st));
            CK(cudaMemsetAsync(c->count_new, 0, sizeof(int32_t) * (size_t)(c->g.ncell + 1), c->st));
            CK(push_q<T>(src, dst, sp.start, c->rk[0], c->rv[0], c->count_new, Eth, B, c->g, sc, c->partial, nbp,
                         c->st));
            CK(reduce_partials(c->partial, nbp, kLedgerSpecies - 1, led + 1, c->st));
            CK(scan_exclusive_i32(c->count_new, sp.start, c->g.ncell, sp.start + c->g.ncell, c->scan_tmp, c->st));
            CK(place3<T>(dst, nullptr, src, nullptr, c->rk[0], c->rv[0], sp.start, sp.n, c->st));
            PROF_END();
        } else if (c->fast_sort) {
            // push, each old cell written back grouped by move direction
            // into the other buffer; then the stable new-cell order back into
            // the current buffer
            PROF_BEGIN(RELSIM_PROF_PUSH);
            // K0 of this step is the kinetic energy the last push (or load) left
            CK(cudaMemcpyAsync(led, led + 4, sizeof(double), cudaMemcpyDeviceToDevice, c->st));
            CK(push_sort<T>(src, dst, sp.start, c->n9, c->off9, Eth, B, (const T*)c->En, c->g, sc, c->partial,
                            nbp, c->dpush, c->st));
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
        } else {
            // general path: push in place order with keys, radix sort, gather
            TRY(ensure_radix(c, sp.n));
            PROF_BEGIN(RELSIM_PROF_GENERAL_SORT);
            CK(cudaMemcpyAsync(led, led + 4, sizeof(double), cudaMemcpyDeviceToDevice, c->st));
            CK(push_general<T>(src, dst, sp.start, c->rk[0], Eth, B, (const T*)c->En, c->g, sc, c->partial, nbp,
                               c->st));
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
    // read back lazily: checked after the next synchronising call
    CK(cudaMemcpyAsync(c->hpush, c->dpush, sizeof(int), cudaMemcpyDeviceToHost, c->st));
    return RELSIM_OK;
}

template <typename T>
int push_impl(relsim_ctx* c)
{
    TRY(push_enqueue<T>(c));
    push_commit(c);
    return RELSIM_OK;
}


// ---------------------------------------------------------------------------
// A whole step as one CUDA graph. The solve's restart loop and Arnoldi loop
// become conditional while nodes whose conditions the control kernels set,
// so a step needs no host decision: one graph launch, then one read-back.

// the graph being captured on stream s
int capture_graph(relsim_ctx* c, cudaStream_t s, cudaGraph_t* g)
{
    cudaStreamCaptureStatus cs;
    CK(cudaStreamGetCaptureInfo(s, &cs, nullptr, g, nullptr, nullptr, nullptr));
    if (cs != cudaStreamCaptureStatusActive) return fail(c, RELSIM_ERR_INTERNAL, "stream not capturing");
    return RELSIM_OK;
}

// append a while node with condition h to the capture on stream s; the
// capture continues after it; *body receives the loop body to capture into
int add_while(relsim_ctx* c, cudaStream_t s, cudaGraphConditionalHandle h, cudaGraph_t* body)
{
    cudaStreamCaptureStatus cs;
    cudaGraph_t cg = nullptr;
    const cudaGraphNode_t* deps = nullptr;
    const cudaGraphEdgeData* ed = nullptr;
    size_t nd = 0;
    CK(cudaStreamGetCaptureInfo(s, &cs, nullptr, &cg, &deps, &ed, &nd));
    // the parameter struct holds a union: zeroed raw storage stands in for
    // its (deleted) default constructor
    alignas(cudaGraphNodeParams) unsigned char raw[sizeof(cudaGraphNodeParams)];
    memset(raw, 0, sizeof(raw));
    cudaGraphNodeParams& np = *reinterpret_cast<cudaGraphNodeParams*>(raw);
    np.type = cudaGraphNodeTypeConditional;
    np.conditional.handle = h;
    np.conditional.type = cudaGraphCondTypeWhile;
    np.conditional.size = 1;
    cudaGraphNode_t node;
    CK(cudaGraphAddNode(&node, cg, deps, ed, nd, &np));
    *body = np.conditional.phGraph_out[0];
    CK(cudaStreamUpdateCaptureDependencies(s, &node, nullptr, 1, cudaStreamSetCaptureDependencies));
    return RELSIM_OK;
}

// capture the enqueue function f into the body graph on stream s
template <class F>
int capture_into(relsim_ctx* c, cudaStream_t s, cudaGraph_t body, long long* tally, F f)
{
    long long* saved = t_capture_count;
    t_capture_count = tally;
    CK(cudaStreamBeginCaptureToGraph(s, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
    int r = f();
    cudaGraph_t out = nullptr;
    const cudaError_t e = cudaStreamEndCapture(s, &out);
    t_capture_count = saved;
    if (r == RELSIM_OK && e != cudaSuccess) r = fail(c, RELSIM_ERR_CUDA, "body capture: %s", cudaGetErrorString(e));
    return r;
}

// The solve: prologue, then while (cycle) { arm; while (iteration) { Arnoldi
// step }; finish the cycle }, then the field update. Each condition handle
// is created on the graph that holds its while node, before the kernels that
// set it are captured.
template <typename T>
int capture_solve(relsim_ctx* c, const GmSetup& S, StepGraph& G)
{
    cudaGraph_t top = nullptr;
    TRY(capture_graph(c, c->st, &top));
    cudaGraphConditionalHandle ho;
    CK(cudaGraphConditionalHandleCreate(&ho, top, 0, cudaGraphCondAssignDefault));
    TRY(solve_prologue<T>(c, S, c->st, GmCond{(unsigned long long)ho, 1}));
    cudaGraph_t outer = nullptr;
    TRY(add_while(c, c->st, ho, &outer));
    cudaGraphConditionalHandle hi;
    CK(cudaGraphConditionalHandleCreate(&hi, outer, 0, cudaGraphCondAssignDefault));
    TRY(capture_into(c, c->aux[0], outer, &G.k_cycle, [&]() -> int {
        CK(gm_arm(c->gms, GmCond{(unsigned long long)hi, 1}, c->aux[0]));
        cudaGraph_t inner = nullptr;
        TRY(add_while(c, c->aux[0], hi, &inner));
        TRY(capture_into(c, c->aux[1], inner, &G.k_iter,
                         [&]() -> int { return arnoldi_body<T>(c, S, c->aux[1], GmCond{(unsigned long long)hi, 1}); }));
        return cycle_end<T>(c, S, c->aux[0], GmCond{(unsigned long long)ho, 1});
    }));
    return solve_epilogue<T>(c, c->st);
}

// capture the step on the graph stream for the current buffer layout
template <typename T>
int capture_step(relsim_ctx* c, StepGraph& G)
{
    const GmSetup S = gm_setup(c);
    TRY(solve_reserve(c, S));
    TRY(ensure_partial(c, (int64_t)push_blocks_for(c) * (kLedgerSpecies - 1)));
    if (G.exec) {
        cudaGraphExecDestroy(G.exec);
        G.exec = nullptr;
    }
    G.k_static = G.k_cycle = G.k_iter = 0;
    cudaStream_t user = c->st;
    c->st = c->gst;
    c->capturing = true;
    t_capture_count = &G.k_static;
    int r = RELSIM_OK;
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamBeginCapture(c->st, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) {
        r = fail(c, RELSIM_ERR_CUDA, "cudaStreamBeginCapture: %s", cudaGetErrorString(e));
    } else {
        r = build_impl<T>(c);
        if (r == RELSIM_OK) r = capture_solve<T>(c, S, G);
        if (r == RELSIM_OK) r = push_enqueue<T>(c);
        e = cudaStreamEndCapture(c->st, &graph);
        if (r == RELSIM_OK && e != cudaSuccess) r = fail(c, RELSIM_ERR_CUDA, "step capture: %s", cudaGetErrorString(e));
    }
    t_capture_count = nullptr;
    c->capturing = false;
    c->st = user;
    if (r == RELSIM_OK) {
        e = cudaGraphInstantiate(&G.exec, graph, 0);
        if (e != cudaSuccess) {
            G.exec = nullptr;
            r = fail(c, RELSIM_ERR_CUDA, "cudaGraphInstantiate: %s", cudaGetErrorString(e));
        }
    }
    if (graph) cudaGraphDestroy(graph);
    (void)cudaGetLastError();
    if (r != RELSIM_OK) return r;
    G.gen = c->gen;
    G.bcur = c->bcur;
    for (int s = 0; s < kMaxSpecies; ++s) G.start[s] = c->sp[s].start;
    return RELSIM_OK;
}

bool graph_matches(const relsim_ctx* c, const StepGraph& G)
{
    if (!G.exec || G.gen != c->gen || G.bcur != c->bcur) return false;
    for (int s = 0; s < kMaxSpecies; ++s)
        if (G.start[s] != c->sp[s].start) return false;
    return true;
}

// one step through the graph of the current layout (captured on first use);
// returns 1 when the graph path is unavailable (the caller steps eagerly)
template <typename T>
int step_graph(relsim_ctx* c, relsim_energy* ledger, int* status)
{
    StepGraph* G = nullptr;
    for (StepGraph& g : c->sg)
        if (graph_matches(c, g)) G = &g;
    if (!G) {
        // replace the slot not matching the other parity's layout
        G = &c->sg[c->sg[0].exec && c->sg[0].gen == c->gen && c->sg[0].bcur != c->bcur ? 1 : 0];
        if (capture_step<T>(c, *G) != RELSIM_OK) {
            c->graph_off = true;
            c->graph_why = c->err;
            c->err.clear();
            return 1;
        }
    }
    CK(cudaEventRecord(c->gjoin[0], c->st));
    CK(cudaStreamWaitEvent(c->gst, c->gjoin[0], 0));
    CK(cudaGraphLaunch(G->exec, c->gst));
    CK(cudaEventRecord(c->gjoin[1], c->gst));
    CK(cudaStreamWaitEvent(c->st, c->gjoin[1], 0));
    push_commit(c);
    c->state = kReady;
    c->have_step = true;
    ++c->step;
    ++c->graph_steps;
    TRY(head_async(c, 0));
    double* h = c->hpin;
    if (ledger) CK(cudaMemcpyAsync(h, c->dled, sizeof(double) * kLedgerLen, cudaMemcpyDeviceToHost, c->st));
    CK(cudaStreamSynchronize(c->st));
    const GmState hd = c->ghead[0];
    count_launches((int)(G->k_static + G->k_cycle * hd.restarts + G->k_iter * hd.total));
    TRY(check_push(c));
    *status = solve_outcome(c, &hd, nullptr, nullptr);
    if (*status != RELSIM_OK && *status != RELSIM_ERR_NOT_CONVERGED) return RELSIM_OK;
    if (ledger) {
        double hl[kLedgerLen];
        memcpy(hl, h, sizeof(hl));
        const int r = ledger_fill(c, hl, ledger);
        if (r != RELSIM_OK) *status = r;
    }
    return RELSIM_OK;
}

// The adjoint of the field part of the solved step (particles held fixed):
// A^T lambda = gE1/theta - dt curl_c^T gB1 by the same device-controlled
// GMRES on the transposed operator, then the gradients of E^n, B^n, Jhat and
// the stored mass-matrix blocks (see fields.cu).
template <typename T>
int adjoint_impl(relsim_ctx* c, const double* gE1, const double* gB1, const double* gEt, double* gE0,
                 double* gB0, double* gJ, double* gM, int* iters, double* relres, int where)
{
    const int64_t n = c->nvec, nm = (int64_t)c->g.ncell * kMBlock;
    if (where == RELSIM_HOST) TRY(ensure_stage(c, 6 * n + nm));
    const double *d1 = nullptr, *d2 = nullptr, *d3 = nullptr;
    TRY(stage_in(c, gE1, n, where, &d1, 0));
    TRY(stage_in(c, gB1, n, where, &d2, n));
    if (gEt) TRY(stage_in(c, gEt, n, where, &d3, 5 * n + nm));
    const GmSetup S = gm_setup(c);
    TRY(solve_reserve(c, S));
    CK(adjoint_pre(d1, d2, d3, c->gb, c->g, c->st));
    CK(gm_dots(c->V, S.ldv, 0, c->gb, S.n, c->partial, S.nb, c->st, c->g.df));
    CK(reduce_partials(c->partial, S.nb, 1, c->dsum, c->st));
    CK(gm_begin(c->gms, c->dsum, c->st));
    CK(cudaMemsetAsync(c->gx, 0, sizeof(double) * (size_t)n, c->st));
    CK(op_residual<T>((const T*)c->M, c->gx, c->gb, S.p.r, c->g, c->partial, c->dpush, c->st, true));
    CK(reduce_partials(c->partial, S.nbo, 1, c->dsum, c->st));
    CK(gm_cycle(c->gms, c->dsum, S.p, S.q, GmCond{0, 0}, c->st));
    TRY(gm_drive<T>(c, S, true));
    const GmState h = c->ghead[0];
    if (iters) *iters = h.total;
    if (relres) *relres = h.relres;
    if (h.status == kGmNonfinite) return fail(c, RELSIM_ERR_NONFINITE, "non-finite value in the adjoint solve");
    const bool host = where == RELSIM_HOST;
    double* oE = gE0 ? (host ? c->stage + 2 * n : gE0) : nullptr;
    double* oB = gB0 ? (host ? c->stage + 3 * n : gB0) : nullptr;
    double* oJ = gJ ? (host ? c->stage + 4 * n : gJ) : nullptr;
    double* oM = gM ? (host ? c->stage + 5 * n : gM) : nullptr;
    CK(adjoint_post(d1, d2, c->gx, oE, oB, oJ, c->g, c->st));
    if (oM) CK(adjoint_mass<T>(c->gx, (const T*)c->Eth, oM, c->g, c->st));
    if (host) {
        if (gE0) CK(cudaMemcpyAsync(gE0, oE, sizeof(double) * (size_t)n, cudaMemcpyDeviceToHost, c->st));
        if (gB0) CK(cudaMemcpyAsync(gB0, oB, sizeof(double) * (size_t)n, cudaMemcpyDeviceToHost, c->st));
        if (gJ) CK(cudaMemcpyAsync(gJ, oJ, sizeof(double) * (size_t)n, cudaMemcpyDeviceToHost, c->st));
        if (gM) CK(cudaMemcpyAsync(gM, oM, sizeof(double) * (size_t)nm, cudaMemcpyDeviceToHost, c->st));
    }
    CK(cudaStreamSynchronize(c->st));
    if (h.status == kGmNotConverged)
        return fail(c, RELSIM_ERR_NOT_CONVERGED, "adjoint GMRES reached %d iterations at relative residual %.3e",
                    h.total, h.relres);
    return RELSIM_OK;
}

// The adjoint of one species' deposit (k_deposit_adjoint); gB is
// overwritten with this species' contribution.
template <typename T>
int deposit_adjoint_impl(relsim_ctx* c, int s, const double* gJ, const double* gM, double* gu0, double* gx0,
                         double* gB, double* gw0, int where)
{
    Species& sp = c->sp[s];
    const int64_t n = sp.n, nf = 3 * (int64_t)c->g.ncell, nm = (int64_t)c->g.ncell * kMBlock;
    const bool host = where == RELSIM_HOST;
    if (host) TRY(ensure_stage(c, nf + nm + 5 * n + nf + n));
    const double *dJ = nullptr, *dM = nullptr;
    TRY(stage_in(c, gJ, nf, where, &dJ, 0));
    TRY(stage_in(c, gM, nm, where, &dM, nf));
    double* ou = host ? c->stage + nf + nm : gu0;
    double* ox = host ? c->stage + nf + nm + 3 * n : gx0;
    double* oB = host ? c->stage + nf + nm + 5 * n : gB;
    double* ow = gw0 ? (host ? c->stage + nf + nm + 5 * n + nf : gw0) : nullptr;
    CK(cudaMemsetAsync(oB, 0, sizeof(double) * (size_t)nf, c->st));
    if (n > 0)
        CK(deposit_adjoint<T>(arrays<T>(sp, sp.cur), sp.start, dJ, dM, ou, ox, ow, oB, (const T*)c->B[c->bcur], c->g,
                              SpeciesConst{c->cfg.q[s], c->cfg.m[s]}, c->st));
    if (host) {
        CK(cudaMemcpyAsync(gu0, ou, sizeof(double) * (size_t)(3 * n), cudaMemcpyDeviceToHost, c->st));
        CK(cudaMemcpyAsync(gx0, ox, sizeof(double) * (size_t)(2 * n), cudaMemcpyDeviceToHost, c->st));
        if (gw0) CK(cudaMemcpyAsync(gw0, ow, sizeof(double) * (size_t)n, cudaMemcpyDeviceToHost, c->st));
        CK(cudaMemcpyAsync(gB, oB, sizeof(double) * (size_t)nf, cudaMemcpyDeviceToHost, c->st));
    }
    CK(cudaStreamSynchronize(c->st));
    return RELSIM_OK;
}

// The adjoint of the push of one species with the fields held fixed
// (particles kernels: k_push_adjoint). Outputs gE, gB are overwritten with
// this species' contribution.
template <typename T>
int push_adjoint_impl(relsim_ctx* c, int s, const double* gu1, const double* gx1, double* gu0, double* gx0,
                      double* gE, double* gB, int where)
{
    Species& sp = c->sp[s];
    const int64_t n = sp.n, nf = 3 * (int64_t)c->g.ncell;
    const bool host = where == RELSIM_HOST;
    if (host) TRY(ensure_stage(c, 10 * n + 2 * nf));
    const double *d1 = nullptr, *d2 = nullptr;
    TRY(stage_in(c, gu1, 3 * n, where, &d1, 0));
    TRY(stage_in(c, gx1, 2 * n, where, &d2, 3 * n));
    double* ou = host ? c->stage + 5 * n : gu0;
    double* ox = host ? c->stage + 8 * n : gx0;
    double* oE = host ? c->stage + 10 * n : gE;
    double* oB = host ? c->stage + 10 * n + nf : gB;
    CK(cudaMemsetAsync(oE, 0, sizeof(double) * (size_t)nf, c->st));
    CK(cudaMemsetAsync(oB, 0, sizeof(double) * (size_t)nf, c->st));
    if (n > 0)
        CK(push_adjoint<T>(arrays<T>(sp, sp.cur), sp.start, d1, d2, ou, ox, oE, oB, (const T*)c->Eth,
                           (const T*)c->B[c->bcur], c->g, SpeciesConst{c->cfg.q[s], c->cfg.m[s]}, c->st));
    if (host) {
        CK(cudaMemcpyAsync(gu0, ou, sizeof(double) * (size_t)(3 * n), cudaMemcpyDeviceToHost, c->st));
        CK(cudaMemcpyAsync(gx0, ox, sizeof(double) * (size_t)(2 * n), cudaMemcpyDeviceToHost, c->st));
        CK(cudaMemcpyAsync(gE, oE, sizeof(double) * (size_t)nf, cudaMemcpyDeviceToHost, c->st));
        CK(cudaMemcpyAsync(gB, oB, sizeof(double) * (size_t)nf, cudaMemcpyDeviceToHost, c->st));
    }
    CK(cudaStreamSynchronize(c->st));
    return RELSIM_OK;
}

// One whole step's adjoint on the solved step, in place on gradients
// indexed by particle id: per species the gradients are gathered into the
// current order, the push adjoint runs (its dL/dE^{n+theta} and dL/dB^n
// summed over species) and its dL/du^n, dL/dx^{n+1/2} are scattered back;
// the field adjoint takes the pushes' dL/dE^{n+theta}; the deposit adjoints
// add their particle terms and dL/dB^n.
template <typename T>
int step_adjoint_impl(relsim_ctx* c, double* gE, double* gB, double* const* gu, double* const* gx,
                      double* const* gw, int* iters, double* relres)
{
    const int64_t nf = 3 * (int64_t)c->g.ncell, nm = (int64_t)c->g.ncell * kMBlock;
    int64_t nmax = 0;
    for (int s = 0; s < c->cfg.nspecies; ++s) nmax = c->sp[s].n > nmax ? c->sp[s].n : nmax;
    TRY(ensure_adj(c, 10 * nmax + 7 * nf + nm));
    double* L = c->adj;           // 5 nmax: a species' gradients in its current order
    double* P = L + 5 * nmax;     // 5 nmax: its push adjoint's dL/du^n, dL/dx^{n+1/2}
    double* sE = P + 5 * nmax;    // dL/dE^{n+theta} of the pushes
    double* sB = sE + nf;         // dL/dB^n of the pushes and the deposits
    double* fE = sB + nf;         // the field adjoint's dL/dE^n, dL/dB^n, dL/dJhat, dL/dM
    double* fB = fE + nf;
    double* fJ = fB + nf;
    double* fM = fJ + nf;
    double* sEn = fM + nm;        // predicted gbar: dL/dE^n of the pushes and the deposits
    const T* Bn = (const T*)c->B[c->bcur];
    // E^n of the predicted gbar (the solve kept it before E^{n+1} replaced it)
    const T* En = c->En ? (const T*)c->En : nullptr;
    CK(cudaMemsetAsync(sE, 0, sizeof(double) * (size_t)(2 * nf), c->st));
    if (En) CK(cudaMemsetAsync(sEn, 0, sizeof(double) * (size_t)nf, c->st));
    for (int s = 0; s < c->cfg.nspecies; ++s) {
        Species& sp = c->sp[s];
        const int64_t n = sp.n;
        if (n == 0) continue;
        const PArrays<T> a = arrays<T>(sp, sp.cur);
        CK(gather_grad(a.id, gu[s], gx[s], L, L + 3 * n, n, c->st));
        CK(push_adjoint<T>(a, sp.start, L, L + 3 * n, P, P + 3 * n, sE, sB, (const T*)c->Eth, Bn, c->g,
                           SpeciesConst{c->cfg.q[s], c->cfg.m[s]}, c->st, En, sEn));
        CK(scatter_grad(a.id, P, P + 3 * n, gu[s], gx[s], n, false, c->st));
    }
    const int fr = adjoint_impl<T>(c, gE, gB, sE, fE, fB, fJ, fM, iters, relres, RELSIM_DEVICE);
    if (fr != RELSIM_OK && fr != RELSIM_ERR_NOT_CONVERGED) return fr;
    for (int s = 0; s < c->cfg.nspecies; ++s) {
        Species& sp = c->sp[s];
        const int64_t n = sp.n;
        if (n == 0) continue;
        const PArrays<T> a = arrays<T>(sp, sp.cur);
        double* lw = gw && gw[s] ? P : nullptr;   // the push adjoint's output was scattered already
        CK(deposit_adjoint<T>(a, sp.start, fJ, fM, L, L + 3 * n, lw, sB, Bn, c->g,
                              SpeciesConst{c->cfg.q[s], c->cfg.m[s]}, c->st, En, sEn));
        CK(scatter_grad(a.id, L, L + 3 * n, gu[s], gx[s], n, true, c->st));
        if (lw) CK(scatter_add_w(a.id, lw, gw[s], n, c->st));
    }
    if (En)
        CK(add_fields(fE, sEn, gE, nf, c->st));
    else
        CK(cudaMemcpyAsync(gE, fE, sizeof(double) * (size_t)nf, cudaMemcpyDeviceToDevice, c->st));
    CK(add_fields(fB, sB, gB, nf, c->st));
    CK(cudaStreamSynchronize(c->st));
    return fr;
}

// each carried id j of a species becomes ids[j] (range-checked first)
int relabel_impl(relsim_ctx* c, int s, const int32_t* ids, int where)
{
    Species& sp = c->sp[s];
    const int64_t n = sp.n;
    if (n == 0) return RELSIM_OK;
    const int32_t* d = ids;
    if (where == RELSIM_HOST) {
        TRY(ensure_adj(c, (n + 1) / 2));
        CK(cudaMemcpyAsync(c->adj, ids, sizeof(int32_t) * (size_t)n, cudaMemcpyHostToDevice, c->st));
        d = (const int32_t*)c->adj;
    }
    int32_t* id = sp.id[sp.cur];
    CK(cudaMemsetAsync(c->dflag, 0, sizeof(int), c->st));
    CK(check_ids(id, d, n, c->dflag, c->st));
    CK(cudaMemcpyAsync(c->hflag, c->dflag, sizeof(int), cudaMemcpyDeviceToHost, c->st));
    CK(cudaStreamSynchronize(c->st));
    if (*c->hflag & 1) return fail(c, RELSIM_ERR_INVALID_ARG, "an id or a new label is outside [0, %lld)", (long long)n);
    CK(relabel_ids(id, d, n, c->st));
    CK(cudaStreamSynchronize(c->st));
    return RELSIM_OK;
}

// ---------------------------------------------------------------------------
// graph steps enqueued back to back (the batch runner): both layouts are
// captured up front, each step is one graph launch on the context's stream
// plus an asynchronous copy of its solve outcome, and nothing waits until
// the caller synchronises the stream.

bool graph_eligible(const relsim_ctx* c)
{
    return c->state == kReady && c->have_step && graph_path(c) && !c->prof.on && !c->graph_off;
}

StepGraph* graph_for_layout(relsim_ctx* c)
{
    for (StepGraph& g : c->sg)
        if (graph_matches(c, g)) return &g;
    return nullptr;
}

}  // namespace

namespace {
// ---------------------------------------------------------------------------
// Shared launches over the instances of a batch: one deposit launch, one push
// launch and one re-sort launch per species cover the row units of every
// instance (numbered across them); each instance's solve (prologue, the
// restart and Arnoldi loops as conditional nodes, field update) and its
// sort tables run as branches of the same graph, forked from and joined back
// to the batch's stream. Both buffer layouts are captured up front, as for
// single contexts.

template <typename T>
struct SharedDesc {
    std::vector<DepDesc<T>> dep;
    std::vector<PushDesc<T>> push;   // [species][instance]
};

template <typename T>
void shared_descs(const std::vector<relsim_ctx*>& cs, SharedDesc<T>& d, int* total)
{
    const int n = (int)cs.size(), nsp = cs[0]->cfg.nspecies;
    d.dep.assign(n, DepDesc<T>{});
    d.push.assign((size_t)n * nsp, PushDesc<T>{});
    int u0 = 0;
    for (int i = 0; i < n; ++i) {
        relsim_ctx* c = cs[i];
        DepDesc<T>& dd = d.dep[i];
        dd.ds = deposit_args<T>(c);
        dd.B = (const T*)c->B[c->bcur];
        dd.En = c->En ? (const T*)c->E : nullptr;
        dd.M = (T*)c->M;
        dd.J = (T*)c->J;
        dd.g = c->g;
        dd.unit0 = u0;
        for (int s = 0; s < nsp; ++s) {
            Species& sp = c->sp[s];
            PushDesc<T>& p = d.push[(size_t)s * n + i];
            p.src = arrays<T>(sp, sp.cur);
            p.dst = arrays<T>(sp, 1 - sp.cur);
            p.start = sp.start;
            p.start_new = sp.start_alt;
            p.n9 = c->n9;
            p.off9 = c->off9;
            p.Eth = (const T*)c->Eth;
            p.B = (const T*)c->B[c->bcur];
            p.En = (const T*)c->En;
            p.g = c->g;
            p.beta = (T)(c->cfg.q[s] * c->g.dt / (2.0 * c->cfg.m[s]));
            p.dt_dx = (T)(c->g.dt / c->g.dx);
            p.dt_dy = (T)(c->g.dt / c->g.dy);
            p.qdt = (T)(c->cfg.q[s] * c->g.dt);
            p.m = (T)c->cfg.m[s];
            p.led = c->dled + kLedgerField + kLedgerSpecies * s + 1;
            p.err = c->dpush;
            p.unit0 = u0;
        }
        u0 += row_units(c->g);
    }
    *total = u0;
}

}  // namespace

// what a shared graph slot was captured for, per instance
struct SharedKey {
    uint64_t gen = 0;
    int bcur = -1;
    int32_t* start[kMaxSpecies] = {};
};

struct relsim_shared {
    std::vector<relsim_ctx*> c;
    std::vector<SharedKey> key[2];
    int prec = 32, nsp = 1;
    bool pred = false;
    cudaStream_t st = nullptr;
    cudaEvent_t fork = nullptr;
    std::vector<cudaEvent_t> join;
    void* desc[2] = {nullptr, nullptr};   // device descriptors of the two layouts
    cudaGraphExec_t exec[2] = {nullptr, nullptr};
    long long k_static[2] = {0, 0};
    std::vector<long long> k_cycle, k_iter;   // per instance
    int total_units = 0;
    int dep_blocks = 0, push_blocks = 0;           // the launches' grids
    int dep_blocks_req = 0, push_blocks_req = 0;   // as asked for (0: default)
    int64_t steps = 0;
};

namespace {

// every instance on the shared path: 2D, linear shapes, one-cell moves, ready
// for graph steps, the same precision, species count and reading of gbar,
// every species loaded
bool shared_eligible(const std::vector<relsim_ctx*>& cs)
{
    if (cs.empty()) return false;
    for (relsim_ctx* c : cs) {
        if (!graph_eligible(c) || !c->fast_sort || c->g.dim != 2 || c->g.shape != 1) return false;
        if (c->prec != cs[0]->prec || c->cfg.nspecies != cs[0]->cfg.nspecies ||
            (c->En != nullptr) != (cs[0]->En != nullptr))
            return false;
        for (int s = 0; s < c->cfg.nspecies; ++s)
            if (c->sp[s].n <= 0) return false;
    }
    return true;
}

// capture one step of every instance for the current buffer layout into
// graph slot k (descriptors already uploaded to sb->desc[k])
template <typename T>
int shared_capture(relsim_shared* sb, int k)
{
    const int n = (int)sb->c.size(), nsp = sb->nsp;
    relsim_ctx* c0 = sb->c[0];
    const DepDesc<T>* ddep = (const DepDesc<T>*)sb->desc[k];
    const PushDesc<T>* dpush = (const PushDesc<T>*)((const unsigned char*)sb->desc[k] + sizeof(DepDesc<T>) * n);
    std::vector<StepGraph> tally(n);
    sb->k_static[k] = 0;
    t_capture_count = &sb->k_static[k];
    int r = RELSIM_OK;
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamBeginCapture(sb->st, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) {
        t_capture_count = nullptr;
        return fail(c0, RELSIM_ERR_CUDA, "cudaStreamBeginCapture: %s", cudaGetErrorString(e));
    }
    auto run = [&]() -> int {
        for (relsim_ctx* c : sb->c) {
            CK(zero_fill(c->M, c->esz * (size_t)c->g.ncell * mblock_of(c->g), sb->st));
            CK(zero_fill(c->J, c->esz * 3 * (size_t)c->g.ncell, sb->st));
        }
        CK_CTX(c0, deposit_batch<T>(ddep, n, sb->total_units, sb->pred, c0->dpush, sb->st, sb->dep_blocks));
        CK_CTX(c0, cudaEventRecord(sb->fork, sb->st));
        for (int i = 0; i < n; ++i) {
            relsim_ctx* c = sb->c[i];
            CK(cudaStreamWaitEvent(c->gst, sb->fork, 0));
            cudaStream_t user = c->st;
            c->st = c->gst;
            c->capturing = true;
            t_capture_count = &tally[i].k_static;
            const GmSetup S = gm_setup(c);
            int rr = capture_solve<T>(c, S, tally[i]);
            for (int s = 0; s < nsp && rr == RELSIM_OK; ++s) {
                double* led = c->dled + kLedgerField + kLedgerSpecies * s;
                // K0 of this step is the kinetic energy the last push left;
                // the shared push adds its sums into the slots after it
                if (cudaMemcpyAsync(led, led + 4, sizeof(double), cudaMemcpyDeviceToDevice, c->st) != cudaSuccess ||
                    cudaMemsetAsync(led + 1, 0, sizeof(double) * (kLedgerSpecies - 1), c->st) != cudaSuccess)
                    rr = fail(c0, RELSIM_ERR_CUDA, "ledger slots: %s", cudaGetErrorString(cudaGetLastError()));
            }
            if (rr == RELSIM_OK && cudaEventRecord(sb->join[i], c->st) != cudaSuccess)
                rr = fail(c0, RELSIM_ERR_CUDA, "join");
            c->st = user;
            c->capturing = false;
            t_capture_count = &sb->k_static[k];
            if (rr != RELSIM_OK) return rr;
            sb->k_static[k] += tally[i].k_static;
            sb->k_cycle[i] = tally[i].k_cycle;
            sb->k_iter[i] = tally[i].k_iter;
        }
        for (int i = 0; i < n; ++i) CK_CTX(c0, cudaStreamWaitEvent(sb->st, sb->join[i], 0));
        for (int s = 0; s < nsp; ++s) {
            const PushDesc<T>* dp = dpush + (size_t)s * n;
            CK_CTX(c0, push_sort_batch<T>(dp, n, sb->total_units, sb->pred, sb->push_blocks, sb->st));
            CK_CTX(c0, cudaEventRecord(sb->fork, sb->st));
            for (int i = 0; i < n; ++i) {
                relsim_ctx* c = sb->c[i];
                Species& sp = c->sp[s];
                CK(cudaStreamWaitEvent(c->gst, sb->fork, 0));
                CK(move_counts(c->n9, c->count_new, c->g, c->gst));
                CK(scan_exclusive_i32(c->count_new, sp.start_alt, c->g.ncell, sp.start_alt + c->g.ncell, c->scan_tmp,
                                      c->gst));
                CK(cudaEventRecord(sb->join[i], c->gst));
            }
            for (int i = 0; i < n; ++i) CK_CTX(c0, cudaStreamWaitEvent(sb->st, sb->join[i], 0));
            CK_CTX(c0, permute_batch<T>(dp, n, sb->total_units, sb->st));
        }
        for (relsim_ctx* c : sb->c) CK(cudaMemcpyAsync(c->hpush, c->dpush, sizeof(int), cudaMemcpyDeviceToHost, sb->st));
        return RELSIM_OK;
    };
    r = run();
    e = cudaStreamEndCapture(sb->st, &graph);
    t_capture_count = nullptr;
    if (r == RELSIM_OK && e != cudaSuccess) r = fail(c0, RELSIM_ERR_CUDA, "shared capture: %s", cudaGetErrorString(e));
    if (r == RELSIM_OK) {
        e = cudaGraphInstantiate(&sb->exec[k], graph, 0);
        if (e != cudaSuccess) {
            sb->exec[k] = nullptr;
            r = fail(c0, RELSIM_ERR_CUDA, "shared cudaGraphInstantiate: %s", cudaGetErrorString(e));
        }
    }
    if (graph) cudaGraphDestroy(graph);
    (void)cudaGetLastError();
    if (r == RELSIM_OK) {
        sb->key[k].assign(n, SharedKey{});
        for (int i = 0; i < n; ++i) {
            SharedKey& q = sb->key[k][i];
            q.gen = sb->c[i]->gen;
            q.bcur = sb->c[i]->bcur;
            for (int s = 0; s < kMaxSpecies; ++s) q.start[s] = sb->c[i]->sp[s].start;
        }
    }
    return r;
}

// the graph slot captured for every instance's current buffer layout, -1 if
// none (an instance was reloaded, retuned or stepped on its own since)
int shared_slot(const relsim_shared* sb)
{
    for (int k = 0; k < 2; ++k) {
        if (!sb->exec[k] || sb->key[k].size() != sb->c.size()) continue;
        bool ok = true;
        for (size_t i = 0; i < sb->c.size() && ok; ++i) {
            const relsim_ctx* c = sb->c[i];
            const SharedKey& q = sb->key[k][i];
            ok = q.gen == c->gen && q.bcur == c->bcur && graph_eligible(c);
            for (int s = 0; s < kMaxSpecies && ok; ++s) ok = q.start[s] == c->sp[s].start;
        }
        if (ok) return k;
    }
    return -1;
}

template <typename T>
int shared_upload(relsim_shared* sb, int k)
{
    SharedDesc<T> d;
    shared_descs<T>(sb->c, d, &sb->total_units);
    const size_t bd = sizeof(DepDesc<T>) * d.dep.size(), bp = sizeof(PushDesc<T>) * d.push.size();
    if (!sb->desc[k] && cudaMalloc(&sb->desc[k], bd + bp) != cudaSuccess) return RELSIM_ERR_OOM;
    if (cudaMemcpy(sb->desc[k], d.dep.data(), bd, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy((unsigned char*)sb->desc[k] + bd, d.push.data(), bp, cudaMemcpyHostToDevice) != cudaSuccess)
        return RELSIM_ERR_CUDA;
    return RELSIM_OK;
}

template <typename T>
int shared_prepare(relsim_shared* sb)
{
    const int n = (int)sb->c.size();
    relsim_ctx* c = sb->c[0];
    for (relsim_ctx* ci : sb->c) {
        TRY(solve_reserve(ci, gm_setup(ci)));
        CK_CTX(ci, cudaStreamSynchronize(ci->st));
    }
    int dev = 0, nsm = 152;
    CK(cudaGetDevice(&dev));
    CK(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    if (sb->dep_blocks <= 0) sb->dep_blocks = 2 * nsm;
    if (sb->push_blocks <= 0) sb->push_blocks = 16 * nsm;
    sb->k_cycle.assign(n, 0);
    sb->k_iter.assign(n, 0);
    for (int k = 0; k < 2; ++k) {
        int r = shared_upload<T>(sb, k);
        if (r == RELSIM_OK) r = shared_capture<T>(sb, k);
        if (r != RELSIM_OK) {
            if (k == 1)
                for (relsim_ctx* ci : sb->c) push_commit(ci);
            return r;
        }
        for (relsim_ctx* ci : sb->c) push_commit(ci);   // the next layout; after both, the first again
    }
    return RELSIM_OK;
}

}  // namespace

namespace relsim {

int shared_create(relsim_ctx* const* ctxs, int count, int dep_blocks, int push_blocks, relsim_shared** out)
{
    *out = nullptr;
    std::vector<relsim_ctx*> cs(ctxs, ctxs + count);
    if (!shared_eligible(cs)) return 0;
    relsim_shared* sb = new (std::nothrow) relsim_shared;
    if (!sb) return RELSIM_ERR_OOM;
    sb->c = cs;
    sb->prec = cs[0]->prec;
    sb->nsp = cs[0]->cfg.nspecies;
    sb->pred = cs[0]->En != nullptr;
    sb->dep_blocks = sb->dep_blocks_req = dep_blocks;
    sb->push_blocks = sb->push_blocks_req = push_blocks;
    sb->join.assign(count, nullptr);
    int r = RELSIM_OK;
    if (cudaStreamCreateWithFlags(&sb->st, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&sb->fork, cudaEventDisableTiming) != cudaSuccess)
        r = RELSIM_ERR_CUDA;
    for (int i = 0; i < count && r == RELSIM_OK; ++i)
        if (cudaEventCreateWithFlags(&sb->join[i], cudaEventDisableTiming) != cudaSuccess) r = RELSIM_ERR_CUDA;
    if (r == RELSIM_OK) r = sb->prec == 32 ? shared_prepare<float>(sb) : shared_prepare<double>(sb);
    if (r != RELSIM_OK) {
        shared_destroy(sb);
        return r;
    }
    *out = sb;
    return 1;
}

void shared_destroy(relsim_shared* sb)
{
    if (!sb) return;
    if (sb->st) cudaStreamSynchronize(sb->st);
    for (int k = 0; k < 2; ++k) {
        if (sb->exec[k]) cudaGraphExecDestroy(sb->exec[k]);
        if (sb->desc[k]) cudaFree(sb->desc[k]);
    }
    for (cudaEvent_t e : sb->join)
        if (e) cudaEventDestroy(e);
    if (sb->fork) cudaEventDestroy(sb->fork);
    if (sb->st) cudaStreamDestroy(sb->st);
    (void)cudaGetLastError();
    delete sb;
}

cudaStream_t shared_stream(const relsim_shared* sb) { return sb->st; }

bool shared_valid(const relsim_shared* sb, relsim_ctx* const* ctxs, int count, int dep_blocks, int push_blocks)
{
    if (!sb || (int)sb->c.size() != count || sb->dep_blocks_req != dep_blocks || sb->push_blocks_req != push_blocks)
        return false;
    for (int i = 0; i < count; ++i)
        if (sb->c[i] != ctxs[i]) return false;
    return shared_slot(sb) >= 0;
}

// one step of every instance: the graph of the current layout, then each
// instance's solve outcome copied to heads + i * head_stride (pinned)
int shared_enqueue(relsim_shared* sb, unsigned char* heads, size_t head_stride)
{
    const int k = shared_slot(sb);
    relsim_ctx* c0 = sb->c[0];
    if (k < 0) return fail(c0, RELSIM_ERR_INTERNAL, "no shared graph for the instances' current layout");
    CK_CTX(c0, cudaGraphLaunch(sb->exec[k], sb->st));
    for (size_t i = 0; i < sb->c.size(); ++i) {
        relsim_ctx* c = sb->c[i];
        CK_CTX(c0, cudaMemcpyAsync(heads + i * head_stride, c->gms, kGmHead, cudaMemcpyDeviceToHost, sb->st));
        push_commit(c);
        c->state = kReady;
        c->have_step = true;
        ++c->step;
        ++c->graph_steps;
    }
    ++sb->steps;
    return RELSIM_OK;
}

// one instance's outcome of a shared step (after the batch's stream was
// synchronised); counts the kernels its branches ran
int shared_outcome(relsim_shared* sb, int i, const void* head, int* iters, bool first)
{
    relsim_ctx* c = sb->c[i];
    GmState h;
    memcpy(&h, head, kGmHead);
    if (first) count_launches((int)sb->k_static[0]);
    count_launches((int)(sb->k_cycle[i] * h.restarts + sb->k_iter[i] * h.total));
    // the shared deposit reports its staging timeouts on the first instance
    if (i != 0 && (*sb->c[0]->hpush & 2))
        return fail(c, RELSIM_ERR_TIMEOUT, "a shared-memory staging wait of the shared deposit gave up");
    TRY(check_push(c));
    return solve_outcome(c, &h, iters, nullptr);
}

size_t ctx_graph_head_bytes() { return kGmHead; }

int ctx_graph_prepare(relsim_ctx* c)
{
    if (!graph_eligible(c)) return 0;
    bool have_a = graph_for_layout(c) != nullptr;
    push_commit(c);
    bool have_b = graph_for_layout(c) != nullptr;
    push_commit(c);
    if (have_a && have_b) return 1;
    for (int k = 0; k < 2; ++k) {
        const int r = c->prec == 32 ? capture_step<float>(c, c->sg[k]) : capture_step<double>(c, c->sg[k]);
        if (r != RELSIM_OK) {
            if (k == 1) push_commit(c);
            c->graph_off = true;
            c->graph_why = c->err;
            c->err.clear();
            return 0;
        }
        push_commit(c);   // the next layout; after both captures, the first again
    }
    return 1;
}

int ctx_graph_enqueue(relsim_ctx* c, void* head)
{
    StepGraph* G = graph_for_layout(c);
    if (!G) return fail(c, RELSIM_ERR_INTERNAL, "no step graph for the current layout");
    CK(cudaGraphLaunch(G->exec, c->st));
    CK(cudaMemcpyAsync(head, c->gms, kGmHead, cudaMemcpyDeviceToHost, c->st));
    push_commit(c);
    c->state = kReady;
    c->have_step = true;
    ++c->step;
    ++c->graph_steps;
    return RELSIM_OK;
}

int ctx_graph_outcome(relsim_ctx* c, const void* head, int* iters)
{
    GmState h;
    memcpy(&h, head, kGmHead);
    const StepGraph& G = c->sg[0];
    count_launches((int)(G.k_static + G.k_cycle * h.restarts + G.k_iter * h.total));
    TRY(check_push(c));
    return solve_outcome(c, &h, iters, nullptr);
}

}  // namespace relsim

namespace {

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
    // rows of nx values along x: ny of them in 2D, ny nz in 3D (contiguous)
    const int nx = c->g.nx, ny = c->g.ny * c->g.nz;
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

// the energy of one mode and its gradient in B (component comp)
template <typename T>
int mode_grad_impl(relsim_ctx* c, int comp, int mode, double* energy, double* gB, int where)
{
    const int nx = c->g.nx, ny = c->g.ny * c->g.nz;
    const int64_t nc = c->g.ncell;
    if (mode + 1 > c->mode_tw_m) {
        dfree(c->mode_tw);
        c->mode_tw_m = 0;
        TRY(dalloc(c, &c->mode_tw, sizeof(T) * 2 * (size_t)nx * (size_t)(mode + 1)));
        CK(mode_twiddles<T>((T*)c->mode_tw, nx, mode + 1, c->st));
        c->mode_tw_m = mode + 1;
    }
    // device scratch: ny row values, the energy, and a 3 ncell gradient
    // staged for host outputs
    const int64_t need = (int64_t)ny + 1 + (where == RELSIM_HOST ? 3 * nc : 0);
    if (need > c->mode_rows_cap) {
        dfree(c->mode_rows);
        c->mode_rows_cap = 0;
        TRY(dalloc(c, &c->mode_rows, sizeof(double) * (size_t)need));
        c->mode_rows_cap = need;
    }
    const int bnow = c->state == kSolved ? 1 - c->bcur : c->bcur;
    const T* Bc = (const T*)c->B[bnow] + (int64_t)comp * nc;
    double* e_dev = where == RELSIM_DEVICE ? energy : c->mode_rows + ny;
    double* g_dev = where == RELSIM_DEVICE ? gB : c->mode_rows + ny + 1;
    CK(cudaMemsetAsync(g_dev, 0, sizeof(double) * 3 * (size_t)nc, c->st));
    CK(mode_gradient<T>(Bc, (const T*)c->mode_tw, nx, ny, mode, c->g.dV, c->mode_rows, e_dev,
                        g_dev + (int64_t)comp * nc, c->st));
    if (where == RELSIM_HOST) {
        CK(cudaMemcpyAsync(energy, e_dev, sizeof(double), cudaMemcpyDeviceToHost, c->st));
        CK(cudaMemcpyAsync(gB, g_dev, sizeof(double) * 3 * (size_t)nc, cudaMemcpyDeviceToHost, c->st));
        CK(cudaStreamSynchronize(c->st));
    }
    return RELSIM_OK;
}

int check_push(relsim_ctx* c)
{
    if (*c->hpush & 2)
        return fail(c, RELSIM_ERR_TIMEOUT, "a shared-memory staging wait gave up (deposit, push or operator)");
    if (*c->hpush)
        return fail(c, RELSIM_ERR_INTERNAL, "particle sort: the moves counted and the new cell starts disagreed");
    return RELSIM_OK;
}

int ledger_impl(relsim_ctx* c, relsim_energy* out)
{
    double h[kLedgerLen];
    TRY(readback(c, c->dled, kLedgerLen, h));
    TRY(check_push(c));
    return ledger_fill(c, h, out);
}

// the ledger from the device sums h (kLedgerLen values)
int ledger_fill(relsim_ctx* c, const double* h, relsim_energy* out)
{
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
    if (cfg->dim != 2 && cfg->dim != 3) { *why = "dim must be 2 or 3"; return 0; }
    if (cfg->nx < 3 || cfg->ny < 3) { *why = "nx and ny must be >= 3"; return 0; }
    if (cfg->dim == 3 && cfg->nz < 3) { *why = "nz must be >= 3 in 3D"; return 0; }
    if (cfg->dim == 3 && !(cfg->dz > 0)) { *why = "dz must be > 0 in 3D"; return 0; }
    if (cfg->dim == 3 && cfg->gamma_pred) { *why = "the 3D form covers the base scheme (gamma_pred = 0)"; return 0; }
    if (cfg->shape < 0 || cfg->shape > 2) { *why = "shape must be 0 or 1 (linear) or 2 (quadratic)"; return 0; }
    if (cfg->shape == 2 && (cfg->dim != 2 || cfg->gamma_pred)) {
        *why = "quadratic shapes cover the 2D base scheme";
        return 0;
    }
    if ((int64_t)cfg->nx * cfg->ny * (cfg->dim == 3 ? cfg->nz : 1) > (int64_t)1 << 28) {
        *why = "grid too large (more than 2^28 cells)";
        return 0;
    }
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
    c->g.dim = cfg->dim;
    c->g.shape = cfg->shape == 2 ? 2 : 1;
    c->g.nz = cfg->dim == 3 ? cfg->nz : 1;
    c->g.dz = cfg->dim == 3 ? cfg->dz : 1.0;
    c->g.ncell = cfg->nx * cfg->ny * c->g.nz;
    c->g.dx = cfg->dx;
    c->g.dy = cfg->dy;
    c->g.dt = cfg->dt;
    c->g.theta = cfg->theta_implicit;
    c->g.dV = cfg->dx * cfg->dy * c->g.dz;
    grid_derive(c->g);
    // the FP32 form of the 2D scheme with linear shapes keeps its GMRES
    // vectors as double-float pairs (FP32-pipe arithmetic at close to FP64
    // precision) unless FP64 vectors are asked for
    c->g.df = cfg->precision == 32 && cfg->dim == 2 && c->g.shape == 1 && !cfg->gmres_fp64 ? 1 : 0;
    // one-cell moves per step: c dt <= min(dx, dy); the 3D form always
    // takes the general push (any move length, radix sort) and host-driven steps
    c->fast_sort = cfg->dim == 2 && c->g.shape == 1 && cfg->dt <= cfg->dx && cfg->dt <= cfg->dy;
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
    if (cfg->gamma_pred) A(dalloc(c, &c->En, c->esz * 3 * nc));
    A(dalloc(c, &c->B[0], c->esz * 3 * nc));
    A(dalloc(c, &c->B[1], c->esz * 3 * nc));
    A(dalloc(c, &c->J, c->esz * 3 * nc));
    A(dalloc(c, &c->M, c->esz * mblock_of(c->g) * nc));
    A(dalloc(c, &c->n9, c->g.dim == 3 ? 16 : sizeof(int32_t) * kNDir * nc));
    A(dalloc(c, &c->off9, c->g.dim == 3 ? 16 : sizeof(int32_t) * kNDir * nc));
    A(dalloc(c, &c->count_new, sizeof(int32_t) * (nc + 1)));
    c->scan_tmp_n = scan_tmp_ints(nc);
    A(dalloc(c, &c->scan_tmp, sizeof(int32_t) * c->scan_tmp_n));
    A(dalloc(c, &c->V, sizeof(double) * (size_t)(c->mrest + 1) * c->nvec));
    A(dalloc(c, &c->gw, sizeof(double) * c->nvec));
    A(dalloc(c, &c->gw2, sizeof(double) * c->nvec));
    A(dalloc(c, &c->gx, sizeof(double) * c->nvec));
    A(dalloc(c, &c->gb, sizeof(double) * c->nvec));
    A(dalloc(c, &c->dsum, sizeof(double) * 4 * (kMaxRestart + 2)));
    A(dalloc(c, &c->gms, sizeof(GmState)));
    if (cudaMemsetAsync(c->gms, 0, sizeof(GmState), c->st) != cudaSuccess) {
        r = fail(c, RELSIM_ERR_CUDA, "cudaMemsetAsync failed");
        goto fail_init;
    }
    if (cudaMallocHost((void**)&c->ghead, 2 * sizeof(GmState)) != cudaSuccess) {
        r = fail(c, RELSIM_ERR_OOM, "cudaMallocHost failed");
        goto fail_init;
    }
    if (cudaStreamCreateWithFlags(&c->gst, cudaStreamNonBlocking) != cudaSuccess ||
        cudaStreamCreateWithFlags(&c->aux[0], cudaStreamNonBlocking) != cudaSuccess ||
        cudaStreamCreateWithFlags(&c->aux[1], cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->gjoin[0], cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->gjoin[1], cudaEventDisableTiming) != cudaSuccess) {
        r = fail(c, RELSIM_ERR_CUDA, "stream or event creation failed");
        goto fail_init;
    }
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
        if (e == cudaSuccess) e = cudaMemsetAsync(c->M, 0, c->esz * mblock_of(c->g) * nc, c->st);
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
            for (int k = 0; k < 7; ++k) dfree(sp.a[b][k]);
            dfree(sp.id[b]);
        }
        dfree(sp.start);
        dfree(sp.start_alt);
    }
    dfree(c->E); dfree(c->Eth); dfree(c->En); dfree(c->B[0]); dfree(c->B[1]); dfree(c->J); dfree(c->M);
    dfree(c->n9); dfree(c->off9); dfree(c->count_new); dfree(c->scan_tmp);
    for (int b = 0; b < 2; ++b) {
        dfree(c->rk[b]);
        dfree(c->rv[b]);
    }
    dfree(c->rtmp);
    dfree(c->V); dfree(c->gw); dfree(c->gw2); dfree(c->gx); dfree(c->gb); dfree(c->partial);
    dfree(c->dsum); dfree(c->dled); dfree(c->dflag); dfree(c->dpush); dfree(c->stage); dfree(c->adj);
    dfree(c->spec_w); dfree(c->spec_c); dfree(c->spec_e);
    dfree(c->mode_tw); dfree(c->mode_rows);
    dfree(c->gms);
    if (c->ghead) cudaFreeHost(c->ghead);
    for (StepGraph& G : c->sg)
        if (G.exec) cudaGraphExecDestroy(G.exec);
    for (cudaStream_t t : {c->gst, c->aux[0], c->aux[1]})
        if (t) cudaStreamDestroy(t);
    for (cudaEvent_t e : c->gjoin)
        if (e) cudaEventDestroy(e);
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
    ++c->gen;
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
    ++c->gen;
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

int relsim_load_particles_native(relsim_ctx* c, int species, int64_t n, const int32_t* start, const void* off,
                                 const void* u, const void* w, const int32_t* id, int where)
{
    if (!c) return RELSIM_ERR_INVALID_ARG;
    ++c->gen;
    if (species < 0 || species >= c->cfg.nspecies)
        return fail(c, RELSIM_ERR_INVALID_ARG, "species %d out of range", species);
    if (n < 0 || n > 2147483647LL) return fail(c, RELSIM_ERR_INVALID_ARG, "bad particle count %lld", (long long)n);
    if (!start) return fail(c, RELSIM_ERR_INVALID_ARG, "null cell start table");
    if (n > 0 && (!off || !u || !w)) return fail(c, RELSIM_ERR_INVALID_ARG, "null particle array");
    if (id && !c->cfg.track_ids) return fail(c, RELSIM_ERR_INVALID_ARG, "ids are not tracked");
    if (where != RELSIM_HOST && where != RELSIM_DEVICE) return fail(c, RELSIM_ERR_INVALID_ARG, "bad where");
    int r = DISPATCH(load_native_impl, c, species, n, start, off, u, w, id, where);
    if (r == RELSIM_OK) {
        c->state = kReady;
        c->have_step = false;
        c->step = 0;
    }
    return r;
}

int relsim_get_particles_native(relsim_ctx* c, int species, int32_t* start, void* off, void* u, void* w,
                                int32_t* id, int where)
{
    if (!c) return RELSIM_ERR_INVALID_ARG;
    if (species < 0 || species >= c->cfg.nspecies)
        return fail(c, RELSIM_ERR_INVALID_ARG, "species %d out of range", species);
    if (id && !c->cfg.track_ids) return fail(c, RELSIM_ERR_INVALID_ARG, "ids are not tracked");
    if (where != RELSIM_HOST && where != RELSIM_DEVICE) return fail(c, RELSIM_ERR_INVALID_ARG, "bad where");
    if (!c->sp[species].start) return fail(c, RELSIM_ERR_BAD_STATE, "species %d was never loaded", species);
    return DISPATCH(get_native_impl, c, species, start, off, u, w, id, where);
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
    const int64_t nm = (int64_t)c->g.ncell * mblock_of(c->g), nj = 3 * (int64_t)c->g.ncell;
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
    ++c->gen;
    if (c->state == kEmpty) return fail(c, RELSIM_ERR_BAD_STATE, "context not initialised");
    if (c->state == kSolved) return fail(c, RELSIM_ERR_BAD_STATE, "push the solved step first");
    const int64_t nm = (int64_t)c->g.ncell * mblock_of(c->g), nj = 3 * (int64_t)c->g.ncell;
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

int relsim_set_launch_shapes(relsim_ctx* c, int deposit_blocks, int push_blocks, int op_rows)
{
    if (!c) return RELSIM_ERR_INVALID_ARG;
    if (deposit_blocks < 0 || push_blocks < 0 || deposit_blocks > (1 << 20) || push_blocks > (1 << 20))
        return fail(c, RELSIM_ERR_INVALID_ARG, "block counts must be 0 .. 2^20");
    const int def = c->prec == 32 ? 8 : 4, alt = c->prec == 32 ? 4 : 2;
    if (op_rows != 0 && op_rows != def && op_rows != alt)
        return fail(c, RELSIM_ERR_INVALID_ARG, "operator tile rows must be 0, %d or %d", def, alt);
    c->dep_blocks = deposit_blocks;
    c->push_cap = push_blocks;
    c->g.op_y = op_rows == alt ? alt : 0;
    ++c->gen;   // step graphs hold the old launch shapes
    return RELSIM_OK;
}

int relsim_autotune(relsim_ctx* c, relsim_tuning* out)
{
    if (!c) return RELSIM_ERR_INVALID_ARG;
    if (c->state != kReady) return fail(c, RELSIM_ERR_BAD_STATE, "autotune needs a loaded state before a build");
    return DISPATCH(autotune_impl, c, out);
}

int relsim_deposit_adjoint(relsim_ctx* c, int species, const double* gJ, const double* gM, double* gu0,
                           double* gx0, double* gB, double* gw0, int where)
{
    if (!c) return RELSIM_ERR_INVALID_ARG;
    if (c->g.dim == 3 || c->g.shape == 2)
        return fail(c, RELSIM_ERR_INVALID_ARG, "the adjoints cover the 2D form with linear shapes");
    if (species < 0 || species >= c->cfg.nspecies) return fail(c, RELSIM_ERR_INVALID_ARG, "species %d out of range", species);
    if (where != RELSIM_HOST && where != RELSIM_DEVICE) return fail(c, RELSIM_ERR_INVALID_ARG, "bad where");
    if (!gJ || !gM || !gB || (c->sp[species].n > 0 && (!gu0 || !gx0)))
        return fail(c, RELSIM_ERR_INVALID_ARG, "null array");
    if (c->En) return fail(c, RELSIM_ERR_INVALID_ARG, "the deposit adjoint covers the base scheme (gamma_pred = 0)");
    if (c->state != kBuilt && c->state != kSolved)
        return fail(c, RELSIM_ERR_BAD_STATE, "the deposit adjoint needs a built step (before the push)");
    return DISPATCH(deposit_adjoint_impl, c, species, gJ, gM, gu0, gx0, gB, gw0, where);
}

int relsim_push_adjoint(relsim_ctx* c, int species, const double* gu1, const double* gx1, double* gu0,
                        double* gx0, double* gE, double* gB, int where)
{
    if (!c) return RELSIM_ERR_INVALID_ARG;
    if (c->g.dim == 3 || c->g.shape == 2)
        return fail(c, RELSIM_ERR_INVALID_ARG, "the adjoints cover the 2D form with linear shapes");
    if (species < 0 || species >= c->cfg.nspecies) return fail(c, RELSIM_ERR_INVALID_ARG, "species %d out of range", species);
    if (where != RELSIM_HOST && where != RELSIM_DEVICE) return fail(c, RELSIM_ERR_INVALID_ARG, "bad where");
    if (c->sp[species].n > 0 && (!gu1 || !gx1 || !gu0 || !gx0)) return fail(c, RELSIM_ERR_INVALID_ARG, "null array");
    if (!gE || !gB) return fail(c, RELSIM_ERR_INVALID_ARG, "null field gradient");
    if (c->En) return fail(c, RELSIM_ERR_INVALID_ARG, "the push adjoint covers the base scheme (gamma_pred = 0)");
    if (c->state != kSolved) return fail(c, RELSIM_ERR_BAD_STATE, "the push adjoint needs a solved step (before the push)");
    return DISPATCH(push_adjoint_impl, c, species, gu1, gx1, gu0, gx0, gE, gB, where);
}

int relsim_step_adjoint(relsim_ctx* c, double* gE, double* gB, double* const* gu, double* const* gx,
                        double* const* gw, int* iters, double* rel_residual)
{
    if (!c) return RELSIM_ERR_INVALID_ARG;
    if (c->g.dim == 3 || c->g.shape == 2)
        return fail(c, RELSIM_ERR_INVALID_ARG, "the adjoints cover the 2D form with linear shapes");
    if (!gE || !gB || !gu || !gx) return fail(c, RELSIM_ERR_INVALID_ARG, "null array");
    for (int s = 0; s < c->cfg.nspecies; ++s)
        if (c->sp[s].n > 0 && (!gu[s] || !gx[s])) return fail(c, RELSIM_ERR_INVALID_ARG, "null particle gradient");
    if (!c->cfg.track_ids) return fail(c, RELSIM_ERR_INVALID_ARG, "the step adjoint needs track_ids");
    if (c->state != kReady) return fail(c, RELSIM_ERR_BAD_STATE, "the step adjoint needs a loaded or pushed state");
    int r = relsim_build_mass_matrix(c);
    if (r != RELSIM_OK) return r;
    const int fs = relsim_field_solve(c, nullptr, nullptr);
    if (fs != RELSIM_OK && fs != RELSIM_ERR_NOT_CONVERGED) return fs;
    r = DISPATCH(step_adjoint_impl, c, gE, gB, gu, gx, gw, iters, rel_residual);
    if (r == RELSIM_OK && fs == RELSIM_ERR_NOT_CONVERGED)
        r = fail(c, RELSIM_ERR_NOT_CONVERGED, "the step's forward solve did not converge");
    return r;
}

int relsim_relabel_particles(relsim_ctx* c, int species, const int32_t* ids, int where)
{
    if (!c) return RELSIM_ERR_INVALID_ARG;
    if (species < 0 || species >= c->cfg.nspecies) return fail(c, RELSIM_ERR_INVALID_ARG, "species %d out of range", species);
    if (where != RELSIM_HOST && where != RELSIM_DEVICE) return fail(c, RELSIM_ERR_INVALID_ARG, "bad where");
    if (!c->cfg.track_ids) return fail(c, RELSIM_ERR_INVALID_ARG, "ids are not tracked");
    if (c->sp[species].n > 0 && !ids) return fail(c, RELSIM_ERR_INVALID_ARG, "null ids");
    return relabel_impl(c, species, ids, where);
}

int relsim_field_adjoint(relsim_ctx* c, const double* gE1, const double* gB1, const double* gEt, double* gE0,
                         double* gB0, double* gJ, double* gM, int* iters, double* rel_residual, int where)
{
    if (!c) return RELSIM_ERR_INVALID_ARG;
    if (c->g.dim == 3 || c->g.shape == 2)
        return fail(c, RELSIM_ERR_INVALID_ARG, "the adjoints cover the 2D form with linear shapes");
    if (!gE1 || !gB1) return fail(c, RELSIM_ERR_INVALID_ARG, "null upstream gradient");
    if (where != RELSIM_HOST && where != RELSIM_DEVICE) return fail(c, RELSIM_ERR_INVALID_ARG, "bad where");
    if (c->state != kSolved) return fail(c, RELSIM_ERR_BAD_STATE, "the adjoint needs a solved step (before the push)");
    return DISPATCH(adjoint_impl, c, gE1, gB1, gEt, gE0, gB0, gJ, gM, iters, rel_residual, where);
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
    // the GMRES work vectors are free outside a solve; with double-float
    // vectors the FP64 input and output are converted on either side
    const double* vin = dv;
    if (c->g.df) {
        CK(vec_from_double(dv, c->gw2, n, 1, c->st));
        vin = c->gw2;
    }
    if (c->prec == 32) CK(apply_A<float>((const float*)c->M, vin, c->gw, c->g, c->dpush, c->st));
    else CK(apply_A<double>((const double*)c->M, vin, c->gw, c->g, c->dpush, c->st));
    const double* res = c->gw;
    if (c->g.df) {
        CK(vec_to_double(c->gw, c->gw2, n, 1, c->st));
        res = c->gw2;
    }
    if (where == RELSIM_DEVICE) return copy_out(c, out, res, n, where);
    CK(cudaMemcpyAsync(c->hpush, c->dpush, sizeof(int), cudaMemcpyDeviceToHost, c->st));
    TRY(copy_out(c, out, res, n, where));
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

int relsim_field_mode_gradient(relsim_ctx* c, int component, int mode, double* energy, double* gB, int where)
{
    if (!c) return RELSIM_ERR_INVALID_ARG;
    if (component < 0 || component > 2) return fail(c, RELSIM_ERR_INVALID_ARG, "component %d out of range", component);
    if (mode < 0 || mode > c->g.nx / 2) return fail(c, RELSIM_ERR_INVALID_ARG, "mode %d outside [0, nx/2]", mode);
    if (!energy || !gB) return fail(c, RELSIM_ERR_INVALID_ARG, "null output");
    if (where != RELSIM_HOST && where != RELSIM_DEVICE) return fail(c, RELSIM_ERR_INVALID_ARG, "bad where");
    return DISPATCH(mode_grad_impl, c, component, mode, energy, gB, where);
}

int relsim_graph_info(const relsim_ctx* c, int64_t* graph_steps, int* disabled, const char** why)
{
    if (!c) return RELSIM_ERR_INVALID_ARG;
    if (graph_steps) *graph_steps = c->graph_steps;
    if (disabled) *disabled = c->graph_off ? 1 : 0;
    if (why) *why = c->graph_why.c_str();
    return RELSIM_OK;
}

int relsim_step(relsim_ctx* c, relsim_energy* ledger)
{
    if (!c) return RELSIM_ERR_INVALID_ARG;
    // after one host-driven step has sized every buffer, steps run as a
    // captured graph (not while profiling: event timing needs host launches)
    if (c->state == kReady && c->have_step && graph_path(c) && !c->prof.on && !c->graph_off) {
        int status = RELSIM_OK;
        const int r = DISPATCH(step_graph, c, ledger, &status);
        if (r == RELSIM_OK) return status;
        if (r != 1) return r;
    }
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
