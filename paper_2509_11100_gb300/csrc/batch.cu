// batch.cu -- independent instances advanced concurrently (a parameter scan
// of tearing runs: uneven grid sizes, sheet thicknesses and magnetisations,
// each instance a context on a stream of its own), and the exponential
// growth-rate fit of a diagnostic series (Sec. 3.1: the tearing rate is the
// best-fit slope of a mode's energy over its linear phase).
//
// Once every instance has taken one host-driven step (which sizes its
// buffers), each instance's step is a captured CUDA graph (deposit, solve
// with its loops as conditional nodes, field update, push, re-sort): the
// runner then enqueues all steps of all instances, step by step across the
// instances, each on its instance's stream with an asynchronous copy of the
// solve's outcome, and waits once at the end. No host decision sits between
// two steps, so the GPU holds work of every instance at once.
//
// With shared launches on, one graph per step covers all instances: one
// deposit, one push and one re-sort launch per species over the particles of
// every instance, and each instance's solve as a branch of its own.
//
// Instances that cannot step as graphs (event profiling on, or moves of more
// than one cell per step) are driven by host threads instead: workers take
// instances largest first and run each one through all its steps, so one
// instance's host waits are filled by the others' kernels.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <exception>
#include <new>
#include <thread>
#include <vector>

#include "launch.cuh"
#include "relsim.h"

struct relsim_batch {
    std::vector<relsim_ctx*> ctx;
    int nworkers = 1;
    int device = 0;
    bool shared = false;
    int dep_blocks = 0, push_blocks = 0;
    int last_path = -1;
    int groups = 1;                          // instance groups of the shared launches
    std::vector<relsim_shared*> sbs;         // their graphs, kept while they fit the instances
    std::vector<std::vector<int>> gmem;      // the instances of each group
};

using namespace relsim;

extern "C" {

int relsim_growth_fit(const double* s, int n, double dt, int window, double* rate, int* first)
{
    if (!s || !rate || n < 2 || window < 2 || window > n || !(dt > 0.0) || !std::isfinite(dt))
        return RELSIM_ERR_INVALID_ARG;
    // centred abscissae k - (window-1)/2 make the slope sum(k' y) / sum(k'^2)
    const double kc = 0.5 * (double)(window - 1);
    double sxx = 0.0;
    for (int k = 0; k < window; ++k) sxx += ((double)k - kc) * ((double)k - kc);
    bool found = false;
    double best = 0.0;
    int best_at = 0;
    for (int a = 0; a + window <= n; ++a) {
        double sxy = 0.0;
        bool ok = true;
        for (int k = 0; k < window && ok; ++k) {
            const double v = s[a + k];
            if (!(v > 0.0) || !std::isfinite(v)) ok = false;
            else sxy += ((double)k - kc) * std::log(v);
        }
        if (!ok) continue;
        const double slope = sxy / sxx / dt;
        if (!found || slope > best) {
            best = slope;
            best_at = a;
            found = true;
        }
    }
    if (!found) return RELSIM_ERR_INVALID_ARG;
    *rate = best;
    if (first) *first = best_at;
    return RELSIM_OK;
}

// residual of the dispersion fit for a given b, with A in closed form
static double dispersion_residual(const double* x, const double* r, int n, double b, double* Aout)
{
    double gg = 0.0, gr = 0.0;
    for (int i = 0; i < n; ++i) {
        const double xb = x[i] * b;
        const double g = xb * (1.0 - xb * xb);
        gg += g * g;
        gr += g * r[i];
    }
    const double A = gg > 0.0 ? gr / gg : 0.0;
    double res = 0.0;
    for (int i = 0; i < n; ++i) {
        const double xb = x[i] * b;
        const double d = A * xb * (1.0 - xb * xb) - r[i];
        res += d * d;
    }
    if (Aout) *Aout = A;
    return res;
}

int relsim_dispersion_fit(const double* modes, int nsamples, int nmodes, double dt, int first, int window,
                          double Lx, double a, double* rates, double* A, double* b)
{
    if (!modes || !rates || !A || !b || nsamples < 2 || nmodes < 3 || window < 2 || first < 0 ||
        first > nsamples - window || !(dt > 0.0) || !std::isfinite(dt) || !(Lx > 0.0) || !std::isfinite(Lx) ||
        !(a > 0.0) || !std::isfinite(a))
        return RELSIM_ERR_INVALID_ARG;
    // per mode: least-squares slope of log energy against time, centred
    // abscissae k - (window-1)/2; half of it is the amplitude's rate
    const double kc = 0.5 * (double)(window - 1);
    double sxx = 0.0;
    for (int k = 0; k < window; ++k) sxx += ((double)k - kc) * ((double)k - kc);
    std::vector<double> xs, rs;
    rates[0] = std::nan("");
    for (int m = 1; m < nmodes; ++m) {
        double sxy = 0.0;
        bool ok = true;
        for (int k = 0; k < window && ok; ++k) {
            const double v = modes[(size_t)(first + k) * (size_t)nmodes + (size_t)m];
            if (!(v > 0.0) || !std::isfinite(v)) ok = false;
            else sxy += ((double)k - kc) * std::log(v);
        }
        rates[m] = ok ? 0.5 * sxy / sxx / dt : std::nan("");
        if (ok) {
            xs.push_back(2.0 * M_PI * (double)m * a / Lx);
            rs.push_back(rates[m]);
        }
    }
    const int n = (int)xs.size();
    if (n < 2) return RELSIM_ERR_INVALID_ARG;
    // b on a grid of step 1e-3 over [0.2, 4], then golden section in the
    // cells either side of the best grid point
    const double lo = 0.2, step = 1e-3;
    const int ng = 3801;
    int bi = 0;
    double best = 0.0;
    for (int i = 0; i < ng; ++i) {
        const double r = dispersion_residual(xs.data(), rs.data(), n, lo + step * i, nullptr);
        if (i == 0 || r < best) {
            best = r;
            bi = i;
        }
    }
    double u = lo + step * (bi > 0 ? bi - 1 : 0), v = lo + step * (bi < ng - 1 ? bi + 1 : ng - 1);
    const double gr = 0.5 * (std::sqrt(5.0) - 1.0);
    double p = v - gr * (v - u), q = u + gr * (v - u);
    double fp = dispersion_residual(xs.data(), rs.data(), n, p, nullptr);
    double fq = dispersion_residual(xs.data(), rs.data(), n, q, nullptr);
    for (int it = 0; it < 200 && v - u > 1e-12; ++it) {
        if (fp <= fq) {
            v = q; q = p; fq = fp;
            p = v - gr * (v - u);
            fp = dispersion_residual(xs.data(), rs.data(), n, p, nullptr);
        } else {
            u = p; p = q; fp = fq;
            q = u + gr * (v - u);
            fq = dispersion_residual(xs.data(), rs.data(), n, q, nullptr);
        }
    }
    double bb = 0.5 * (u + v);
    double Af = 0.0;
    const double rb = dispersion_residual(xs.data(), rs.data(), n, bb, &Af);
    if (best < rb) {   // the grid point itself was better (flat residual)
        bb = lo + step * bi;
        dispersion_residual(xs.data(), rs.data(), n, bb, &Af);
    }
    *A = Af;
    *b = bb;
    return RELSIM_OK;
}

int relsim_batch_create(relsim_ctx* const* ctxs, int count, int nworkers, relsim_batch** out)
{
    if (!out) return RELSIM_ERR_INVALID_ARG;
    *out = nullptr;
    if (!ctxs || count < 1 || nworkers < 1 || nworkers > 256) return RELSIM_ERR_INVALID_ARG;
    for (int i = 0; i < count; ++i) {
        if (!ctxs[i]) return RELSIM_ERR_INVALID_ARG;
        for (int j = 0; j < i; ++j)
            if (ctxs[j] == ctxs[i]) return RELSIM_ERR_INVALID_ARG;   // one thread per context
    }
    relsim_batch* b = new (std::nothrow) relsim_batch;
    if (!b) return RELSIM_ERR_OOM;
    try {
        b->ctx.assign(ctxs, ctxs + count);
    } catch (...) {
        delete b;
        return RELSIM_ERR_OOM;
    }
    b->nworkers = std::min(nworkers, count);
    if (cudaGetDevice(&b->device) != cudaSuccess) {
        delete b;
        return RELSIM_ERR_CUDA;
    }
    *out = b;
    return RELSIM_OK;
}

}  // extern "C"

namespace {

// merge one step's solve outcome r into an instance's status: the first
// error sticks; NOT_CONVERGED is kept unless an error follows
void merge_status(int& st, int r)
{
    if (r != RELSIM_OK && (st == RELSIM_OK || st == RELSIM_ERR_NOT_CONVERGED) &&
        !(r == RELSIM_ERR_NOT_CONVERGED && st == RELSIM_ERR_NOT_CONVERGED))
        st = r;
}

// the instances split into g groups of about equal particle count (largest
// first onto the lightest group); a group keeps the instances' order
std::vector<std::vector<int>> shared_groups(const relsim_batch* b, int g)
{
    const int count = (int)b->ctx.size();
    if (g > count) g = count;
    if (g < 1) g = 1;
    std::vector<int> order(count);
    for (int i = 0; i < count; ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(),
                     [&](int x, int y) { return ctx_particles(b->ctx[x]) > ctx_particles(b->ctx[y]); });
    std::vector<int64_t> load(g, 0);
    std::vector<int> owner(count, 0);
    for (int i : order) {
        int best = 0;
        for (int q = 1; q < g; ++q)
            if (load[q] < load[best]) best = q;
        owner[i] = best;
        load[best] += ctx_particles(b->ctx[i]);
    }
    std::vector<std::vector<int>> groups(g);
    for (int i = 0; i < count; ++i) groups[owner[i]].push_back(i);
    return groups;
}

void shared_drop(relsim_batch* b)
{
    for (relsim_shared* sb : b->sbs) shared_destroy(sb);
    b->sbs.clear();
    b->gmem.clear();
}

// steps first .. nsteps-1 of every instance through shared launches, one
// graph per group of instances and step, each group on its own stream (the
// groups' deposits, solves and pushes overlap as single instances' do); -1
// when the instances are not eligible (nothing enqueued)
int run_shared(relsim_batch* b, int nsteps, int first, int component, int nmodes, double* dmodes, size_t per,
               int* status, int* iters)
{
    const int count = (int)b->ctx.size();
    std::vector<std::vector<int>> groups = shared_groups(b, b->groups);
    const int ng = (int)groups.size();
    bool valid = (int)b->sbs.size() == ng && b->gmem == groups;
    std::vector<relsim_ctx*> gc;
    for (int g = 0; g < ng && valid; ++g) {
        gc.clear();
        for (int i : groups[g]) gc.push_back(b->ctx[i]);
        valid = shared_valid(b->sbs[g], gc.data(), (int)gc.size(), b->dep_blocks, b->push_blocks);
    }
    if (!valid) {
        shared_drop(b);
        for (int g = 0; g < ng; ++g) {
            gc.clear();
            for (int i : groups[g]) gc.push_back(b->ctx[i]);
            relsim_shared* sb = nullptr;
            const int made = shared_create(gc.data(), (int)gc.size(), b->dep_blocks, b->push_blocks, &sb);
            if (made != 1) {
                shared_drop(b);
                return made == 0 ? -1 : made;
            }
            b->sbs.push_back(sb);
        }
        b->gmem = groups;
    }
    const size_t hb = ctx_graph_head_bytes();
    const int ns = nsteps - first;
    // heads: group by group, instance by instance, step by step
    std::vector<size_t> off(ng + 1, 0);
    for (int g = 0; g < ng; ++g) off[g + 1] = off[g] + groups[g].size();
    unsigned char* heads = nullptr;
    std::vector<cudaEvent_t> ev(count + ng, nullptr);
    int rc = RELSIM_OK;
    if (cudaMallocHost((void**)&heads, hb * (size_t)count * (size_t)ns) != cudaSuccess) rc = RELSIM_ERR_OOM;
    for (size_t i = 0; i < ev.size() && rc == RELSIM_OK; ++i)
        if (cudaEventCreateWithFlags(&ev[i], cudaEventDisableTiming) != cudaSuccess) rc = RELSIM_ERR_CUDA;
    // a group's stream follows its instances' earlier work; the mode
    // energies of step s run on each instance's stream between the group's
    // steps
    auto join_group = [&](int g) -> int {
        cudaStream_t to = shared_stream(b->sbs[g]);
        for (int i : groups[g])
            if (cudaEventRecord(ev[i], ctx_stream(b->ctx[i])) != cudaSuccess ||
                cudaStreamWaitEvent(to, ev[i], 0) != cudaSuccess)
                return RELSIM_ERR_CUDA;
        return RELSIM_OK;
    };
    for (int g = 0; g < ng && rc == RELSIM_OK; ++g) rc = join_group(g);
    for (int s = first; s < nsteps && rc == RELSIM_OK; ++s)
        for (int g = 0; g < ng && rc == RELSIM_OK; ++g) {
            relsim_shared* sb = b->sbs[g];
            rc = shared_enqueue(sb, heads + hb * (size_t)ns * off[g] + hb * (size_t)(s - first), hb * (size_t)ns);
            if (rc != RELSIM_OK || nmodes == 0) continue;
            if (cudaEventRecord(ev[count + g], shared_stream(sb)) != cudaSuccess) {
                rc = RELSIM_ERR_CUDA;
                break;
            }
            for (int i : groups[g]) {
                relsim_ctx* c = b->ctx[i];
                if (cudaStreamWaitEvent(ctx_stream(c), ev[count + g], 0) != cudaSuccess) {
                    rc = RELSIM_ERR_CUDA;
                    break;
                }
                rc = relsim_field_modes(c, component, nmodes, dmodes + per * (size_t)i + (size_t)(s + 1) * nmodes,
                                        RELSIM_DEVICE);
                if (rc != RELSIM_OK) break;
            }
            if (rc == RELSIM_OK) rc = join_group(g);
        }
    for (relsim_shared* sb : b->sbs)
        if (cudaStreamSynchronize(shared_stream(sb)) != cudaSuccess && rc == RELSIM_OK) rc = RELSIM_ERR_CUDA;
    for (int i = 0; i < count; ++i)
        if (cudaStreamSynchronize(ctx_stream(b->ctx[i])) != cudaSuccess && rc == RELSIM_OK) rc = RELSIM_ERR_CUDA;
    if (rc == RELSIM_OK)
        for (int s = first; s < nsteps; ++s)
            for (int g = 0; g < ng; ++g)
                for (size_t il = 0; il < groups[g].size(); ++il) {
                    const int i = groups[g][il];
                    int it = 0;
                    const unsigned char* h = heads + hb * (size_t)ns * (off[g] + il) + hb * (size_t)(s - first);
                    const int r = shared_outcome(b->sbs[g], (int)il, h, &it, il == 0);
                    if (iters) iters[(size_t)i * nsteps + s] = it;
                    merge_status(status[i], r);
                }
    for (cudaEvent_t e : ev)
        if (e) cudaEventDestroy(e);
    if (heads) cudaFreeHost(heads);
    if (rc != RELSIM_OK) shared_drop(b);
    return rc;
}

}  // namespace

extern "C" {

int relsim_batch_set_shared(relsim_batch* b, int on, int groups, int deposit_blocks, int push_blocks)
{
    if (!b || (on != 0 && on != 1) || groups > 4096 || deposit_blocks > (1 << 20) || push_blocks > (1 << 20))
        return RELSIM_ERR_INVALID_ARG;
    b->shared = on != 0;
    b->groups = groups > 0 ? groups : 1;
    b->dep_blocks = deposit_blocks > 0 ? deposit_blocks : 0;
    b->push_blocks = push_blocks > 0 ? push_blocks : 0;
    if (!b->sbs.empty()) {
        cudaSetDevice(b->device);
        shared_drop(b);
    }
    return RELSIM_OK;
}

int relsim_batch_last_path(const relsim_batch* b) { return b ? b->last_path : -1; }

int relsim_batch_run(relsim_batch* b, int nsteps, int component, int nmodes, double* modes, int* status,
                     int* iters)
{
    if (!b || !status || nsteps < 0 || component < 0 || component > 2 || nmodes < 0)
        return RELSIM_ERR_INVALID_ARG;
    const int count = (int)b->ctx.size();
    if (!modes) nmodes = 0;
    for (int i = 0; i < count; ++i) status[i] = RELSIM_OK;
    if (nsteps == 0) return RELSIM_OK;
    if (cudaSetDevice(b->device) != cudaSuccess) return RELSIM_ERR_CUDA;

    // device slots for the mode energies: (instance, step, mode); one
    // call per context first, on the loaded state, sizes the context's
    // diagnostic buffers before the workers start (no allocation while
    // other instances run)
    double* dmodes = nullptr;
    const size_t per = (size_t)(nsteps + 1) * (size_t)nmodes;
    if (nmodes > 0) {
        if (cudaMalloc((void**)&dmodes, sizeof(double) * per * (size_t)count) != cudaSuccess)
            return RELSIM_ERR_OOM;
        for (int i = 0; i < count; ++i) {
            const int r = relsim_field_modes(b->ctx[i], component, nmodes, dmodes + per * (size_t)i, RELSIM_DEVICE);
            if (r != RELSIM_OK) {
                cudaDeviceSynchronize();
                cudaFree(dmodes);
                return r;
            }
        }
    }

    // the first host-driven step of fresh instances, then the graphs
    std::vector<int> done(count, 0);
    bool graphs = true;
    for (int i = 0; i < count; ++i) {
        relsim_ctx* c = b->ctx[i];
        if (cudaStreamSynchronize(ctx_stream(c)) != cudaSuccess) graphs = false;
        if (!ctx_graph_prepare(c)) {
            const int r = relsim_step(c, nullptr);
            if (r != RELSIM_OK && r != RELSIM_ERR_NOT_CONVERGED) {
                status[i] = r;
                done[i] = nsteps;   // failed: no further steps
                continue;
            }
            if (r == RELSIM_ERR_NOT_CONVERGED) status[i] = r;
            if (iters) iters[(size_t)i * nsteps] = ctx_last_iters(c);
            if (nmodes > 0 &&
                relsim_field_modes(c, component, nmodes, dmodes + per * (size_t)i + (size_t)nmodes, RELSIM_DEVICE) !=
                    RELSIM_OK)
                graphs = false;
            done[i] = 1;
            if (nsteps > 1 && !ctx_graph_prepare(c)) graphs = false;
        }
    }
    b->last_path = 0;
    bool same = true;
    for (int i = 1; i < count; ++i) same = same && done[i] == done[0] && status[i] == RELSIM_OK;
    if (graphs && b->shared && same && status[0] == RELSIM_OK && done[0] < nsteps) {
        const int rc = run_shared(b, nsteps, done[0], component, nmodes, dmodes, per, status, iters);
        if (rc < 0) {   // not eligible: per-instance graphs
        } else if (rc != RELSIM_OK) {
            cudaDeviceSynchronize();
            cudaFree(dmodes);
            return rc;
        } else {
            for (int i = 0; i < count; ++i) done[i] = nsteps;
            graphs = false;
            b->last_path = 2;
        }
    }
    if (graphs) {
        b->last_path = 1;
        const size_t hb = ctx_graph_head_bytes();
        unsigned char* heads = nullptr;
        if (cudaMallocHost((void**)&heads, hb * (size_t)count * (size_t)nsteps) != cudaSuccess) {
            cudaGetLastError();
            graphs = false;
        } else {
            int rc = RELSIM_OK;
            for (int s = 0; s < nsteps && rc == RELSIM_OK; ++s)
                for (int i = 0; i < count && rc == RELSIM_OK; ++i) {
                    if (s < done[i]) continue;
                    relsim_ctx* c = b->ctx[i];
                    rc = ctx_graph_enqueue(c, heads + hb * ((size_t)i * nsteps + s));
                    if (rc == RELSIM_OK && nmodes > 0)
                        rc = relsim_field_modes(c, component, nmodes,
                                                dmodes + per * (size_t)i + (size_t)(s + 1) * nmodes, RELSIM_DEVICE);
                }
            for (int i = 0; i < count; ++i)
                if (cudaStreamSynchronize(ctx_stream(b->ctx[i])) != cudaSuccess && rc == RELSIM_OK) rc = RELSIM_ERR_CUDA;
            if (rc == RELSIM_OK)
                for (int i = 0; i < count; ++i)
                    for (int s = done[i]; s < nsteps; ++s) {
                        int it = 0;
                        const int r = ctx_graph_outcome(b->ctx[i], heads + hb * ((size_t)i * nsteps + s), &it);
                        if (iters) iters[(size_t)i * nsteps + s] = it;
                        merge_status(status[i], r);
                    }
            cudaFreeHost(heads);
            if (rc != RELSIM_OK) {
                cudaDeviceSynchronize();
                cudaFree(dmodes);
                return rc;
            }
            for (int i = 0; i < count; ++i) done[i] = nsteps;
        }
    }

    // the rest host-driven: largest instances first
    std::vector<int> order(count);
    std::vector<int64_t> size(count);
    for (int i = 0; i < count; ++i) {
        order[i] = i;
        size[i] = ctx_particles(b->ctx[i]);
    }
    std::stable_sort(order.begin(), order.end(), [&](int a, int c) { return size[a] > size[c]; });

    std::atomic<int> next{0};
    auto worker = [&]() {
        if (cudaSetDevice(b->device) != cudaSuccess) {
            for (int k = next.fetch_add(count); k < count; ++k) status[order[k]] = RELSIM_ERR_CUDA;
            return;
        }
        for (int k = next.fetch_add(1); k < count; k = next.fetch_add(1)) {
            const int i = order[k];
            relsim_ctx* c = b->ctx[i];
            if (done[i] >= nsteps) continue;
            int st = status[i];
            for (int s = done[i]; s < nsteps; ++s) {
                const int r = relsim_step(c, nullptr);
                if (r != RELSIM_OK && r != RELSIM_ERR_NOT_CONVERGED) {
                    st = r;
                    break;
                }
                if (r == RELSIM_ERR_NOT_CONVERGED && st == RELSIM_OK) st = r;
                if (iters) iters[(size_t)i * nsteps + s] = ctx_last_iters(c);
                if (nmodes > 0) {
                    const int q = relsim_field_modes(c, component, nmodes,
                                                     dmodes + per * (size_t)i + (size_t)(s + 1) * nmodes,
                                                     RELSIM_DEVICE);
                    if (q != RELSIM_OK) {
                        st = q;
                        break;
                    }
                }
            }
            if (cudaStreamSynchronize(ctx_stream(c)) != cudaSuccess && st == RELSIM_OK) st = RELSIM_ERR_CUDA;
            status[i] = st;
        }
    };

    int rc = RELSIM_OK;
    std::vector<std::thread> pool;
    try {
        pool.reserve((size_t)b->nworkers);
        for (int t = 0; t < b->nworkers; ++t) pool.emplace_back(worker);
    } catch (...) {
        rc = RELSIM_ERR_OOM;   // fewer threads started: the ones running finish the queue
        if (pool.empty()) worker();
    }
    for (std::thread& t : pool) t.join();

    if (nmodes > 0) {
        cudaError_t e = cudaDeviceSynchronize();
        std::vector<double> h;
        try {
            h.resize(per * (size_t)count);
        } catch (...) {
            cudaFree(dmodes);
            return RELSIM_ERR_OOM;
        }
        if (e == cudaSuccess) e = cudaMemcpy(h.data(), dmodes, sizeof(double) * h.size(), cudaMemcpyDeviceToHost);
        cudaFree(dmodes);
        if (e != cudaSuccess) return RELSIM_ERR_CUDA;
        for (int i = 0; i < count; ++i)
            std::copy(h.begin() + (ptrdiff_t)(per * (size_t)i + (size_t)nmodes),
                      h.begin() + (ptrdiff_t)(per * (size_t)(i + 1)),
                      modes + (size_t)i * nsteps * nmodes);
    }
    if (rc != RELSIM_OK) return rc;
    for (int i = 0; i < count; ++i)
        if (status[i] != RELSIM_OK) return status[i];
    return RELSIM_OK;
}

void relsim_batch_destroy(relsim_batch* b)
{
    if (!b) return;
    if (!b->sbs.empty()) {
        cudaSetDevice(b->device);
        shared_drop(b);
    }
    delete b;
}

}  // extern "C"
