// api.cu -- the C ABI of libhfv (declared in include/hfv.h): argument checks,
// object lifetime, and dispatch to the setup and hot-path launchers.
#include <cuda_runtime.h>

#include <atomic>
#include <chrono>
#include <algorithm>
#include <cstring>
#include <memory>
#include <new>
#include <string>
#include <vector>

#include "hfv_internal.h"

namespace hfv {

static thread_local std::string g_last_error;

void set_error(const std::string& msg) { g_last_error = msg; }

static std::atomic<int64_t> g_launches{0};
void note_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

bool residual_supported(int d, int r, int fam);

}  // namespace hfv

using namespace hfv;

#define API_CUDA(x)                                                                          \
    do {                                                                                     \
        cudaError_t e_ = (x);                                                                \
        if (e_ != cudaSuccess) {                                                             \
            set_error(std::string("CUDA: ") + cudaGetErrorString(e_) + " at " #x);           \
            return HFV_ERR_CUDA;                                                             \
        }                                                                                    \
    } while (0)

extern "C" const char* hfv_last_error(void) { return g_last_error.c_str(); }

extern "C" int hfv_default_params(hfv_scheme_params* p)
{
    if (!p) { set_error("hfv_default_params: NULL"); return HFV_ERR_ARG; }
    std::memset(p, 0, sizeof *p);
    p->order = 3;
    p->flux = HFV_HLLC;
    p->scheme = HFV_HYBRID;
    p->nad_vars = 3;
    p->precision = HFV_FP64;
    p->gamma = 1.4;
    p->alpha_m = 5e-3;
    p->beta_m = 0.5;
    p->alpha_w = 0.0;
    p->beta_w = 0.0;
    p->kappa = 1.0;
    p->n_exp = 1.0;
    p->lambda1_prime = 1e3;
    p->cweno_eps = 1e-3;
    p->cweno_b = 4.0;
    p->time_scheme = HFV_SSPRK3;
    p->limiter = HFV_BARTH_JESPERSEN;
    p->venkat_k = 5.0;
    p->harten_theta = 0.9;
    p->harten_eps = 1e-14;
    p->stencil_factor = 2.0;
    p->mu0 = 0.0;
    p->t0 = 1.0;
    p->sutherland_s = 110.4 / 288.15;
    p->prandtl = 0.72;
    p->visc_alpha = 4.0 / 3.0;
    p->step_chain = 0;
    return HFV_OK;
}

static void timer_free(KernelTimer& t)
{
    for (void* e : t.ev) cudaEventDestroy((cudaEvent_t)e);
    t.ev.clear();
    t.kid.clear();
    t.used = 0;
    t.on = false;
}

extern "C" void hfv_scheme_destroy(hfv_scheme* s)
{
    if (!s) return;
    timer_free(s->timer);
    if (s->side) cudaStreamDestroy((cudaStream_t)s->side);
    if (s->ev_fork) cudaEventDestroy((cudaEvent_t)s->ev_fork);
    if (s->ev_join) cudaEventDestroy((cudaEvent_t)s->ev_join);
    adjoint_free(s);
    if (s->arena) cudaFree(s->arena);
    delete s;
}

extern "C" int hfv_scheme_create(hfv_mesh* mesh, const hfv_scheme_params* p, void* stream, hfv_scheme** out)
{
    if (!mesh || !p || !out) { set_error("hfv_scheme_create: NULL argument"); return HFV_ERR_ARG; }
    *out = nullptr;
    const int r = p->order - 1;
    const int fam = element_family(mesh);
    if (r < 1 || !residual_supported(mesh->dim, r, fam)) {
        set_error("hfv_scheme_create: order " + std::to_string(p->order) + " is not built for dim " +
                  std::to_string(mesh->dim) + (fam == 1 ? " tetrahedra" : fam == 2 ? " mixed elements" : ""));
        return HFV_ERR_ARG;
    }
    if (p->stencil_factor != 2.0) { set_error("hfv_scheme_create: only stencil_factor = 2 (M = 2K) is built"); return HFV_ERR_ARG; }
    if (p->flux < HFV_RUSANOV || p->flux > HFV_HLL || p->scheme < HFV_HYBRID || p->scheme > HFV_PURE_MUSCL ||
        (p->precision != HFV_FP64 && p->precision != HFV_FP32) || (p->nad_vars & ~7) ||
        (p->time_scheme != HFV_SSPRK3 && p->time_scheme != HFV_SSPRK54) ||
        (p->limiter != HFV_BARTH_JESPERSEN && p->limiter != HFV_VENKATAKRISHNAN) || !(p->venkat_k >= 0.0) ||
        (p->cweno_vars != HFV_CONSERVED && p->cweno_vars != HFV_CHARACTERISTIC) ||
        !(p->gamma > 1.0) || !(p->lambda1_prime > 1.0) || !(p->harten_theta > 0.0) || !(p->cweno_eps > 0.0) ||
        !(p->mu0 >= 0.0) || !(p->t0 > 0.0) || !(p->sutherland_s >= 0.0) || !(p->prandtl > 0.0) ||
        !(p->visc_alpha >= 0.0) || (p->step_chain != 0 && p->step_chain != 1)) {
        set_error("hfv_scheme_create: parameter out of range");
        return HFV_ERR_ARG;
    }
    hfv_scheme* s = nullptr;
    try {
        s = new hfv_scheme();
    } catch (const std::bad_alloc&) {
        set_error("hfv_scheme_create: out of host memory");
        return HFV_ERR_OOM;
    }
    s->mesh = mesh;
    s->p = *p;
    int rc;
    const auto t0 = std::chrono::steady_clock::now();
    try {
        rc = build_stencils(s);
    } catch (const std::bad_alloc&) {
        rc = HFV_ERR_OOM;
        set_error("hfv_scheme_create: out of host memory");
    }
    const auto t1 = std::chrono::steady_clock::now();
    if (rc == HFV_OK) rc = build_operators(s, stream);
    const auto t2 = std::chrono::steady_clock::now();
    s->setup_ms[0] = std::chrono::duration<double, std::milli>(t1 - t0).count();
    s->setup_ms[1] = std::chrono::duration<double, std::milli>(t2 - t1).count();
    if (rc == HFV_OK) {
        cudaStream_t side;
        cudaEvent_t e1, e2;
        if (cudaStreamCreateWithFlags(&side, cudaStreamNonBlocking) != cudaSuccess) {
            rc = HFV_ERR_CUDA;
        } else {
            s->side = side;
            if (cudaEventCreateWithFlags(&e1, cudaEventDisableTiming) != cudaSuccess) rc = HFV_ERR_CUDA;
            else s->ev_fork = e1;
            if (rc == HFV_OK && cudaEventCreateWithFlags(&e2, cudaEventDisableTiming) != cudaSuccess) rc = HFV_ERR_CUDA;
            else if (rc == HFV_OK) s->ev_join = e2;
        }
        if (rc != HFV_OK) set_error("hfv_scheme_create: stream or event creation failed");
    }
    if (rc != HFV_OK) {
        hfv_scheme_destroy(s);
        return rc;
    }
    *out = s;
    return HFV_OK;
}

extern "C" int hfv_scheme_info(const hfv_scheme* s, int64_t* info)
{
    if (!s || !info) { set_error("hfv_scheme_info: NULL argument"); return HFV_ERR_ARG; }
    info[0] = s->N; info[1] = s->M; info[2] = s->Md; info[3] = s->nq; info[4] = s->nfp; info[5] = s->nv;
    info[6] = s->qtot; info[7] = s->p.precision;
    return HFV_OK;
}

extern "C" int hfv_scheme_setup_ms(const hfv_scheme* s, double* ms)
{
    if (!s || !ms) { set_error("hfv_scheme_setup_ms: NULL argument"); return HFV_ERR_ARG; }
    ms[0] = s->setup_ms[0];
    ms[1] = s->setup_ms[1];
    return HFV_OK;
}

extern "C" int hfv_scheme_set_kind(hfv_scheme* s, int scheme)
{
    if (!s || scheme < HFV_HYBRID || scheme > HFV_PURE_MUSCL) { set_error("hfv_scheme_set_kind: bad argument"); return HFV_ERR_ARG; }
    s->p.scheme = scheme;
    s->chain_ok = false;
    return HFV_OK;
}

extern "C" int hfv_scheme_device_bytes(const hfv_scheme* s, int64_t* bytes)
{
    if (!s || !bytes) { set_error("hfv_scheme_device_bytes: NULL argument"); return HFV_ERR_ARG; }
    *bytes = (int64_t)s->arena_bytes;
    return HFV_OK;
}

extern "C" int hfv_get_stencils(const hfv_scheme* s, int32_t* central, int32_t* dir)
{
    if (!s || !central) { set_error("hfv_get_stencils: NULL argument"); return HFV_ERR_ARG; }
    std::memcpy(central, s->sten.data(), s->sten.size() * sizeof(int32_t));
    if (dir) {
        const int64_t nc = s->mesh->nc;
        for (int64_t c = 0; c < nc; ++c)
            for (int f = 0; f < kMaxFaces; ++f) {
                int n = f < type_nfaces(s->mesh->type[c]) ? s->nd[c * kMaxFaces + f] : 0;
                for (int k = 0; k < s->Md; ++k)
                    dir[(c * kMaxFaces + f) * s->Md + k] = k < n ? s->dir[(c * kMaxFaces + f) * s->Md + k] : -1;
            }
    }
    return HFV_OK;
}

extern "C" int hfv_stencils_host(const hfv_mesh* mesh, int order, int32_t* sizes, int32_t* central, int32_t* dir)
{
    if (!mesh || !sizes) { set_error("hfv_stencils_host: NULL argument"); return HFV_ERR_ARG; }
    if (order < 2 || order > 7) { set_error("hfv_stencils_host: order must be 2..7"); return HFV_ERR_ARG; }
    // the builder of hfv_scheme_create on a scheme that never reaches the
    // device: only its host fields are filled, and its destructor frees
    // host memory only
    std::unique_ptr<hfv_scheme> s;
    try {
        s.reset(new hfv_scheme());
        s->mesh = const_cast<hfv_mesh*>(mesh);
        hfv_default_params(&s->p);
        s->p.order = order;
        const int rc = build_stencils(s.get());
        if (rc != HFV_OK) return rc;
    } catch (const std::bad_alloc&) {
        set_error("hfv_stencils_host: out of host memory");
        return HFV_ERR_OOM;
    }
    sizes[0] = s->M;
    sizes[1] = s->Md;
    return central ? hfv_get_stencils(s.get(), central, dir) : HFV_OK;
}

extern "C" int hfv_residual(hfv_scheme* s, const void* U, void* R, const uint8_t* forced, uint8_t* cls_out, void* stream)
{
    if (!s || !U || !R) { set_error("hfv_residual: NULL argument"); return HFV_ERR_ARG; }
    return launch_residual(s, U, R, forced, cls_out, stream);
}

extern "C" int hfv_compute_dt(hfv_scheme* s, const double* U, double cfl, double* dt_dev, void* stream)
{
    if (!s || !U || !dt_dev || !(cfl > 0)) { set_error("hfv_compute_dt: bad argument"); return HFV_ERR_ARG; }
    return launch_dt(s, U, cfl, dt_dev, stream);
}

extern "C" int hfv_step(hfv_scheme* s, double* U, double cfl, double dt, double* dt_used, void* stream)
{
    if (!s || !U || (!(dt > 0) && !(cfl > 0))) { set_error("hfv_step: bad argument"); return HFV_ERR_ARG; }
    int rc = launch_step(s, U, cfl, dt, stream);
    if (rc != HFV_OK) return rc;
    if (dt_used) {
        API_CUDA(cudaMemcpyAsync(dt_used, s->a.dt, s->nseg * sizeof(double), cudaMemcpyDeviceToHost,
                                 (cudaStream_t)stream));
        API_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
    }
    return HFV_OK;
}

extern "C" int hfv_residual_vjp(hfv_scheme* s, const double* U, const uint8_t* cls, const double* lam, double* g,
                                void* stream)
{
    if (!s || !U || !cls || !lam || !g) { set_error("hfv_residual_vjp: NULL argument"); return HFV_ERR_ARG; }
    if (s->p.precision != HFV_FP64) { set_error("hfv_residual_vjp: FP64 schemes only"); return HFV_ERR_ARG; }
    if (s->p.cweno_vars != HFV_CONSERVED) {
        set_error("hfv_residual_vjp: CWENOZ in conserved variables only");
        return HFV_ERR_ARG;
    }
    if (s->p.mu0 > 0.0) {
        set_error("hfv_residual_vjp: the Euler residual only (mu0 = 0)");
        return HFV_ERR_ARG;
    }
    return launch_vjp(s, U, cls, lam, g, stream);
}

static int vjp_scheme_ok(const hfv_scheme* s, const char* who)
{
    if (s->p.precision != HFV_FP64 || s->p.cweno_vars != HFV_CONSERVED || s->p.mu0 > 0.0) {
        set_error(std::string(who) + ": FP64, conserved-variable, Euler (mu0 = 0) schemes only");
        return HFV_ERR_ARG;
    }
    return HFV_OK;
}

extern "C" int hfv_step_classes(hfv_scheme* s, const double* U, double dt, uint8_t* cls, int forced, double* U_out,
                                void* stream)
{
    if (!s || !U || !cls || !U_out || !(dt > 0.0) || U == U_out) { set_error("hfv_step_classes: bad argument"); return HFV_ERR_ARG; }
    int rc = vjp_scheme_ok(s, "hfv_step_classes");
    return rc != HFV_OK ? rc : launch_step_classes(s, U, dt, cls, forced, U_out, stream);
}

extern "C" int hfv_step_vjp(hfv_scheme* s, const double* U, const uint8_t* cls, double dt, double* lam, void* stream)
{
    if (!s || !U || !cls || !lam || !(dt > 0.0) || U == lam) { set_error("hfv_step_vjp: bad argument"); return HFV_ERR_ARG; }
    int rc = vjp_scheme_ok(s, "hfv_step_vjp");
    return rc != HFV_OK ? rc : launch_step_vjp(s, U, cls, dt, lam, stream);
}

extern "C" int hfv_autotune(hfv_scheme* s, const void* U, int reps, void* stream, int* shape)
{
    if (!s || !U || reps <= 0) { set_error("hfv_autotune: bad argument"); return HFV_ERR_ARG; }
    cudaStream_t st = (cudaStream_t)stream;
    cudaEvent_t e0, e1;
    API_CUDA(cudaEventCreate(&e0));
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        set_error("hfv_autotune: event creation failed");
        return HFV_ERR_CUDA;
    }
    int rc = HFV_OK;
    // time `reps` residuals of U with the scheme's current shape (after one untimed)
    auto measure = [&](float* ms) -> int {
        int r = launch_residual(s, U, s->a.Rs, nullptr, nullptr, st);
        if (r != HFV_OK) return r;
        if (cudaEventRecord(e0, st) != cudaSuccess) return HFV_ERR_CUDA;
        for (int k = 0; k < reps && r == HFV_OK; ++k) r = launch_residual(s, U, s->a.Rs, nullptr, nullptr, st);
        if (r != HFV_OK) return r;
        if (cudaEventRecord(e1, st) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
            cudaEventElapsedTime(ms, e0, e1) != cudaSuccess)
            return HFV_ERR_CUDA;
        return HFV_OK;
    };
    // the best of two timings: a candidate is not judged on one noisy burst
    auto measure2 = [&](float* ms) -> int {
        float a = 0.0f, b = 0.0f;
        int r = measure(&a);
        if (r == HFV_OK) r = measure(&b);
        *ms = a < b ? a : b;
        return r;
    };
    // coordinate descent over the knobs, each from its current value; a
    // candidate replaces the current value only when 2 % faster
    auto tune = [&](int* knob, const int* cand, int n) -> int {
        int best = *knob;
        float tbest = 0.0f;
        int r = measure2(&tbest);
        for (int i = 0; i < n && r == HFV_OK; ++i) {
            if (cand[i] == best) continue;
            const int keep = *knob;
            *knob = cand[i];
            float t = 0.0f;
            r = measure2(&t);
            if (r == HFV_OK && t < 0.98f * tbest) { tbest = t; best = cand[i]; }
            else *knob = keep;
        }
        *knob = best;
        return r;
    };
    auto sync = [&]() -> int {
        const cudaError_t e = cudaStreamSynchronize(st);
        if (e == cudaSuccess) return HFV_OK;
        set_error(std::string("hfv_autotune: ") + cudaGetErrorString(e));
        return HFV_ERR_CUDA;
    };
    if (rc == HFV_OK) rc = launch_residual(s, U, s->a.Rs, nullptr, nullptr, st);   // fills sms and the occupancy bound
    if (rc == HFV_OK) rc = sync();
    if (rc == HFV_OK && s->linear_tiles > 1) {
        // the candidate kernel's tile shape first, each at its full occupancy
        static const int tiles[] = {0, 1};
        const int keep = s->tune_linear_per_sm;
        s->tune_linear_per_sm = 0;
        rc = tune(&s->tune_linear_tile, tiles, 2);
        if (rc == HFV_OK) rc = launch_residual(s, U, s->a.Rs, nullptr, nullptr, st);   // the chosen shape's bound
        if (rc == HFV_OK) rc = sync();
        if (rc != HFV_OK) s->tune_linear_per_sm = keep;
    }
    if (rc == HFV_OK) {
        int per[8], n = 0;
        for (int k = 1; k <= s->linear_per_sm_max && n < 8; ++k) per[n++] = k;
        if (s->tune_linear_per_sm <= 0) s->tune_linear_per_sm = s->linear_per_sm_max;
        rc = tune(&s->tune_linear_per_sm, per, n);
    }
    static const int nl[] = {2, 4, 8, 16, 32};
    static const int pct[] = {50, 67, 75, 85, 95};
    if (rc == HFV_OK) rc = tune(&s->tune_nl_per_sm, nl, 5);
    if (rc == HFV_OK) rc = tune(&s->tune_nl_cweno_pct, pct, 5);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc != HFV_OK) return rc;
    if (shape) {
        shape[0] = s->tune_linear_per_sm;
        shape[1] = s->tune_nl_per_sm;
        shape[2] = s->tune_nl_cweno_pct;
        shape[3] = s->tune_linear_tile;
    }
    return HFV_OK;
}

extern "C" int hfv_scheme_set_shape(hfv_scheme* s, const int* shape)
{
    if (!s || !shape || shape[0] < 0 || shape[0] > 64 || shape[1] < 1 || shape[1] > 64 || shape[2] < 1 ||
        shape[2] > 99 || (shape[3] != 0 && shape[3] != 1)) {
        set_error("hfv_scheme_set_shape: NULL argument or a value out of range");
        return HFV_ERR_ARG;
    }
    s->tune_linear_per_sm = shape[0];
    s->tune_nl_per_sm = shape[1];
    s->tune_nl_cweno_pct = shape[2];
    s->tune_linear_tile = shape[3];
    return HFV_OK;
}

extern "C" int hfv_step_many(hfv_scheme* const* schemes, double* const* U, int n, double cfl, double dt, void* stream)
{
    if (!schemes || !U || n <= 0 || (!(dt > 0) && !(cfl > 0))) {
        set_error("hfv_step_many: bad argument");
        return HFV_ERR_ARG;
    }
    for (int k = 0; k < n; ++k) {
        if (!schemes[k] || !U[k]) { set_error("hfv_step_many: NULL scheme or state"); return HFV_ERR_ARG; }
        // each scheme's fork / join events and scratch serve one step at a time
        for (int j = 0; j < k; ++j)
            if (schemes[j] == schemes[k]) { set_error("hfv_step_many: a scheme is listed twice"); return HFV_ERR_ARG; }
    }
    // fork: every scheme's side stream waits for the caller's stream; each
    // step runs on its own side stream; join: the caller's stream waits for
    // all of them.  Under stream capture this records one graph with a
    // branch per scheme.  A failure still joins the branches already forked.
    cudaStream_t st = (cudaStream_t)stream;
    int rc = HFV_OK, forked = 0;
    for (int k = 0; k < n && rc == HFV_OK; ++k) {
        hfv_scheme* s = schemes[k];
        cudaError_t e = cudaEventRecord((cudaEvent_t)s->ev_fork, st);
        if (e == cudaSuccess) e = cudaStreamWaitEvent((cudaStream_t)s->side, (cudaEvent_t)s->ev_fork, 0);
        if (e != cudaSuccess) {
            set_error(std::string("hfv_step_many: ") + cudaGetErrorString(e));
            rc = HFV_ERR_CUDA;
            break;
        }
        ++forked;
        rc = launch_step(s, U[k], cfl, dt, s->side);
        e = cudaEventRecord((cudaEvent_t)s->ev_join, (cudaStream_t)s->side);
        if (rc == HFV_OK && e != cudaSuccess) {
            set_error(std::string("hfv_step_many: ") + cudaGetErrorString(e));
            rc = HFV_ERR_CUDA;
        }
    }
    for (int k = 0; k < forked; ++k) {
        const cudaError_t e = cudaStreamWaitEvent(st, (cudaEvent_t)schemes[k]->ev_join, 0);
        if (e != cudaSuccess && rc == HFV_OK) {
            set_error(std::string("hfv_step_many: ") + cudaGetErrorString(e));
            rc = HFV_ERR_CUDA;
        }
    }
    return rc;
}

extern "C" int hfv_advance_host(hfv_scheme* s, double* U_host, int n_steps, double cfl, double dt, void* stream)
{
    if (!s || !U_host || n_steps < 0) { set_error("hfv_advance_host: bad argument"); return HFV_ERR_ARG; }
    cudaStream_t st = (cudaStream_t)stream;
    const size_t bytes = (size_t)s->nv * s->mesh->nc * sizeof(double);
    double* work = s->a.Uio;   // device state owned by the scheme: no allocation here
    s->chain_ok = false;       // new contents from the host: a chain starts afresh
    API_CUDA(cudaMemcpyAsync(work, U_host, bytes, cudaMemcpyHostToDevice, st));
    int rc = HFV_OK;
    for (int k = 0; k < n_steps && rc == HFV_OK; ++k) rc = launch_step(s, work, cfl, dt, stream);
    if (rc == HFV_OK) {
        API_CUDA(cudaMemcpyAsync(U_host, work, bytes, cudaMemcpyDeviceToHost, st));
        API_CUDA(cudaStreamSynchronize(st));
    }
    return rc;
}

extern "C" int hfv_get_queues(const hfv_scheme* s, int32_t* counts, int32_t* queues)
{
    if (!s || !counts) { set_error("hfv_get_queues: NULL argument"); return HFV_ERR_ARG; }
    API_CUDA(cudaDeviceSynchronize());
    API_CUDA(cudaMemcpy(counts, s->a.counts, 2 * sizeof(int32_t), cudaMemcpyDeviceToHost));
    const int64_t nc = s->mesh->nc;
    if (counts[0] < 0 || counts[1] < 0 || counts[0] > nc || counts[1] > nc) {
        set_error("hfv_get_queues: queue lengths outside 0..n_cells on the device");
        return HFV_ERR_CUDA;
    }
    if (queues) {
        // the device queues hold each block's cells in ascending order, the
        // blocks in the order of their range reservations: sort the copies
        API_CUDA(cudaMemcpy(queues, s->a.queue, 2 * nc * sizeof(int32_t), cudaMemcpyDeviceToHost));
        for (int q = 0; q < 2; ++q) std::sort(queues + q * nc, queues + q * nc + counts[q]);
    }
    return HFV_OK;
}

extern "C" int hfv_debug_wait(hfv_scheme* s, int64_t consumer_wait_ns, int withhold_copies)
{
    if (!s || consumer_wait_ns < 0 || consumer_wait_ns > 2000000000ll) {
        set_error("hfv_debug_wait: NULL scheme or a limit outside 0..2e9 ns");
        return HFV_ERR_ARG;
    }
    s->wait_ns = consumer_wait_ns > 0 ? (uint64_t)consumer_wait_ns : 2000000000ull;
    s->withhold_copies = withhold_copies != 0;
    return HFV_OK;
}

extern "C" int hfv_status(hfv_scheme* s, int* flags, int reset)
{
    if (!s || !flags) { set_error("hfv_status: NULL argument"); return HFV_ERR_ARG; }
    API_CUDA(cudaDeviceSynchronize());
    API_CUDA(cudaMemcpy(flags, s->a.status, sizeof(int), cudaMemcpyDeviceToHost));
    if (reset) API_CUDA(cudaMemset(s->a.status, 0, sizeof(int)));
    if (*flags & 4) {
        set_error("hfv_status: a bounded device wait gave up");
        return HFV_ERR_TIMEOUT;
    }
    return (*flags & 1) ? HFV_ERR_NONPHYSICAL : HFV_OK;
}

extern "C" int hfv_kernel_timer(hfv_scheme* s, int enable)
{
    if (!s) { set_error("hfv_kernel_timer: NULL scheme"); return HFV_ERR_ARG; }
    API_CUDA(cudaDeviceSynchronize());
    KernelTimer& t = s->timer;
    if (!enable) { timer_free(t); return HFV_OK; }
    if (t.ev.empty()) {
        t.ev.resize(1024, nullptr);
        t.kid.assign(512, 0);
        for (auto& e : t.ev) {
            cudaEvent_t ev;
            const cudaError_t err = cudaEventCreate(&ev);
            if (err != cudaSuccess) {
                t.ev.erase(std::remove(t.ev.begin(), t.ev.end(), nullptr), t.ev.end());
                timer_free(t);   // no half-built timer survives a failure
                set_error(std::string("hfv_kernel_timer: ") + cudaGetErrorString(err));
                return HFV_ERR_CUDA;
            }
            e = ev;
        }
    }
    t.used = 0;
    t.on = true;
    return HFV_OK;
}

extern "C" int hfv_kernel_times(hfv_scheme* s, double* ms, int64_t* launches, int reset)
{
    if (!s || !ms || !launches) { set_error("hfv_kernel_times: NULL argument"); return HFV_ERR_ARG; }
    KernelTimer& t = s->timer;
    for (int i = 0; i < t.used; ++i) {
        API_CUDA(cudaEventSynchronize((cudaEvent_t)t.ev[2 * i + 1]));
        float f = 0.0f;
        API_CUDA(cudaEventElapsedTime(&f, (cudaEvent_t)t.ev[2 * i], (cudaEvent_t)t.ev[2 * i + 1]));
        t.ms[t.kid[i]] += f;
        t.n[t.kid[i]] += 1;
    }
    t.used = 0;
    for (int k = 0; k < 16; ++k) { ms[k] = t.ms[k]; launches[k] = t.n[k]; }
    if (reset)
        for (int k = 0; k < 16; ++k) { t.ms[k] = 0.0; t.n[k] = 0; }
    return HFV_OK;
}

extern "C" int hfv_launch_count(int64_t* count)
{
    if (!count) { set_error("hfv_launch_count: NULL"); return HFV_ERR_ARG; }
    *count = g_launches.load();
    return HFV_OK;
}
