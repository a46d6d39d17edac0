// Host runtime behind the C ABI of include/lmreg.h: argument validation,
// context scratch, the ordering of the kernels of one LM iteration (with
// its rejected retries unrolled so no host round trip is needed), CUDA
// graph replay of iterations, the coarse-to-fine schedule, checkpoints.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <vector>

#include <cstdlib>
#include <mutex>

#include "lm_fused.cuh"
#include "lm_kernels.cuh"
#include "lm_pyramid.cuh"

using namespace lmk;

namespace {

thread_local char g_err[512] = "";

int fail(int code, const char* fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
    return code;
}

#define LM_CK(call)                                                        \
    do {                                                                   \
        cudaError_t e_ = (call);                                           \
        if (e_ != cudaSuccess)                                             \
            return fail(LM_ECUDA, "%s failed: %s", #call,                  \
                        cudaGetErrorString(e_));                           \
    } while (0)

}  // namespace

void lmk::set_last_error(const char* msg) {
    snprintf(g_err, sizeof(g_err), "%s", msg);
}

namespace {

bool is_device_ptr(const void* p) {
    if (!p) return false;
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

Taps make_taps(double sigma) {
    Taps t;
    memset(&t, 0, sizeof(t));
    if (!(sigma > 0)) {
        t.R = 0;
        t.t[0] = 1.f;
        return t;
    }
    int R = (int)std::ceil(3.0 * sigma);
    double w[2 * MAX_R + 1], s = 0;
    for (int j = -R; j <= R; ++j) {
        w[j + R] = std::exp(-(double)j * j / (2.0 * sigma * sigma));
        s += w[j + R];
    }
    t.R = R;
    for (int j = 0; j <= 2 * R; ++j) t.t[j] = (float)(w[j] / s);
    return t;
}

int check_params(const lm_params* p) {
    if (!(p->win >= 3 && p->win <= 9 && (p->win & 1)))
        return fail(LM_EINVAL, "win must be odd in [3, 9], got %d", p->win);
    if (!(p->eps_nr >= 0) || !(p->eps_dr > 0) || !std::isfinite(p->eps_nr) ||
        !std::isfinite(p->eps_dr))
        return fail(LM_EINVAL, "eps_nr must be >= 0 and eps_dr > 0");
    if (!(p->sigma_grad >= 0 && p->sigma_grad <= 2) ||
        !(p->sigma_warp >= 0 && p->sigma_warp <= 2))
        return fail(LM_EINVAL, "sigma_grad / sigma_warp must be in [0, 2]");
    if (!(p->step > 0) || !std::isfinite(p->step))
        return fail(LM_EINVAL, "step must be finite and > 0");
    if (!(p->lambda0 > 0) || !std::isfinite(p->lambda0))
        return fail(LM_EINVAL, "lambda0 must be finite and > 0");
    if (!(p->mu_inc > 1) || !std::isfinite(p->mu_inc))
        return fail(LM_EINVAL, "mu_inc must be finite and > 1");
    if (!(p->mu_dec > 0 && p->mu_dec < 1))
        return fail(LM_EINVAL, "mu_dec must be in (0, 1)");
    if (!(p->lambda_max >= p->lambda0))
        return fail(LM_EINVAL, "lambda_max must be >= lambda0");
    if (p->reject != 0 && p->reject != 1)
        return fail(LM_EINVAL, "reject must be 0 or 1");
    if (!(p->tau >= 0) || !std::isfinite(p->tau))
        return fail(LM_EINVAL, "tau must be finite and >= 0");
    if (p->max_retries < 0 || p->max_retries > 32)
        return fail(LM_EINVAL, "max_retries must be in [0, 32]");
    return LM_OK;
}

// Shape and dtype checks (host only, no CUDA call).
int check_volume(const lm_volume* v, const char* name) {
    if (!v) return fail(LM_EINVAL, "%s is NULL", name);
    if (v->D < 1 || v->H < 1 || v->W < 1)
        return fail(LM_EINVAL, "%s has a non-positive dimension", name);
    if ((long long)v->D * v->H * v->W > (1LL << 31) - 1)
        return fail(LM_EINVAL, "%s exceeds 2^31 - 1 voxels", name);
    if (v->dtype != LM_F32 && v->dtype != LM_BF16)
        return fail(LM_EINVAL, "%s has an unknown dtype %d", name, v->dtype);
    if (!v->data) return fail(LM_EINVAL, "%s data is NULL", name);
    return LM_OK;
}

}  // namespace

struct lm_ctx {
    Geom g{};
    int dtype = LM_F32;
    const void* F = nullptr;
    const void* M = nullptr;
    lm_params p{};
    cudaStream_t stream = nullptr;
    cudaStream_t cap_stream = nullptr;
    int device = 0;
    LnccConsts lc{};
    DecideConsts dc{};
    Taps wtaps{};

    // device buffers
    float* u1 = nullptr;         // field slot 1
    float* gs[2] = {nullptr, nullptr};
    float* tmpA = nullptr;       // warp smoothing temporaries
    float* tmpB = nullptr;
    StagedScratch sc{};
    bool staged = false;         // staged evaluation schedule (debug aid)
    FusedPlan plan{};
    QScale* qs = nullptr;        // fixed-point scale of the window moments
    float2* mm_part = nullptr;   // image range partials
    float* dldj = nullptr;       // dL/dJ between the fused kernels
    float* gdiscard = nullptr;   // gradient sink for lm_eval without g_out
    Partials part{};
    DevState* st = nullptr;
    LogEntry* log = nullptr;
    EvalOut* eout = nullptr;
    std::vector<void*> allocs;

    // pinned host mirrors
    DevState* h_st = nullptr;
    EvalOut* h_eout = nullptr;
    LogEntry* h_log = nullptr;

    float* bound_u = nullptr;
    bool have_reset = false;

    cudaGraphExec_t gexec = nullptr;
    float* graph_u = nullptr;
    int graph_launches = 0;      // kernels per replay of gexec
    long long launches = 0;      // kernels enqueued since lm_reset

    // coarse levels for lm_register (factor -> context), built lazily
    struct Level {
        int factor = 0;
        lm_ctx* ctx = nullptr;
        void* Fl = nullptr;
        void* Ml = nullptr;
        float* ul = nullptr;
    };
    std::vector<Level> levels;
    float* u_tmp = nullptr;      // full-res field staging for resampling
};

namespace {

template <typename T>
int dalloc(lm_ctx* c, T** out, size_t bytes) {
    void* p = nullptr;
    cudaError_t e = cudaMalloc(&p, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(LM_ENOMEM, "cudaMalloc(%zu) failed: %s", bytes,
                    cudaGetErrorString(e));
    }
    c->allocs.push_back(p);
    *out = (T*)p;
    return LM_OK;
}

int run_eval(lm_ctx* c, int mode, const float* u_in, float* g_out, float* u0,
             int attempt, cudaStream_t s);

EvalLaunch make_eval(lm_ctx* c, int mode, const float* u_in, float* g_out,
                     float* u0, int attempt) {
    EvalLaunch a;
    a.g = c->g;
    a.F = c->F;
    a.M = c->M;
    a.dtype = c->dtype;
    a.io.u_in = u_in;
    a.io.g_out = g_out;
    a.io.u0 = u0;
    a.io.u1 = c->u1;
    a.io.g0 = c->gs[0];
    a.io.g1 = c->gs[1];
    a.io.st = c->st;
    a.io.mode = mode;
    a.io.attempt = attempt;
    a.c = c->lc;
    a.part = c->part;
    a.sc = c->sc;
    return a;
}

// Pass 1 in the context's schedule; returns the number of kernels.
int run_eval(lm_ctx* c, int mode, const float* u_in, float* g_out, float* u0,
             int attempt, cudaStream_t s) {
    EvalLaunch e = make_eval(c, mode, u_in, g_out, u0, attempt);
    if (c->staged) return eval_staged(e, s);
    FusedLaunch f;
    f.g = e.g;
    f.F = e.F;
    f.M = e.M;
    f.dtype = e.dtype;
    f.io = e.io;
    f.c = e.c;
    f.plan = c->plan;
    f.qs = c->qs;
    f.dldj = c->dldj;
    f.part = c->part;
    return eval_fused(f, s);
}

FinLaunch make_fin(lm_ctx* c, int mode, int attempt) {
    FinLaunch f;
    f.part = c->part;
    f.st = c->st;
    f.out = c->eout;
    f.log = c->log;
    f.d = c->dc;
    f.inv_V = 1.0 / (double)c->g.V;
    f.mode = mode;
    f.attempt = attempt;
    return f;
}

// Enqueue one LM iteration on stream s: attempts 0..max_retries when
// rejection is on (later attempts are no-ops once the iteration is done).
int enqueue_iteration(lm_ctx* c, float* u, cudaStream_t s) {
    int attempts = c->p.reject ? c->p.max_retries + 1 : 1;
    int n = 0;
    for (int j = 0; j < attempts; ++j) {
        StepLaunch sl;
        sl.g = c->g;
        sl.u0 = u;
        sl.u1 = c->u1;
        sl.g0 = c->gs[0];
        sl.g1 = c->gs[1];
        sl.st = c->st;
        sl.step = c->p.step;
        sl.attempt = j;
        sl.wtaps = c->wtaps;
        sl.tmpA = c->tmpA;
        sl.tmpB = c->tmpB;
        n += step_compose(sl, s);
        n += run_eval(c, EVAL_TRIAL, nullptr, nullptr, u, j, s);
        n += finalize(make_fin(c, FIN_DECIDE, j), s);
    }
    return n;
}

int read_state(lm_ctx* c) {
    LM_CK(cudaMemcpyAsync(c->h_st, c->st, sizeof(DevState),
                          cudaMemcpyDeviceToHost, c->stream));
    LM_CK(cudaStreamSynchronize(c->stream));
    if (c->h_st->status & STATUS_NONFINITE)
        return fail(LM_ENONFINITE, "loss or gradient is not finite");
    return LM_OK;
}

void fill_info(const DevState& s, lm_step_info* info) {
    info->loss = s.L;
    info->loss_first = s.L_first;
    info->lambda = s.lambda;
    info->gmax = s.gmax;
    info->accepted = s.accepted;
    info->retries = s.retries;
    info->evals = s.retries + 1;
}

int check_bound(lm_ctx* c, float* u) {
    if (!c) return fail(LM_EINVAL, "ctx is NULL");
    if (!c->have_reset) return fail(LM_ESTATE, "lm_reset was not called");
    if (u != c->bound_u)
        return fail(LM_ESTATE, "u is not the field passed to lm_reset");
    return LM_OK;
}

}  // namespace

extern "C" {

int lm_default_params(lm_params* p) {
    if (!p) return fail(LM_EINVAL, "p is NULL");
    p->win = 5;
    p->eps_nr = 1e-5f;
    p->eps_dr = 1e-5f;
    p->sigma_grad = 1.0f;
    p->sigma_warp = 0.0f;
    p->step = 0.5f;
    p->lambda0 = 0.006;
    p->mu_inc = 1.5;
    p->mu_dec = 0.975;
    p->lambda_max = INFINITY;
    p->reject = 0;
    p->tau = 1.0;
    p->max_retries = 10;
    return LM_OK;
}

const char* lm_strerror(int code) {
    switch (code) {
        case LM_OK: return "ok";
        case LM_EINVAL: return "invalid argument";
        case LM_ENOMEM: return "out of memory";
        case LM_ECUDA: return "CUDA error";
        case LM_ENONFINITE: return "non-finite loss or gradient";
        case LM_ETIMEOUT: return "device wait timed out";
        case LM_EUNSUPPORTED: return "unsupported";
        case LM_ESTATE: return "call out of order";
        default: return "unknown error";
    }
}

const char* lm_last_error(void) { return g_err; }

void lm_destroy(lm_ctx* c) {
    if (!c) return;
    if (c->stream) cudaStreamSynchronize(c->stream);
    else cudaDeviceSynchronize();
    for (auto& l : c->levels) lm_destroy(l.ctx);
    if (c->gexec) cudaGraphExecDestroy(c->gexec);
    if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
    for (void* p : c->allocs) cudaFree(p);
    if (c->h_st) cudaFreeHost(c->h_st);
    if (c->h_eout) cudaFreeHost(c->h_eout);
    if (c->h_log) cudaFreeHost(c->h_log);
    delete c;
}

int lm_init(lm_ctx** out, const lm_volume* fixed, const lm_volume* moving,
            const lm_params* p, void* cuda_stream) {
    g_err[0] = 0;
    if (!out) return fail(LM_EINVAL, "ctx out-pointer is NULL");
    *out = nullptr;
    int rc;
    if ((rc = check_volume(fixed, "fixed")) != LM_OK) return rc;
    if ((rc = check_volume(moving, "moving")) != LM_OK) return rc;
    if (fixed->D != moving->D || fixed->H != moving->H ||
        fixed->W != moving->W)
        return fail(LM_EINVAL, "fixed and moving shapes differ");
    if (fixed->dtype != moving->dtype)
        return fail(LM_EINVAL, "fixed and moving dtypes differ");
    lm_params prm;
    if (p) prm = *p;
    else lm_default_params(&prm);
    if ((rc = check_params(&prm)) != LM_OK) return rc;
    if (!is_device_ptr(fixed->data))
        return fail(LM_EINVAL, "fixed data is not a device pointer");
    if (!is_device_ptr(moving->data))
        return fail(LM_EINVAL, "moving data is not a device pointer");

    lm_ctx* c = new lm_ctx();
    c->g.nx = fixed->W;
    c->g.ny = fixed->H;
    c->g.nz = fixed->D;
    c->g.V = (long long)fixed->W * fixed->H * fixed->D;
    c->dtype = fixed->dtype;
    c->F = fixed->data;
    c->M = moving->data;
    c->p = prm;
    c->stream = (cudaStream_t)cuda_stream;
    cudaGetDevice(&c->device);

    c->lc.win = prm.win;
    c->lc.eps_nr = prm.eps_nr;
    c->lc.eps_dr = prm.eps_dr;
    c->lc.inv_k3 = (float)(1.0 / ((double)prm.win * prm.win * prm.win));
    c->lc.inv_V = (float)(1.0 / (double)c->g.V);
    c->lc.gtaps = make_taps(prm.sigma_grad);
    c->lc.shift = 0.f;
    c->wtaps = make_taps(prm.sigma_warp);
    c->dc.lambda0 = prm.lambda0;
    c->dc.mu_inc = prm.mu_inc;
    c->dc.mu_dec = prm.mu_dec;
    c->dc.lambda_max = prm.lambda_max;
    c->dc.tau = prm.tau;
    c->dc.reject = prm.reject;
    c->dc.max_retries = prm.max_retries;

    const size_t V = (size_t)c->g.V;
    const size_t f4 = sizeof(float);
    {
        const char* e = getenv("LMREG_STAGED");
        c->staged = e && e[0] == '1';
    }
    static std::once_flag setup_once;
    static cudaError_t setup_err = cudaSuccess;
    std::call_once(setup_once, [] { setup_err = fused_setup(); });
    if (setup_err != cudaSuccess) {
        lm_destroy(c);
        return fail(LM_ECUDA, "kernel setup failed: %s",
                    cudaGetErrorString(setup_err));
    }
    int num_sms = 0;
    if (cudaDeviceGetAttribute(&num_sms, cudaDevAttrMultiProcessorCount,
                               c->device) != cudaSuccess || num_sms < 1) {
        cudaGetLastError();
        num_sms = 148;
    }
    c->plan = fused_plan(c->g, prm.win, num_sms);
    int nl, ng;
    if (c->staged) {
        eval_staged_partials(c->g, &nl, &ng);
    } else {
        nl = c->plan.e1_ctas;
        ng = c->plan.e2_ctas;
    }
    int nl_alloc = std::max(nl, (int)std::min<long long>((c->g.V + 255) / 256, 1024));
    c->part.n_loss = nl;
    c->part.n_g2 = ng;
    if ((rc = dalloc(c, &c->u1, 3 * V * f4)) ||
        (rc = dalloc(c, &c->gs[0], 3 * V * f4)) ||
        (rc = dalloc(c, &c->gs[1], 3 * V * f4)) ||
        (rc = dalloc(c, &c->gdiscard, 3 * V * f4)) ||
        (rc = dalloc(c, &c->part.loss, (size_t)nl_alloc * sizeof(double))) ||
        (rc = dalloc(c, &c->part.g2max, (size_t)ng * sizeof(float))) ||
        (rc = dalloc(c, &c->st, sizeof(DevState))) ||
        (rc = dalloc(c, &c->log, LOG_CAP * sizeof(LogEntry))) ||
        (rc = dalloc(c, &c->eout, sizeof(EvalOut)))) {
        lm_destroy(c);
        return rc;
    }
    if (c->staged) {
        if ((rc = dalloc(c, &c->sc.J, V * f4)) ||
            (rc = dalloc(c, &c->sc.dJ, 3 * V * f4)) ||
            (rc = dalloc(c, &c->sc.S, 5 * V * f4)) ||
            (rc = dalloc(c, &c->sc.T, 5 * V * f4)) ||
            (rc = dalloc(c, &c->sc.abc, 3 * V * f4)) ||
            (rc = dalloc(c, &c->sc.graw, 3 * V * f4))) {
            lm_destroy(c);
            return rc;
        }
    } else {
        if ((rc = dalloc(c, &c->dldj, V * f4)) ||
            (rc = dalloc(c, &c->qs, sizeof(QScale))) ||
            (rc = dalloc(c, &c->mm_part,
                         (size_t)c->plan.minmax_ctas * sizeof(float2)))) {
            lm_destroy(c);
            return rc;
        }
    }
    if (c->wtaps.R > 0) {
        if ((rc = dalloc(c, &c->tmpA, 3 * V * f4)) ||
            (rc = dalloc(c, &c->tmpB, 3 * V * f4))) {
            lm_destroy(c);
            return rc;
        }
    }
    if (cudaMallocHost(&c->h_st, sizeof(DevState)) != cudaSuccess ||
        cudaMallocHost(&c->h_eout, sizeof(EvalOut)) != cudaSuccess ||
        cudaMallocHost(&c->h_log, LOG_CAP * sizeof(LogEntry)) != cudaSuccess) {
        cudaGetLastError();
        lm_destroy(c);
        return fail(LM_ENOMEM, "pinned host allocation failed");
    }
    if (cudaMemsetAsync(c->st, 0, sizeof(DevState), c->stream) != cudaSuccess) {
        lm_destroy(c);
        return fail(LM_ECUDA, "cudaMemsetAsync failed");
    }
    if (c->staged) {
        // common shift of the staged box sums: the mean intensity of F
        float mean = 0.f;
        if ((rc = lmk::image_mean(c->F, c->dtype, c->g.V, c->part.loss,
                                  &mean, c->stream)) != 0) {
            lm_destroy(c);
            return fail(LM_ECUDA, "image mean failed");
        }
        c->lc.shift = mean;
    }
    *out = c;
    return LM_OK;
}

int lm_eval(lm_ctx* c, const float* u, double* loss, float* g_out,
            float* gmax) {
    if (!c) return fail(LM_EINVAL, "ctx is NULL");
    if (!is_device_ptr(u)) return fail(LM_EINVAL, "u is not a device pointer");
    if (g_out && !is_device_ptr(g_out))
        return fail(LM_EINVAL, "g_out is not a device pointer");
    float* gdst = g_out ? g_out : c->gdiscard;
    if (!c->staged)
        fused_qscale(c->F, c->M, c->dtype, c->g, c->plan, c->p.win,
                     c->mm_part, c->qs, c->stream);
    run_eval(c, EVAL_EXPLICIT, u, gdst, (float*)u, 0, c->stream);
    finalize(make_fin(c, FIN_EXPLICIT, 0), c->stream);
    LM_CK(cudaGetLastError());
    LM_CK(cudaMemcpyAsync(c->h_eout, c->eout, sizeof(EvalOut),
                          cudaMemcpyDeviceToHost, c->stream));
    LM_CK(cudaStreamSynchronize(c->stream));
    if (loss) *loss = c->h_eout->L;
    if (gmax) *gmax = c->h_eout->gmax;
    if (c->h_eout->status & STATUS_NONFINITE)
        return fail(LM_ENONFINITE, "loss or gradient is not finite");
    return LM_OK;
}

int lm_reset(lm_ctx* c, float* u) {
    if (!c) return fail(LM_EINVAL, "ctx is NULL");
    if (!is_device_ptr(u)) return fail(LM_EINVAL, "u is not a device pointer");
    c->launches = 0;
    if (!c->staged)
        c->launches += fused_qscale(c->F, c->M, c->dtype, c->g, c->plan,
                                    c->p.win, c->mm_part, c->qs, c->stream);
    c->launches += run_eval(c, EVAL_RESET, nullptr, nullptr, u, 0, c->stream);
    c->launches += finalize(make_fin(c, FIN_RESET, 0), c->stream);
    LM_CK(cudaGetLastError());
    c->bound_u = u;
    c->have_reset = true;
    return LM_OK;
}

int lm_step(lm_ctx* c, float* u, lm_step_info* info) {
    int rc = check_bound(c, u);
    if (rc) return rc;
    c->launches += enqueue_iteration(c, u, c->stream);
    c->launches += sync_back(c->g, u, c->u1, c->st, c->stream);
    LM_CK(cudaGetLastError());
    if (info) {
        if ((rc = read_state(c)) != LM_OK) return rc;
        fill_info(*c->h_st, info);
    }
    return LM_OK;
}

int lm_iterate(lm_ctx* c, float* u, int n, lm_step_info* info) {
    int rc = check_bound(c, u);
    if (rc) return rc;
    if (n < 0) return fail(LM_EINVAL, "n must be >= 0");
    if (n > 0) {
        if (!c->gexec || c->graph_u != u) {
            if (c->gexec) {
                cudaGraphExecDestroy(c->gexec);
                c->gexec = nullptr;
            }
            if (!c->cap_stream)
                LM_CK(cudaStreamCreateWithFlags(&c->cap_stream,
                                                cudaStreamNonBlocking));
            cudaGraph_t graph;
            LM_CK(cudaStreamBeginCapture(c->cap_stream,
                                         cudaStreamCaptureModeThreadLocal));
            c->graph_launches = enqueue_iteration(c, u, c->cap_stream);
            cudaError_t e = cudaStreamEndCapture(c->cap_stream, &graph);
            if (e != cudaSuccess)
                return fail(LM_ECUDA, "graph capture failed: %s",
                            cudaGetErrorString(e));
            e = cudaGraphInstantiate(&c->gexec, graph, 0);
            cudaGraphDestroy(graph);
            if (e != cudaSuccess)
                return fail(LM_ECUDA, "graph instantiate failed: %s",
                            cudaGetErrorString(e));
            c->graph_u = u;
        }
        for (int i = 0; i < n; ++i) LM_CK(cudaGraphLaunch(c->gexec, c->stream));
        c->launches += (long long)n * c->graph_launches;
        c->launches += sync_back(c->g, u, c->u1, c->st, c->stream);
        LM_CK(cudaGetLastError());
    }
    if (info) {
        if ((rc = read_state(c)) != LM_OK) return rc;
        fill_info(*c->h_st, info);
    }
    return LM_OK;
}

int lm_get_state(lm_ctx* c, lm_state* out) {
    if (!c || !out) return fail(LM_EINVAL, "NULL argument");
    LM_CK(cudaMemcpyAsync(c->h_st, c->st, sizeof(DevState),
                          cudaMemcpyDeviceToHost, c->stream));
    LM_CK(cudaStreamSynchronize(c->stream));
    const DevState& s = *c->h_st;
    out->loss = s.L;
    out->loss_prev = s.L_prev;
    out->lambda = s.lambda;
    out->gmax = s.gmax;
    out->has_prev = s.has_prev;
    out->iter = s.iter;
    out->evals = s.evals;
    out->kernel_launches = c->launches;
    return LM_OK;
}

int lm_set_state(lm_ctx* c, const lm_state* in) {
    if (!c || !in) return fail(LM_EINVAL, "NULL argument");
    if (!c->have_reset) return fail(LM_ESTATE, "lm_reset was not called");
    if (!(in->lambda > 0) || !std::isfinite(in->lambda) ||
        !std::isfinite(in->loss) || !std::isfinite(in->loss_prev))
        return fail(LM_EINVAL, "state scalars must be finite, lambda > 0");
    LM_CK(cudaMemcpyAsync(c->h_st, c->st, sizeof(DevState),
                          cudaMemcpyDeviceToHost, c->stream));
    LM_CK(cudaStreamSynchronize(c->stream));
    DevState s = *c->h_st;
    s.L = in->loss;
    s.L_prev = in->loss_prev;
    s.lambda = in->lambda;
    s.gmax = in->gmax;
    s.has_prev = in->has_prev ? 1 : 0;
    s.iter = in->iter;
    s.evals = in->evals;
    *c->h_st = s;
    LM_CK(cudaMemcpyAsync(c->st, c->h_st, sizeof(DevState),
                          cudaMemcpyHostToDevice, c->stream));
    LM_CK(cudaStreamSynchronize(c->stream));
    return LM_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------
// Checkpoints: a small header, the device state, then the current
// gradient (3V floats).  The field itself is the caller's.
// ---------------------------------------------------------------------
namespace {
struct CkptHeader {
    char magic[8];
    int nx, ny, nz, version;
};
}  // namespace

extern "C" int lm_state_save(lm_ctx* c, void* buf, size_t* nbytes) {
    if (!c || !nbytes) return fail(LM_EINVAL, "NULL argument");
    if (!c->have_reset) return fail(LM_ESTATE, "lm_reset was not called");
    size_t need = sizeof(CkptHeader) + sizeof(DevState) +
                  3 * (size_t)c->g.V * sizeof(float);
    if (!buf) {
        *nbytes = need;
        return LM_OK;
    }
    if (*nbytes < need) return fail(LM_EINVAL, "buffer too small");
    // make sure the field sits in the caller's slot
    sync_back(c->g, c->bound_u, c->u1, c->st, c->stream);
    LM_CK(cudaMemcpyAsync(c->h_st, c->st, sizeof(DevState),
                          cudaMemcpyDeviceToHost, c->stream));
    LM_CK(cudaStreamSynchronize(c->stream));
    CkptHeader h;
    memcpy(h.magic, "LMREGCK1", 8);
    h.nx = c->g.nx;
    h.ny = c->g.ny;
    h.nz = c->g.nz;
    h.version = 1;
    char* p = (char*)buf;
    memcpy(p, &h, sizeof(h));
    memcpy(p + sizeof(h), c->h_st, sizeof(DevState));
    LM_CK(cudaMemcpy(p + sizeof(h) + sizeof(DevState), c->gs[c->h_st->cg],
                     3 * (size_t)c->g.V * sizeof(float),
                     cudaMemcpyDeviceToHost));
    *nbytes = need;
    return LM_OK;
}

extern "C" int lm_state_load(lm_ctx* c, const void* buf, size_t nbytes) {
    if (!c || !buf) return fail(LM_EINVAL, "NULL argument");
    if (!c->have_reset) return fail(LM_ESTATE, "lm_reset was not called");
    size_t need = sizeof(CkptHeader) + sizeof(DevState) +
                  3 * (size_t)c->g.V * sizeof(float);
    if (nbytes < need) return fail(LM_EINVAL, "checkpoint too small");
    CkptHeader h;
    memcpy(&h, buf, sizeof(h));
    if (memcmp(h.magic, "LMREGCK1", 8) != 0 || h.version != 1)
        return fail(LM_EINVAL, "not an lmreg checkpoint");
    if (h.nx != c->g.nx || h.ny != c->g.ny || h.nz != c->g.nz)
        return fail(LM_EINVAL, "checkpoint shape differs from the context");
    DevState s;
    memcpy(&s, (const char*)buf + sizeof(h), sizeof(DevState));
    s.cu = 0;       // the field is the caller's (slot 0)
    s.cg = 0;       // the gradient is restored into slot 0
    s.done = 0;
    *c->h_st = s;
    LM_CK(cudaMemcpyAsync(c->st, c->h_st, sizeof(DevState),
                          cudaMemcpyHostToDevice, c->stream));
    LM_CK(cudaMemcpyAsync(c->gs[0],
                          (const char*)buf + sizeof(h) + sizeof(DevState),
                          3 * (size_t)c->g.V * sizeof(float),
                          cudaMemcpyHostToDevice, c->stream));
    LM_CK(cudaStreamSynchronize(c->stream));
    return LM_OK;
}

// ---------------------------------------------------------------------
// Coarse-to-fine registration.
// ---------------------------------------------------------------------
extern "C" int lm_time_passes(lm_ctx* c, float* u, int n, double* ms_eval,
                              double* ms_step) {
    int rc = check_bound(c, u);
    if (rc) return rc;
    if (n < 1 || !ms_eval || !ms_step)
        return fail(LM_EINVAL, "n must be >= 1 and outputs non-NULL");
    cudaEvent_t e0, e1, e2;
    LM_CK(cudaEventCreate(&e0));
    LM_CK(cudaEventCreate(&e1));
    LM_CK(cudaEventCreate(&e2));
    StepLaunch sl;
    sl.g = c->g;
    sl.u0 = u;
    sl.u1 = c->u1;
    sl.g0 = c->gs[0];
    sl.g1 = c->gs[1];
    sl.st = c->st;
    sl.step = c->p.step;
    sl.attempt = 0;
    sl.wtaps = c->wtaps;
    sl.tmpA = c->tmpA;
    sl.tmpB = c->tmpB;
    LM_CK(cudaEventRecord(e0, c->stream));
    for (int i = 0; i < n; ++i) step_compose(sl, c->stream);
    LM_CK(cudaEventRecord(e1, c->stream));
    for (int i = 0; i < n; ++i)
        run_eval(c, EVAL_TRIAL, nullptr, nullptr, u, 0, c->stream);
    LM_CK(cudaEventRecord(e2, c->stream));
    LM_CK(cudaEventSynchronize(e2));
    float a = 0.f, b = 0.f;
    cudaEventElapsedTime(&a, e0, e1);
    cudaEventElapsedTime(&b, e1, e2);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaEventDestroy(e2);
    *ms_step = a / n;
    *ms_eval = b / n;
    LM_CK(cudaGetLastError());
    return LM_OK;
}

extern "C" int lm_register(lm_ctx* c, const lm_schedule* s, float* u,
                           lm_report* rep) {
    if (!c || !s) return fail(LM_EINVAL, "NULL argument");
    if (!is_device_ptr(u)) return fail(LM_EINVAL, "u is not a device pointer");
    if (s->nlevels < 1 || s->nlevels > LM_MAX_LEVELS)
        return fail(LM_EINVAL, "nlevels must be in [1, %d]", LM_MAX_LEVELS);
    for (int l = 0; l < s->nlevels; ++l) {
        int f = s->factor[l];
        if (f != 1 && f != 2 && f != 4)
            return fail(LM_EINVAL, "factor[%d] must be 1, 2 or 4", l);
        if (s->iters[l] < 0) return fail(LM_EINVAL, "iters[%d] < 0", l);
    }
    auto t0 = std::chrono::steady_clock::now();
    int rc;
    const size_t V = (size_t)c->g.V;
    if (!c->u_tmp) {
        if ((rc = dalloc(c, &c->u_tmp, 3 * V * sizeof(float))) != LM_OK)
            return rc;
    }
    lm_report r;
    memset(&r, 0, sizeof(r));
    r.nlevels = s->nlevels;
    // the field travels between levels in `cur` (dims cx, cy, cz, factor cf)
    float* cur = u;
    int cx = c->g.nx, cy = c->g.ny, cz = c->g.nz, cf = 1;
    for (int l = 0; l < s->nlevels; ++l) {
        int f = s->factor[l];
        lm_ctx* lc = c;
        float* ul = u;
        if (f != 1) {
            lm_ctx::Level* lv = nullptr;
            for (auto& x : c->levels)
                if (x.factor == f) lv = &x;
            if (!lv) {
                lm_ctx::Level nl;
                nl.factor = f;
                int lx, ly, lz;
                level_dims(c->g.nx, c->g.ny, c->g.nz, f, &lx, &ly, &lz);
                size_t Vl = (size_t)lx * ly * lz;
                size_t es = c->dtype == LM_BF16 ? 2 : 4;
                if ((rc = dalloc(c, &nl.Fl, Vl * es)) ||
                    (rc = dalloc(c, &nl.Ml, Vl * es)) ||
                    (rc = dalloc(c, &nl.ul, 3 * Vl * sizeof(float))))
                    return rc;
                // level images must exist before the level context reads
                // their mean
                if ((rc = downsample_image(c->F, c->dtype, c->g, f, nl.Fl,
                                           c->u_tmp, c->stream)) ||
                    (rc = downsample_image(c->M, c->dtype, c->g, f, nl.Ml,
                                           c->u_tmp, c->stream)))
                    return fail(LM_ECUDA, "downsample failed");
                lm_volume vf = {lz, ly, lx, c->dtype, nl.Fl};
                lm_volume vm = {lz, ly, lx, c->dtype, nl.Ml};
                if ((rc = lm_init(&nl.ctx, &vf, &vm, &c->p, c->stream)))
                    return rc;
                c->levels.push_back(nl);
                lv = &c->levels.back();
            }
            else {
                // the caller may have changed F or M since the last call
                if ((rc = downsample_image(c->F, c->dtype, c->g, f, lv->Fl,
                                           c->u_tmp, c->stream)) ||
                    (rc = downsample_image(c->M, c->dtype, c->g, f, lv->Ml,
                                           c->u_tmp, c->stream)))
                    return fail(LM_ECUDA, "downsample failed");
            }
            lc = lv->ctx;
            ul = lv->ul;
        }
        // carry the field from (cur, cf) into this level's buffer
        if (ul != cur || cf != f) {
            Geom ga{cx, cy, cz, (long long)cx * cy * cz};
            float* src = cur;
            if (ul == cur) {   // resample in place through the staging copy
                LM_CK(cudaMemcpyAsync(c->u_tmp, cur, 3 * ga.V * sizeof(float),
                                      cudaMemcpyDeviceToDevice, c->stream));
                src = c->u_tmp;
            }
            if ((rc = resample_field(src, ga, cf, ul, lc->g, f, c->stream)))
                return fail(LM_ECUDA, "field resampling failed");
        }
        if ((rc = lm_reset(lc, ul)) != LM_OK) return rc;
        lm_step_info info;
        if ((rc = lm_iterate(lc, ul, s->iters[l], &info)) != LM_OK) return rc;
        DevState hs = *lc->h_st;
        r.level_dims[l][0] = lc->g.nz;
        r.level_dims[l][1] = lc->g.ny;
        r.level_dims[l][2] = lc->g.nx;
        r.level_iters[l] = hs.iter;
        r.level_evals[l] = hs.evals;
        r.level_accepted[l] = 0;
        int nlog = hs.log_pos < LOG_CAP ? hs.log_pos : LOG_CAP;
        if (nlog > 0) {
            LM_CK(cudaMemcpy(lc->h_log, lc->log, nlog * sizeof(LogEntry),
                             cudaMemcpyDeviceToHost));
            for (int i = 0; i < nlog; ++i)
                r.level_accepted[l] += lc->h_log[i].accepted;
        }
        r.level_loss[l] = hs.L;
        r.voxel_evals += (long long)lc->g.V * hs.evals;
        cur = ul;
        cx = lc->g.nx;
        cy = lc->g.ny;
        cz = lc->g.nz;
        cf = f;
    }
    if (cur != u) {
        Geom ga{cx, cy, cz, (long long)cx * cy * cz};
        if ((rc = resample_field(cur, ga, cf, u, c->g, 1, c->stream)))
            return fail(LM_ECUDA, "field resampling failed");
    }
    LM_CK(cudaStreamSynchronize(c->stream));
    r.final_loss = r.level_loss[s->nlevels - 1];
    auto t1 = std::chrono::steady_clock::now();
    r.wall_ms = std::chrono::duration<double, std::milli>(t1 - t0).count();
    if (rep) *rep = r;
    return LM_OK;
}
