// Host runtime behind the C ABI of include/lmreg.h: argument validation,
// device scratch, the ordering of the kernels of one LM iteration (rejected
// retries unrolled so no host round trip is needed), CUDA graph replay of
// iterations, the coarse-to-fine schedule, batches of pairs, checkpoints.
//
// A Core holds a batch of pairs: a device table of PairDesc entries, the
// per-pair buffers and state, and the shared partial arrays.  The
// single-pair context (lm_ctx) is a Core of one pair; lm_batch is a Core of
// many.  All kernels of an iteration read the table at run time, so one
// captured CUDA graph serves any caller field pointers.
#include <algorithm>
#include <chrono>
#include <limits>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <memory>
#include <mutex>
#include <vector>

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

}  // namespace

void lmk::set_last_error(const char* msg) {
    snprintf(g_err, sizeof(g_err), "%s", msg);
}

bool lmk::is_device_ptr(const void* p) {
    if (!p) return false;
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

Taps lmk::make_taps(double sigma) {
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

int lmk::check_params(const lm_params* p) {
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
    if (p->tile < 1 || p->tile > 16)
        return fail(LM_EINVAL, "tile must be in [1, 16], got %d", p->tile);
    if (p->loss != LM_LOSS_LNCC && p->loss != LM_LOSS_MSE &&
        p->loss != LM_LOSS_MI)
        return fail(LM_EINVAL,
                    "loss must be LM_LOSS_LNCC, LM_LOSS_MSE or LM_LOSS_MI");
    if (p->bins < 4 || p->bins > MI_MAX_BINS)
        return fail(LM_EINVAL, "bins must be in [4, %d], got %d", MI_MAX_BINS,
                    p->bins);
    if (p->method != LM_METHOD_LM && p->method != LM_METHOD_DEMONS)
        return fail(LM_EINVAL,
                    "method must be LM_METHOD_LM or LM_METHOD_DEMONS");
    if (!(p->alpha > 0) || !std::isfinite(p->alpha))
        return fail(LM_EINVAL, "alpha must be finite and > 0");
    if (p->method == LM_METHOD_DEMONS &&
        (p->loss != LM_LOSS_MSE || p->tile != 1 || p->reject != 0))
        return fail(LM_EINVAL,
                    "method LM_METHOD_DEMONS needs loss LM_LOSS_MSE, tile 1 "
                    "and reject 0");
    return LM_OK;
}

namespace {

#define LM_CK(call)                                                        \
    do {                                                                   \
        cudaError_t e_ = (call);                                           \
        if (e_ != cudaSuccess)                                             \
            return fail(LM_ECUDA, "%s failed: %s", #call,                  \
                        cudaGetErrorString(e_));                           \
    } while (0)

// Shape and dtype checks (host only, no CUDA call).
int check_volume(const lm_volume* v, const char* name) {
    if (!v) return fail(LM_EINVAL, "%s is NULL", name);
    if (v->D < 1 || v->H < 1 || v->W < 1)
        return fail(LM_EINVAL, "%s has a non-positive dimension", name);
    // fields of 3 V floats are indexed with 32-bit offsets in the kernels
    if (3LL * v->D * v->H * v->W > (1LL << 31) - 1)
        return fail(LM_EINVAL, "%s exceeds (2^31 - 1) / 3 voxels", name);
    if (v->dtype != LM_F32 && v->dtype != LM_BF16)
        return fail(LM_EINVAL, "%s has an unknown dtype %d", name, v->dtype);
    if (!v->data) return fail(LM_EINVAL, "%s data is NULL", name);
    return LM_OK;
}

int check_pair(const lm_volume* f, const lm_volume* m) {
    int rc;
    if ((rc = check_volume(f, "fixed")) != LM_OK) return rc;
    if ((rc = check_volume(m, "moving")) != LM_OK) return rc;
    if (f->D != m->D || f->H != m->H || f->W != m->W)
        return fail(LM_EINVAL, "fixed and moving shapes differ");
    if (f->dtype != m->dtype)
        return fail(LM_EINVAL, "fixed and moving dtypes differ");
    return LM_OK;
}

// Host-side fault injection: an environment variable read as an integer
// (0 when unset or not a number).
int env_int(const char* name) {
    const char* v = getenv(name);
    return v ? atoi(v) : 0;
}

// Error code of a pair's device status word: a wait that ran out comes
// before a non-finite result (its partials are void).
int status_error(int status, int pair) {
    if (status & STATUS_TIMEOUT)
        return fail(LM_ETIMEOUT, "a bounded device wait ran out (pair %d)",
                    pair);
    if (status & STATUS_NONFINITE)
        return fail(LM_ENONFINITE, "loss or gradient is not finite (pair %d)",
                    pair);
    return LM_OK;
}

// ---------------------------------------------------------------------
// Core: a batch of pairs with its device scratch and state.
// ---------------------------------------------------------------------
struct Core {
    int npairs = 0;
    int dtype = LM_F32;
    lm_params p{};
    cudaStream_t stream = nullptr;
    cudaStream_t cap_stream = nullptr;
    int device = 0;
    std::vector<PairDesc> hpd;     // host copy of the table
    PairDesc* dpd = nullptr;       // device table
    Batch b{};
    std::vector<void*> allocs;
    EvalOut* eout = nullptr;       // npairs
    DevState* h_st = nullptr;      // pinned, npairs
    EvalOut* h_eout = nullptr;     // pinned, npairs
    LogEntry* h_log = nullptr;     // pinned, LOG_CAP
    std::vector<float*> gsink;     // lm_eval gradient sinks (lazy)
    bool have_reset = false;
    // the captured iteration, once (gexec) and GRAPH_ITERS times in a row
    // (gexec_n: one replay per GRAPH_ITERS iterations, so that a run of
    // short iterations pays the launch of a graph once per group)
    static constexpr int GRAPH_ITERS = 8;
    cudaGraphExec_t gexec = nullptr;
    cudaGraphExec_t gexec_n = nullptr;
    int graph_launches = 0;        // kernels of one graph launch
    long long launches = 0;
    int num_sms = 0;
    int e1_cap = 0, e2_cap = 0;    // partial slots allocated (any plan fits)
    int nalloc = 0;                // device allocations so far
    int fault_alloc = env_int("LM_FAULT_ALLOC");   // 0: no injected failure

    ~Core() {
        if (stream) cudaStreamSynchronize(stream);
        else cudaDeviceSynchronize();
        drop_graphs();
        if (cap_stream) cudaStreamDestroy(cap_stream);
        for (void* q : allocs) cudaFree(q);
        if (h_st) cudaFreeHost(h_st);
        if (h_eout) cudaFreeHost(h_eout);
        if (h_log) cudaFreeHost(h_log);
    }

#ifdef LM_DEBUG_BOUNDS
    // Guard bands of GUARD bytes before and after every device buffer,
    // filled with 0xFF (NaN as a float, -1 as an integer): a kernel that
    // writes outside its buffer changes a band (check_guards), one that
    // reads outside it reads NaN or -1 and fails parity.
    static constexpr size_t GUARD = 1 << 16;
    std::vector<std::pair<unsigned char*, size_t>> guarded;
#else
    static constexpr size_t GUARD = 0;
#endif

    template <typename T>
    int dalloc(T** out, size_t bytes) {
        void* q = nullptr;
        // LM_FAULT_ALLOC=n: the context's n-th device allocation fails
        if (++nalloc == fault_alloc)
            return fail(LM_ENOMEM, "cudaMalloc(%zu) failed: injected by "
                                   "LM_FAULT_ALLOC=%d", bytes, fault_alloc);
        cudaError_t e = cudaMalloc(&q, bytes + 2 * GUARD);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return fail(LM_ENOMEM, "cudaMalloc(%zu) failed: %s", bytes,
                        cudaGetErrorString(e));
        }
        allocs.push_back(q);
#ifdef LM_DEBUG_BOUNDS
        unsigned char* base = (unsigned char*)q;
        LM_CK(cudaMemset(base, 0xFF, GUARD));
        LM_CK(cudaMemset(base + GUARD + bytes, 0xFF, GUARD));
        // the bands are in place before any kernel on any stream runs
        LM_CK(cudaDeviceSynchronize());
        guarded.emplace_back(base, bytes);
#endif
        *out = (T*)((unsigned char*)q + GUARD);
        return LM_OK;
    }

    // Debug-bounds build: LM_OK if every guard band is intact, LM_EBOUNDS
    // naming the first changed byte otherwise.
    int check_guards() {
#ifdef LM_DEBUG_BOUNDS
        LM_CK(cudaStreamSynchronize(stream));
        LM_CK(cudaDeviceSynchronize());
        std::vector<unsigned char> h(GUARD);
        for (size_t a = 0; a < guarded.size(); ++a) {
            for (int side = 0; side < 2; ++side) {
                const unsigned char* band =
                    guarded[a].first + (side ? GUARD + guarded[a].second : 0);
                LM_CK(cudaMemcpy(h.data(), band, GUARD, cudaMemcpyDeviceToHost));
                for (size_t i = 0; i < GUARD; ++i)
                    if (h[i] != 0xFF)
                        return fail(LM_EBOUNDS,
                                    "a kernel wrote byte %lld of buffer %zu "
                                    "(%zu bytes long)",
                                    side ? (long long)(guarded[a].second + i)
                                         : (long long)i - (long long)GUARD,
                                    a, guarded[a].second);
            }
        }
        return LM_OK;
#else
        return fail(LM_EUNSUPPORTED, "built without LM_DEBUG_BOUNDS");
#endif
    }

    // Host table -> device (pageable source: safe to modify on return).
    int push_table() {
        LM_CK(cudaMemcpyAsync(dpd, hpd.data(), npairs * sizeof(PairDesc),
                              cudaMemcpyHostToDevice, stream));
        return LM_OK;
    }

    int read_states() {
        LM_CK(cudaMemcpyAsync(h_st, hpd[0].st, npairs * sizeof(DevState),
                              cudaMemcpyDeviceToHost, stream));
        LM_CK(cudaStreamSynchronize(stream));
        for (int i = 0; i < npairs; ++i)
            if (int rc = status_error(h_st[i].status, i)) return rc;
        return LM_OK;
    }

    // One LM iteration for every pair: attempts 0..max_retries when
    // rejection is on (later attempts are no-ops once a pair is decided).
    int enqueue_iteration(cudaStream_t s) {
        int attempts = p.reject ? p.max_retries + 1 : 1;
        int n = 0;
        for (int j = 0; j < attempts; ++j) {
            n += batch_step(b, j, s);
            n += batch_eval(b, EVAL_TRIAL, j, s, !step_resamples(b));
            n += batch_finalize(b, FIN_DECIDE, j, nullptr, s);
        }
        return n;
    }

    // With rejection a replayed iteration is one state-driven attempt
    // (kernels given attempt -1): the decision leaves each pair's next
    // attempt in its device state, so a replay after a rejection retries
    // the iteration and a replay after a decision starts the next one.  An
    // iteration without rejections therefore costs one replay, and the
    // graph holds no conditional node.  iterate() bounds each pair's run
    // by iter_end and replays until every pair has finished its n
    // iterations (or stopped), reading the states in between.
    bool replay_retries() const { return p.reject && p.max_retries > 0; }

    // Captures iters passes in a row and instantiates them.
    int capture_graph(int iters, cudaGraphExec_t* exec) {
        if (!cap_stream)
            LM_CK(cudaStreamCreateWithFlags(&cap_stream,
                                            cudaStreamNonBlocking));
        LM_CK(cudaStreamBeginCapture(cap_stream,
                                     cudaStreamCaptureModeThreadLocal));
        for (int i = 0; i < iters; ++i) {
            if (!replay_retries()) {
                graph_launches = enqueue_iteration(cap_stream);
            } else {
                graph_launches = batch_step(b, -1, cap_stream);
                graph_launches += batch_eval(b, EVAL_TRIAL, -1, cap_stream,
                                             !step_resamples(b));
                graph_launches += batch_finalize(b, FIN_DECIDE, -1, nullptr,
                                                 cap_stream);
            }
        }
        cudaGraph_t graph;
        LM_CK(cudaStreamEndCapture(cap_stream, &graph));
        cudaError_t e = cudaGraphInstantiate(exec, graph, 0);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess)
            return fail(LM_ECUDA, "graph instantiate failed: %s",
                        cudaGetErrorString(e));
        return LM_OK;
    }

    void drop_graphs() {
        if (gexec) cudaGraphExecDestroy(gexec);
        if (gexec_n) cudaGraphExecDestroy(gexec_n);
        gexec = gexec_n = nullptr;
    }

    // n passes (graph_launches kernels each): whole groups from gexec_n,
    // the rest one at a time.
    int replay(int n) {
        for (int i = 0; i < n / GRAPH_ITERS; ++i)
            LM_CK(cudaGraphLaunch(gexec_n, stream));
        for (int i = 0; i < n % GRAPH_ITERS; ++i)
            LM_CK(cudaGraphLaunch(gexec, stream));
        launches += (long long)n * graph_launches;
        return LM_OK;
    }

    // Replays until every pair has reached its iter_end or stopped; the
    // passes of one round are the largest number of iterations any pair
    // still owes.  Each round reads the states (a synchronisation).  Every
    // pass either finishes a pair's iteration or uses one of its retries,
    // so n iterations take at most (max_retries + 1) n passes; more means
    // the device state is inconsistent, reported rather than looped on.
    int replay_until_done(int n, int done) {
        const long long cap = (long long)(p.max_retries + 1) * n;
        long long passes = done;
        for (;;) {
            if (int rc = read_states()) return rc;
            int owe = 0;
            for (int i = 0; i < npairs; ++i) {
                const DevState& s = h_st[i];
                if (!s.stopped && s.iter_end > 0 && s.iter_end - s.iter > owe)
                    owe = s.iter_end - s.iter;
            }
            if (owe == 0) return LM_OK;
            if (passes + owe > cap)
                return fail(LM_ESTATE, "%lld replays left iterations undone",
                            passes);
            if (int rc = replay(owe)) return rc;
            passes += owe;
        }
    }

    int iterate(int n) {
        if (n <= 0) return LM_OK;
        if (!gexec) {
            int rc = capture_graph(1, &gexec);
            if (rc == LM_OK) rc = capture_graph(GRAPH_ITERS, &gexec_n);
            if (rc != LM_OK) {
                drop_graphs();
                return rc;
            }
        }
        int rc = LM_OK;
        if (!replay_retries()) {
            rc = replay(n);
        } else {
            launches += batch_set_iter_end(b, n, stream);
            rc = replay(n);
            if (rc == LM_OK) rc = replay_until_done(n, n);
            // the limit ends with the run, whatever its outcome
            launches += batch_set_iter_end(b, 0, stream);
        }
        // the current field back in the caller's slot, whatever the outcome
        launches += batch_sync_back(b, stream);
        if (rc != LM_OK) return rc;
        LM_CK(cudaGetLastError());
        return LM_OK;
    }
};

// Wave counts the autotuner tries (CTAs per SM in total for E1 and E2).
constexpr int kE1Waves[] = {1, 2, 4, 8};
constexpr int kE2Waves[] = {2, 3, 4, 8, 16};
constexpr int kMinSlices[] = {8, 4, 2, 1};
constexpr int kStepBlocks[] = {512, 1024, 2048, 4096};
constexpr int kMaxE1Waves = 8, kMaxE2Waves = 16;

// Creates a Core for npairs pairs (all of one dtype).
int core_create(std::unique_ptr<Core>& out, int npairs,
                const lm_volume* fixed, const lm_volume* moving,
                const lm_params* p, void* stream) {
    if (npairs < 1) return fail(LM_EINVAL, "npairs must be >= 1");
    if (!fixed || !moving) return fail(LM_EINVAL, "fixed / moving is NULL");
    int rc;
    for (int i = 0; i < npairs; ++i)
        if ((rc = check_pair(&fixed[i], &moving[i])) != LM_OK) return rc;
    for (int i = 1; i < npairs; ++i)
        if (fixed[i].dtype != fixed[0].dtype)
            return fail(LM_EINVAL, "all pairs of a batch share one dtype");
    lm_params prm;
    if (p) prm = *p;
    else lm_default_params(&prm);
    if ((rc = check_params(&prm)) != LM_OK) return rc;
    for (int i = 0; i < npairs; ++i)
        if (!is_device_ptr(fixed[i].data) || !is_device_ptr(moving[i].data))
            return fail(LM_EINVAL, "image data of pair %d is not a device "
                                   "pointer", i);
    static std::once_flag setup_once;
    static cudaError_t setup_err = cudaSuccess;
    std::call_once(setup_once, [] { setup_err = fused_setup(); });
    if (setup_err != cudaSuccess)
        return fail(LM_ECUDA, "kernel setup failed: %s",
                    cudaGetErrorString(setup_err));

    auto c = std::make_unique<Core>();
    c->npairs = npairs;
    c->dtype = fixed[0].dtype;
    c->p = prm;
    c->stream = (cudaStream_t)stream;
    cudaGetDevice(&c->device);
    int num_sms = 0;
    if (cudaDeviceGetAttribute(&num_sms, cudaDevAttrMultiProcessorCount,
                               c->device) != cudaSuccess || num_sms < 1) {
        cudaGetLastError();
        num_sms = 148;
    }
    c->hpd.resize(npairs);
    c->gsink.assign(npairs, nullptr);
    for (int i = 0; i < npairs; ++i) {
        PairDesc& d = c->hpd[i];
        memset(&d, 0, sizeof(d));
        d.g.nx = fixed[i].W;
        d.g.ny = fixed[i].H;
        d.g.nz = fixed[i].D;
        d.g.V = (long long)fixed[i].W * fixed[i].H * fixed[i].D;
        d.F = fixed[i].data;
        d.M = moving[i].data;
    }
    BatchPlan plan = plan_batch(c->hpd.data(), npairs, prm.win, num_sms);
    c->num_sms = num_sms;
    // partial slots for the largest plan the autotuner may pick
    c->e1_cap = kMaxE1Waves * num_sms + npairs;
    c->e2_cap = kMaxE2Waves * num_sms + npairs;
    const size_t f4 = sizeof(float);
    const bool smooth = prm.sigma_warp > 0;
    // per-pair buffers
    DevState* st = nullptr;
    QScale* qs = nullptr;
    LogEntry* lg = nullptr;
    unsigned* flags = nullptr;
    if ((rc = c->dalloc(&st, npairs * sizeof(DevState))) ||
        (rc = c->dalloc(&flags, npairs * sizeof(unsigned))) ||
        (rc = c->dalloc(&qs, npairs * sizeof(QScale))) ||
        (rc = c->dalloc(&lg, npairs * sizeof(LogEntry) * LOG_CAP)) ||
        (rc = c->dalloc(&c->eout, npairs * sizeof(EvalOut))) ||
        (rc = c->dalloc(&c->dpd, npairs * sizeof(PairDesc))) ||
        (rc = c->dalloc(&c->b.part.loss, c->e1_cap * sizeof(long long))) ||
        (rc = c->dalloc(&c->b.part.g2max, c->e2_cap * sizeof(float))) ||
        (rc = c->dalloc(&c->b.mm_part,
                        (size_t)npairs * plan.mm_ctas * sizeof(float2))))
        return rc;
    for (int i = 0; i < npairs; ++i) {
        PairDesc& d = c->hpd[i];
        size_t V = (size_t)d.g.V;
        // jq and fq: halo-padded for the LNCC moment kernel
        const long long nq = set_q_layout(d, prm.win, prm.loss);
        if (nq > (1LL << 31) - 1)
            return fail(LM_EINVAL, "pair %d is too large for the padded "
                                   "fixed-point layout", i);
        if ((rc = c->dalloc(&d.u1, 3 * V * f4)) ||
            (rc = c->dalloc(&d.g0, 3 * V * f4)) ||
            (rc = c->dalloc(&d.g1, 3 * V * f4)) ||
            (rc = c->dalloc(&d.graw, graw_floats(d.g) * f4)) ||
            (rc = c->dalloc(&d.jq, (size_t)nq * sizeof(int))) ||
            (rc = c->dalloc(&d.dj, 3 * V * f4)) ||
            (rc = c->dalloc(&d.fq, (size_t)nq * sizeof(int))) ||
            (rc = c->dalloc(&d.fsum, V * sizeof(int))) ||
            (rc = c->dalloc(&d.fvar, V * f4)))
            return rc;
        if (smooth && ((rc = c->dalloc(&d.wtmpA, 3 * V * f4)) ||
                       (rc = c->dalloc(&d.wtmpB, 3 * V * f4))))
            return rc;
        d.tileH = nullptr;
        d.flags = flags + i;
        d.st = st + i;
        d.qs = qs + i;
        d.target = std::numeric_limits<double>::quiet_NaN();
        d.gp_w = graw_pitch(d.g.nx);
        d.log = lg + (size_t)i * LOG_CAP;
        d.u0 = nullptr;
        d.fault_wait = env_int("LM_FAULT_TIMEOUT") != 0;
    }
    // tensor maps of the g_raw buffers (E2 tiles them with TMA)
    {
        const int R = make_taps(prm.sigma_grad).R;
        std::vector<unsigned char> maps((size_t)npairs * 128);
        unsigned char* dmaps = nullptr;
        if ((rc = c->dalloc(&dmaps, maps.size())) != LM_OK) return rc;
        for (int i = 0; i < npairs; ++i) {
            PairDesc& d = c->hpd[i];
            if ((rc = encode_graw_map(maps.data() + 128 * i, d.graw, d.g, R)) != LM_OK)
                return rc;
            d.tm_graw = dmaps + 128 * i;
        }
        LM_CK(cudaMemcpy(dmaps, maps.data(), maps.size(), cudaMemcpyHostToDevice));
    }
    if (cudaMallocHost(&c->h_st, npairs * sizeof(DevState)) != cudaSuccess ||
        cudaMallocHost(&c->h_eout, npairs * sizeof(EvalOut)) != cudaSuccess ||
        cudaMallocHost(&c->h_log, LOG_CAP * sizeof(LogEntry)) != cudaSuccess) {
        cudaGetLastError();
        return fail(LM_ENOMEM, "pinned host allocation failed");
    }
    LM_CK(cudaMemsetAsync(st, 0, npairs * sizeof(DevState), c->stream));
    LM_CK(cudaMemsetAsync(flags, 0, npairs * sizeof(unsigned), c->stream));
    c->b.pd = c->dpd;
    c->b.npairs = npairs;
    c->b.dtype = c->dtype;
    c->b.plan = plan;
    c->b.c.win = prm.win;
    c->b.c.eps_nr = prm.eps_nr;
    c->b.c.eps_dr = prm.eps_dr;
    c->b.c.inv_k3 = (float)(1.0 / ((double)prm.win * prm.win * prm.win));
    c->b.c.gtaps = make_taps(prm.sigma_grad);
    c->b.d.lambda0 = prm.lambda0;
    c->b.d.mu_inc = prm.mu_inc;
    c->b.d.mu_dec = prm.mu_dec;
    c->b.d.lambda_max = prm.lambda_max;
    c->b.d.tau = prm.tau;
    c->b.d.reject = prm.reject;
    c->b.d.max_retries = prm.max_retries;
    c->b.d.mse = prm.loss == LM_LOSS_MSE;
    c->b.d.mi = prm.loss == LM_LOSS_MI;
    c->b.d.demons = prm.method == LM_METHOD_DEMONS;
    c->b.loss = prm.loss;
    c->b.method = prm.method;
    c->b.alpha = prm.alpha;
    c->b.bins = prm.bins;
    if (prm.loss == LM_LOSS_MI) {
        const size_t bb = (size_t)prm.bins * prm.bins;
        if ((rc = c->dalloc(&c->b.part.mi_hist,
                            npairs * bb * sizeof(unsigned long long))) ||
            (rc = c->dalloc(&c->b.part.mi_loss, npairs * sizeof(double))) ||
            (rc = c->dalloc(&c->b.part.mi_table, npairs * bb * sizeof(float))))
            return rc;
        // the histogram kernel adds to it; the table kernel clears it
        LM_CK(cudaMemsetAsync(c->b.part.mi_hist, 0,
                              npairs * bb * sizeof(unsigned long long),
                              c->stream));
    }
    c->b.wtaps = make_taps(prm.sigma_warp);
    c->b.step = prm.step;
    c->b.tile = prm.tile;
    c->b.th_blocks = 0;
    if (prm.tile > 1) {
        c->b.th_blocks = plan_tiles(c->hpd.data(), npairs, prm.tile);
        for (int i = 0; i < npairs; ++i) {
            PairDesc& d = c->hpd[i];
            const size_t nt = (size_t)d.th_nx * d.th_ny * d.th_nz;
            if ((rc = c->dalloc(&d.tileH, nt * 8 * f4)) != LM_OK) return rc;
        }
    }
    if ((rc = c->push_table()) != LM_OK) return rc;
    out = std::move(c);
    return LM_OK;
}

// Evaluation of explicit fields (no optimiser state change); losses and
// gmax to host.  Without g_out a pair's gradient goes to a sink volume
// allocated on first use.
int core_eval(Core* c, const float* const* u, float* const* g_out,
              double* loss, float* gmax) {
    for (int i = 0; i < c->npairs; ++i) {
        if (!is_device_ptr(u[i]))
            return fail(LM_EINVAL, "u of pair %d is not a device pointer", i);
        if (g_out && g_out[i] && !is_device_ptr(g_out[i]))
            return fail(LM_EINVAL, "g_out of pair %d is not a device pointer",
                        i);
    }
    int rc;
    for (int i = 0; i < c->npairs; ++i) {
        if ((g_out && g_out[i]) || c->gsink[i]) continue;
        if ((rc = c->dalloc(&c->gsink[i],
                            3 * (size_t)c->hpd[i].g.V * sizeof(float))) != LM_OK)
            return rc;
    }
    std::vector<PairDesc> save = c->hpd;
    for (int i = 0; i < c->npairs; ++i) {
        c->hpd[i].u_in = u[i];
        c->hpd[i].g_out = (g_out && g_out[i]) ? g_out[i] : c->gsink[i];
    }
    rc = c->push_table();
    if (rc != LM_OK) return rc;
    batch_prepare(c->b, c->stream);
    batch_eval(c->b, EVAL_EXPLICIT, 0, c->stream);
    batch_finalize(c->b, FIN_EXPLICIT, 0, c->eout, c->stream);
    LM_CK(cudaGetLastError());
    LM_CK(cudaMemcpyAsync(c->h_eout, c->eout, c->npairs * sizeof(EvalOut),
                          cudaMemcpyDeviceToHost, c->stream));
    LM_CK(cudaStreamSynchronize(c->stream));
    c->hpd = save;
    if ((rc = c->push_table()) != LM_OK) return rc;
    for (int i = 0; i < c->npairs; ++i) {
        if (loss) loss[i] = c->h_eout[i].L;
        if (gmax) gmax[i] = c->h_eout[i].gmax;
        if ((rc = status_error(c->h_eout[i].status, i)) != LM_OK) return rc;
    }
    return LM_OK;
}

int core_reset(Core* c, float* const* u) {
    for (int i = 0; i < c->npairs; ++i)
        if (!is_device_ptr(u[i]))
            return fail(LM_EINVAL, "u of pair %d is not a device pointer", i);
    for (int i = 0; i < c->npairs; ++i) c->hpd[i].u0 = u[i];
    int rc = c->push_table();
    if (rc != LM_OK) return rc;
    c->launches = batch_prepare(c->b, c->stream);
    c->launches += batch_eval(c->b, EVAL_RESET, 0, c->stream);
    c->launches += batch_finalize(c->b, FIN_RESET, 0, nullptr, c->stream);
    LM_CK(cudaGetLastError());
    c->have_reset = true;
    return LM_OK;
}

int core_check_bound(Core* c, float* const* u) {
    if (!c->have_reset) return fail(LM_ESTATE, "lm_reset was not called");
    for (int i = 0; i < c->npairs; ++i)
        if (u[i] != c->hpd[i].u0)
            return fail(LM_ESTATE,
                        "u of pair %d is not the field passed to reset", i);
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
    info->stopped = s.stopped;
}

}  // namespace

struct lm_ctx {
    std::unique_ptr<Core> core;
    // coarse levels for lm_register (factor -> context), built lazily
    struct Level {
        int factor = 0;
        lm_ctx* ctx = nullptr;
        void* Fl = nullptr;
        void* Ml = nullptr;
        float* ul = nullptr;
        bool tuned = false;        // work split autotuned
    };
    std::vector<Level> levels;
    float* u_tmp = nullptr;      // full-res staging (3V floats)
    ~lm_ctx();
};

struct lm_batch {
    std::unique_ptr<Core> core;
    struct Level {
        int factor = 0;
        lm_batch* b = nullptr;
        std::vector<void*> Fl, Ml;
        std::vector<float*> ul;
    };
    std::vector<Level> levels;
    std::vector<float*> u_tmp;
    ~lm_batch();
};

lm_ctx::~lm_ctx() {
    for (auto& l : levels) lm_destroy(l.ctx);
}

lm_batch::~lm_batch() {
    for (auto& l : levels) lm_batch_destroy(l.b);
}

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
    p->tile = 1;
    p->loss = LM_LOSS_LNCC;
    p->method = LM_METHOD_LM;
    p->alpha = 1.f;
    p->bins = 32;
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
        case LM_EBOUNDS: return "a kernel wrote outside its buffer";
        case LM_EUNSUPPORTED: return "unsupported";
        case LM_ESTATE: return "call out of order";
        default: return "unknown error";
    }
}

const char* lm_last_error(void) { return g_err; }

static_assert(LM_LOG_CAP == LOG_CAP, "device log ring and public cap");

int lm_get_log(lm_ctx* c, lm_log_entry* out, int cap, int* n) {
    if (!c || !n) return fail(LM_EINVAL, "NULL argument");
    if (out && cap < 0) return fail(LM_EINVAL, "cap must be >= 0");
    Core* k = c->core.get();
    LM_CK(cudaMemcpyAsync(k->h_st, k->hpd[0].st, sizeof(DevState),
                          cudaMemcpyDeviceToHost, k->stream));
    LM_CK(cudaStreamSynchronize(k->stream));
    const int pos = k->h_st[0].log_pos;
    const int avail = pos < LOG_CAP ? pos : LOG_CAP;
    if (!out) {
        *n = avail;
        return LM_OK;
    }
    const int m = cap < avail ? cap : avail;
    if (m > 0) {
        LM_CK(cudaMemcpy(k->h_log, k->hpd[0].log, LOG_CAP * sizeof(LogEntry),
                         cudaMemcpyDeviceToHost));
        for (int i = 0; i < m; ++i) {
            const LogEntry& e = k->h_log[(pos - m + i) % LOG_CAP];
            out[i].loss = e.loss;
            out[i].lambda = e.lambda;
            out[i].gmax = e.gmax;
            out[i].accepted = e.accepted;
            out[i].retries = e.retries;
        }
    }
    *n = m;
    return LM_OK;
}

int lm_debug_check(lm_ctx* c) {
    if (!c) return fail(LM_EINVAL, "ctx is NULL");
    int rc = c->core->check_guards();
    for (auto& l : c->levels)
        if (rc == LM_OK && l.ctx) rc = lm_debug_check(l.ctx);
    return rc;
}

void lm_destroy(lm_ctx* c) {
    if (!c) return;
    delete c;   // the Core's destructor synchronises and frees
}

int lm_init(lm_ctx** out, const lm_volume* fixed, const lm_volume* moving,
            const lm_params* p, void* cuda_stream) {
    g_err[0] = 0;
    if (!out) return fail(LM_EINVAL, "ctx out-pointer is NULL");
    *out = nullptr;
    auto c = new lm_ctx();
    int rc = core_create(c->core, 1, fixed, moving, p, cuda_stream);
    if (rc != LM_OK) {
        delete c;
        return rc;
    }
    *out = c;
    return LM_OK;
}

int lm_eval(lm_ctx* c, const float* u, double* loss, float* g_out,
            float* gmax) {
    if (!c) return fail(LM_EINVAL, "ctx is NULL");
    float* gs[1] = {g_out};
    return core_eval(c->core.get(), &u, g_out ? gs : nullptr, loss, gmax);
}

int lm_reset(lm_ctx* c, float* u) {
    if (!c) return fail(LM_EINVAL, "ctx is NULL");
    return core_reset(c->core.get(), &u);
}

int lm_step(lm_ctx* c, float* u, lm_step_info* info) {
    if (!c) return fail(LM_EINVAL, "ctx is NULL");
    Core* k = c->core.get();
    int rc = core_check_bound(k, &u);
    if (rc) return rc;
    k->launches += k->enqueue_iteration(k->stream);
    k->launches += batch_sync_back(k->b, k->stream);
    LM_CK(cudaGetLastError());
    if (info) {
        if ((rc = k->read_states()) != LM_OK) return rc;
        fill_info(k->h_st[0], info);
    }
    return LM_OK;
}

int lm_iterate(lm_ctx* c, float* u, int n, lm_step_info* info) {
    if (!c) return fail(LM_EINVAL, "ctx is NULL");
    Core* k = c->core.get();
    int rc = core_check_bound(k, &u);
    if (rc) return rc;
    if (n < 0) return fail(LM_EINVAL, "n must be >= 0");
    if ((rc = k->iterate(n)) != LM_OK) return rc;
    if (info) {
        if ((rc = k->read_states()) != LM_OK) return rc;
        fill_info(k->h_st[0], info);
    }
    return LM_OK;
}

int lm_get_state(lm_ctx* c, lm_state* out) {
    if (!c || !out) return fail(LM_EINVAL, "NULL argument");
    Core* k = c->core.get();
    LM_CK(cudaMemcpyAsync(k->h_st, k->hpd[0].st, sizeof(DevState),
                          cudaMemcpyDeviceToHost, k->stream));
    LM_CK(cudaStreamSynchronize(k->stream));
    const DevState& s = k->h_st[0];
    out->loss = s.L;
    out->loss_prev = s.L_prev;
    out->lambda = s.lambda;
    out->gmax = s.gmax;
    out->has_prev = s.has_prev;
    out->iter = s.iter;
    out->evals = s.evals;
    out->kernel_launches = k->launches;
    return LM_OK;
}

int lm_set_state(lm_ctx* c, const lm_state* in) {
    if (!c || !in) return fail(LM_EINVAL, "NULL argument");
    Core* k = c->core.get();
    if (!k->have_reset) return fail(LM_ESTATE, "lm_reset was not called");
    if (!(in->lambda > 0) || !std::isfinite(in->lambda) ||
        !std::isfinite(in->loss) || !std::isfinite(in->loss_prev))
        return fail(LM_EINVAL, "state scalars must be finite, lambda > 0");
    LM_CK(cudaMemcpyAsync(k->h_st, k->hpd[0].st, sizeof(DevState),
                          cudaMemcpyDeviceToHost, k->stream));
    LM_CK(cudaStreamSynchronize(k->stream));
    DevState s = k->h_st[0];
    s.L = in->loss;
    s.L_prev = in->loss_prev;
    s.lambda = in->lambda;
    s.gmax = in->gmax;
    s.has_prev = in->has_prev ? 1 : 0;
    s.iter = in->iter;
    s.evals = in->evals;
    k->h_st[0] = s;
    LM_CK(cudaMemcpyAsync(k->hpd[0].st, k->h_st, sizeof(DevState),
                          cudaMemcpyHostToDevice, k->stream));
    LM_CK(cudaStreamSynchronize(k->stream));
    return LM_OK;
}

int lm_time_passes(lm_ctx* c, float* u, int n, double* ms_eval,
                   double* ms_step) {
    if (!c) return fail(LM_EINVAL, "ctx is NULL");
    Core* k = c->core.get();
    int rc = core_check_bound(k, &u);
    if (rc) return rc;
    if (n < 1 || !ms_eval || !ms_step)
        return fail(LM_EINVAL, "n must be >= 1 and outputs non-NULL");
    cudaEvent_t e0, e1, e2;
    LM_CK(cudaEventCreate(&e0));
    LM_CK(cudaEventCreate(&e1));
    LM_CK(cudaEventCreate(&e2));
    LM_CK(cudaEventRecord(e0, k->stream));
    for (int i = 0; i < n; ++i) batch_step(k->b, 0, k->stream);
    LM_CK(cudaEventRecord(e1, k->stream));
    for (int i = 0; i < n; ++i)
        batch_eval(k->b, EVAL_TRIAL, 0, k->stream, !step_resamples(k->b));
    LM_CK(cudaEventRecord(e2, k->stream));
    LM_CK(cudaEventSynchronize(e2));
    float a = 0.f, bb = 0.f;
    cudaEventElapsedTime(&a, e0, e1);
    cudaEventElapsedTime(&bb, e1, e2);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaEventDestroy(e2);
    *ms_step = a / n;
    *ms_eval = bb / n;
    LM_CK(cudaGetLastError());
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
    Core* k = c->core.get();
    if (!k->have_reset) return fail(LM_ESTATE, "lm_reset was not called");
    const PairDesc& d = k->hpd[0];
    size_t need = sizeof(CkptHeader) + sizeof(DevState) +
                  3 * (size_t)d.g.V * sizeof(float);
    if (!buf) {
        *nbytes = need;
        return LM_OK;
    }
    if (*nbytes < need) return fail(LM_EINVAL, "buffer too small");
    // make sure the field sits in the caller's slot
    batch_sync_back(k->b, k->stream);
    LM_CK(cudaMemcpyAsync(k->h_st, d.st, sizeof(DevState),
                          cudaMemcpyDeviceToHost, k->stream));
    LM_CK(cudaStreamSynchronize(k->stream));
    CkptHeader h;
    memcpy(h.magic, "LMREGCK1", 8);
    h.nx = d.g.nx;
    h.ny = d.g.ny;
    h.nz = d.g.nz;
    h.version = 3;
    char* q = (char*)buf;
    memcpy(q, &h, sizeof(h));
    memcpy(q + sizeof(h), k->h_st, sizeof(DevState));
    LM_CK(cudaMemcpy(q + sizeof(h) + sizeof(DevState),
                     k->h_st[0].cg ? d.g1 : d.g0,
                     3 * (size_t)d.g.V * sizeof(float),
                     cudaMemcpyDeviceToHost));
    *nbytes = need;
    return LM_OK;
}

extern "C" int lm_state_load(lm_ctx* c, const void* buf, size_t nbytes) {
    if (!c || !buf) return fail(LM_EINVAL, "NULL argument");
    Core* k = c->core.get();
    if (!k->have_reset) return fail(LM_ESTATE, "lm_reset was not called");
    const PairDesc& d = k->hpd[0];
    size_t need = sizeof(CkptHeader) + sizeof(DevState) +
                  3 * (size_t)d.g.V * sizeof(float);
    if (nbytes < need) return fail(LM_EINVAL, "checkpoint too small");
    CkptHeader h;
    memcpy(&h, buf, sizeof(h));
    if (memcmp(h.magic, "LMREGCK1", 8) != 0 || h.version != 3)
        return fail(LM_EINVAL, "not an lmreg checkpoint");
    if (h.nx != d.g.nx || h.ny != d.g.ny || h.nz != d.g.nz)
        return fail(LM_EINVAL, "checkpoint shape differs from the context");
    DevState s;
    memcpy(&s, (const char*)buf + sizeof(h), sizeof(DevState));
    s.cu = 0;       // the field is the caller's (slot 0)
    s.cg = 0;       // the gradient is restored into slot 0
    s.done = 0;
    s.att = 0;
    s.iter_end = 0;
    k->h_st[0] = s;
    LM_CK(cudaMemcpyAsync(d.st, k->h_st, sizeof(DevState),
                          cudaMemcpyHostToDevice, k->stream));
    LM_CK(cudaMemcpyAsync(d.g0, (const char*)buf + sizeof(h) + sizeof(DevState),
                          3 * (size_t)d.g.V * sizeof(float),
                          cudaMemcpyHostToDevice, k->stream));
    LM_CK(cudaStreamSynchronize(k->stream));
    return LM_OK;
}

// ---------------------------------------------------------------------
// Coarse-to-fine registration.
// ---------------------------------------------------------------------
namespace {

int core_autotune(Core* c, const float* const* u, int reps, int* e1_tile,
                  int* e1_waves, int* e2_waves, double* ms_best);

int check_schedule(const lm_schedule* s) {
    if (!s) return fail(LM_EINVAL, "schedule is NULL");
    if (s->nlevels < 1 || s->nlevels > LM_MAX_LEVELS)
        return fail(LM_EINVAL, "nlevels must be in [1, %d]", LM_MAX_LEVELS);
    for (int l = 0; l < s->nlevels; ++l) {
        int f = s->factor[l];
        if (f != 1 && f != 2 && f != 4)
            return fail(LM_EINVAL, "factor[%d] must be 1, 2 or 4", l);
        if (s->iters[l] < 0) return fail(LM_EINVAL, "iters[%d] < 0", l);
    }
    return LM_OK;
}

// Per-level accounting from a Core's state and log after a level's run.
int level_report(Core* k, int pair, lm_report* r, int l) {
    const DevState& hs = k->h_st[pair];
    const PairDesc& d = k->hpd[pair];
    r->level_dims[l][0] = d.g.nz;
    r->level_dims[l][1] = d.g.ny;
    r->level_dims[l][2] = d.g.nx;
    r->level_iters[l] = hs.iter;
    r->level_evals[l] = hs.evals;
    r->level_accepted[l] = 0;
    int nlog = hs.log_pos < LOG_CAP ? hs.log_pos : LOG_CAP;
    if (nlog > 0) {
        LM_CK(cudaMemcpy(k->h_log, d.log, nlog * sizeof(LogEntry),
                         cudaMemcpyDeviceToHost));
        for (int i = 0; i < nlog; ++i)
            r->level_accepted[l] += k->h_log[i].accepted;
    }
    r->level_loss[l] = hs.L;
    r->voxel_evals += (long long)d.g.V * hs.evals;
    return LM_OK;
}

}  // namespace

extern "C" int lm_register(lm_ctx* c, const lm_schedule* s, float* u,
                           lm_report* rep) {
    if (!c) return fail(LM_EINVAL, "NULL argument");
    int rc = check_schedule(s);
    if (rc) return rc;
    if (!is_device_ptr(u)) return fail(LM_EINVAL, "u is not a device pointer");
    Core* top = c->core.get();
    const PairDesc td = top->hpd[0];
    const Geom G = td.g;
    auto t0 = std::chrono::steady_clock::now();
    if (!c->u_tmp) {
        if ((rc = top->dalloc(&c->u_tmp, 3 * (size_t)G.V * sizeof(float))) !=
            LM_OK)
            return rc;
    }
    lm_report r;
    memset(&r, 0, sizeof(r));
    r.nlevels = s->nlevels;
    float* cur = u;
    Geom cg = G;
    int cf = 1;
    for (int l = 0; l < s->nlevels; ++l) {
        const int f = s->factor[l];
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
                level_dims(G.nx, G.ny, G.nz, f, &lx, &ly, &lz);
                size_t Vl = (size_t)lx * ly * lz;
                size_t es = top->dtype == LM_BF16 ? 2 : 4;
                if ((rc = top->dalloc(&nl.Fl, Vl * es)) ||
                    (rc = top->dalloc(&nl.Ml, Vl * es)) ||
                    (rc = top->dalloc(&nl.ul, 3 * Vl * sizeof(float))))
                    return rc;
                lm_volume vf = {lz, ly, lx, top->dtype, nl.Fl};
                lm_volume vm = {lz, ly, lx, top->dtype, nl.Ml};
                if ((rc = lm_init(&nl.ctx, &vf, &vm, &top->p, top->stream)))
                    return rc;
                c->levels.push_back(nl);
                lv = &c->levels.back();
            }
            // the caller may change F or M between calls: resample each time
            if (downsample_image(td.F, top->dtype, G, f, lv->Fl, c->u_tmp,
                                 top->stream) ||
                downsample_image(td.M, top->dtype, G, f, lv->Ml, c->u_tmp,
                                 top->stream))
                return fail(LM_ECUDA, "downsample failed");
            lc = lv->ctx;
            ul = lv->ul;
        }
        const Geom lg = lc->core->hpd[0].g;
        if (ul != cur || cf != f) {
            float* src = cur;
            if (ul == cur) {   // resample in place through the staging copy
                LM_CK(cudaMemcpyAsync(c->u_tmp, cur, 3 * cg.V * sizeof(float),
                                      cudaMemcpyDeviceToDevice, top->stream));
                src = c->u_tmp;
            }
            if (resample_field(src, cg, cf, ul, lg, f, top->stream))
                return fail(LM_ECUDA, "field resampling failed");
        }
        Core* k = lc->core.get();
        if (f != 1) {
            // a coarse level's context is tuned once, when first used: its
            // volumes are small enough for the work split to decide the time
            lm_ctx::Level* lv = nullptr;
            for (auto& x : c->levels)
                if (x.factor == f) lv = &x;
            if (lv && !lv->tuned) {
                if ((rc = core_autotune(k, &ul, 2, nullptr, nullptr, nullptr,
                                        nullptr)) != LM_OK)
                    return rc;
                lv->tuned = true;
            }
        }
        if ((rc = core_reset(k, &ul)) != LM_OK) return rc;
        if ((rc = k->iterate(s->iters[l])) != LM_OK) return rc;
        if ((rc = k->read_states()) != LM_OK) return rc;
        if ((rc = level_report(k, 0, &r, l)) != LM_OK) return rc;
        cur = ul;
        cg = lg;
        cf = f;
    }
    if (cur != u) {
        if (resample_field(cur, cg, cf, u, G, 1, top->stream))
            return fail(LM_ECUDA, "field resampling failed");
    }
    LM_CK(cudaStreamSynchronize(top->stream));
    r.final_loss = r.level_loss[s->nlevels - 1];
    auto t1 = std::chrono::steady_clock::now();
    r.wall_ms = std::chrono::duration<double, std::milli>(t1 - t0).count();
    if (rep) *rep = r;
    return LM_OK;
}

// ---------------------------------------------------------------------
// Batches of pairs.
// ---------------------------------------------------------------------
extern "C" int lm_batch_init(lm_batch** out, int npairs,
                             const lm_volume* fixed, const lm_volume* moving,
                             const lm_params* p, void* cuda_stream) {
    g_err[0] = 0;
    if (!out) return fail(LM_EINVAL, "batch out-pointer is NULL");
    *out = nullptr;
    auto b = new lm_batch();
    int rc = core_create(b->core, npairs, fixed, moving, p, cuda_stream);
    if (rc != LM_OK) {
        delete b;
        return rc;
    }
    *out = b;
    return LM_OK;
}

extern "C" int lm_batch_debug_check(lm_batch* b) {
    if (!b) return fail(LM_EINVAL, "batch is NULL");
    int rc = b->core->check_guards();
    for (auto& l : b->levels)
        if (rc == LM_OK && l.b) rc = lm_batch_debug_check(l.b);
    return rc;
}

extern "C" void lm_batch_destroy(lm_batch* b) {
    if (!b) return;
    delete b;
}

extern "C" int lm_batch_eval(lm_batch* b, const float* const* u,
                             float* const* g_out, double* loss,
                             float* gmax) {
    if (!b || !u) return fail(LM_EINVAL, "NULL argument");
    return core_eval(b->core.get(), u, g_out, loss, gmax);
}

extern "C" int lm_batch_reset(lm_batch* b, float* const* u) {
    if (!b || !u) return fail(LM_EINVAL, "NULL argument");
    return core_reset(b->core.get(), u);
}

extern "C" int lm_batch_iterate(lm_batch* b, float* const* u, int n,
                                lm_step_info* infos) {
    if (!b || !u) return fail(LM_EINVAL, "NULL argument");
    Core* k = b->core.get();
    int rc = core_check_bound(k, u);
    if (rc) return rc;
    if (n < 0) return fail(LM_EINVAL, "n must be >= 0");
    if ((rc = k->iterate(n)) != LM_OK) return rc;
    if (infos) {
        if ((rc = k->read_states()) != LM_OK) return rc;
        for (int i = 0; i < k->npairs; ++i) fill_info(k->h_st[i], &infos[i]);
    }
    return LM_OK;
}

namespace {
// Re-split the evaluation kernels' CTAs with the given wave counts and
// moment-kernel tile; the captured iteration graph is dropped (its grids
// change).
int core_replan(Core* c, int e1w, int e2w, int tile, int min_slices,
                int st_target) {
    BatchPlan plan = plan_batch(c->hpd.data(), c->npairs, c->p.win, c->num_sms,
                                e1w, e2w, tile, min_slices, st_target);

    if (plan.e1_ctas > c->e1_cap || plan.e2_ctas > c->e2_cap)
        return fail(LM_EINVAL, "plan exceeds the partial slots");
    c->b.plan = plan;
    c->drop_graphs();
    return c->push_table();
}

// Times reps evaluations at u for every candidate (moment-kernel tile, E1
// waves, E2 waves) and keeps the fastest plan.
int core_autotune(Core* c, const float* const* u, int reps, int* e1_tile,
                  int* e1_waves, int* e2_waves, double* ms_best) {
    if (!u) return fail(LM_EINVAL, "NULL argument");
    if (reps < 1) return fail(LM_EINVAL, "reps must be >= 1");
    int rc;
    for (int i = 0; i < c->npairs; ++i)
        if (!is_device_ptr(u[i]))
            return fail(LM_EINVAL, "u of pair %d is not a device pointer", i);
    for (int i = 0; i < c->npairs; ++i) {
        if (c->gsink[i]) continue;
        if ((rc = c->dalloc(&c->gsink[i],
                            3 * (size_t)c->hpd[i].g.V * sizeof(float))) != LM_OK)
            return rc;
    }
    std::vector<PairDesc> save = c->hpd;
    for (int i = 0; i < c->npairs; ++i) {
        c->hpd[i].u_in = u[i];
        c->hpd[i].g_out = c->gsink[i];
        // the trial passes read the current field: before any lm_reset
        // there is none bound, so the tuning field stands in (between API
        // calls the current field is always in slot 0 and the trial goes
        // to the library's slot 1)
        if (!c->hpd[i].u0)   // only read: with no reset the trial slot is 1
            c->hpd[i].u0 = const_cast<float*>(u[i]);
    }
    if ((rc = c->push_table()) != LM_OK) return rc;
    batch_prepare(c->b, c->stream);
    cudaEvent_t e0, e1;
    LM_CK(cudaEventCreate(&e0));
    LM_CK(cudaEventCreate(&e1));
    double best = 1e300;
    int bt = c->b.plan.e1_tile, b1 = 0, b2 = 0, bm = 8;
    const int bs = c->b.plan.st_target;
    // the tile only matters to the LNCC moment kernel
    const int ntiles = c->p.loss == LM_LOSS_LNCC ? E1_NTILES : 1;
    for (int t = 0; t < ntiles && rc == LM_OK; ++t) {
        if (!e1_tile_ok(t, c->p.win)) continue;
        for (int mn : kMinSlices)
        for (int w1 : kE1Waves)
            for (int w2 : kE2Waves) {
                if ((rc = core_replan(c, w1, w2, t, mn, bs)) != LM_OK) break;
                batch_eval(c->b, EVAL_EXPLICIT, 0, c->stream);   // warm-up
                LM_CK(cudaEventRecord(e0, c->stream));
                for (int r = 0; r < reps; ++r)
                    batch_eval(c->b, EVAL_EXPLICIT, 0, c->stream);
                LM_CK(cudaEventRecord(e1, c->stream));
                LM_CK(cudaEventSynchronize(e1));
                float ms = 0.f;
                cudaEventElapsedTime(&ms, e0, e1);
                if (ms / reps < best) {
                    best = ms / reps;
                    bt = t;
                    b1 = w1;
                    b2 = w2;
                    bm = mn;
                }
            }
    }
    // then the step kernel's z chunking, timed on its own (it writes only
    // the trial slot and the resampling scratch, which the next iteration
    // recomputes)
    int bsb = bs;
    if (rc == LM_OK && !c->have_reset) {
        // no gradient computed yet: a zero step (the trial reads u from
        // shared memory, as the usual sub-voxel steps do)
        for (int i = 0; i < c->npairs; ++i) {
            LM_CK(cudaMemsetAsync(c->hpd[i].g0, 0,
                                  3 * (size_t)c->hpd[i].g.V * sizeof(float),
                                  c->stream));
            LM_CK(cudaMemsetAsync(c->hpd[i].g1, 0,
                                  3 * (size_t)c->hpd[i].g.V * sizeof(float),
                                  c->stream));
        }
    }
    if (rc == LM_OK) {
        double bst = 1e300;
        for (int st : kStepBlocks) {
            if ((rc = core_replan(c, b1, b2, bt, bm, st)) != LM_OK) break;
            batch_step(c->b, 0, c->stream);   // warm-up
            LM_CK(cudaEventRecord(e0, c->stream));
            for (int r = 0; r < reps; ++r) batch_step(c->b, 0, c->stream);
            LM_CK(cudaEventRecord(e1, c->stream));
            LM_CK(cudaEventSynchronize(e1));
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (ms / reps < bst) {
                bst = ms / reps;
                bsb = st;
            }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc != LM_OK) return rc;
    // restore the table's pointers, keep the chosen plan
    c->hpd = save;
    if ((rc = core_replan(c, b1, b2, bt, bm, bsb)) != LM_OK) return rc;
    LM_CK(cudaStreamSynchronize(c->stream));
    LM_CK(cudaGetLastError());
    if (e1_tile) *e1_tile = bt;
    if (e1_waves) *e1_waves = b1;
    if (e2_waves) *e2_waves = b2;
    if (ms_best) *ms_best = best;
    return LM_OK;
}
}  // namespace

extern "C" int lm_batch_autotune(lm_batch* b, float* const* u, int reps,
                                 int* e1_tile, int* e1_waves, int* e2_waves,
                                 double* ms_best) {
    if (!b) return fail(LM_EINVAL, "NULL argument");
    return core_autotune(b->core.get(), u, reps, e1_tile, e1_waves, e2_waves,
                         ms_best);
}

extern "C" int lm_autotune(lm_ctx* c, const float* u, int reps, int* e1_tile,
                           int* e1_waves, int* e2_waves, double* ms_best) {
    if (!c) return fail(LM_EINVAL, "NULL argument");
    return core_autotune(c->core.get(), &u, reps, e1_tile, e1_waves, e2_waves,
                         ms_best);
}

extern "C" int lm_field_resample(const float* src, int Da, int Ha, int Wa,
                                 int fa, float* dst, int Db, int Hb, int Wb,
                                 int fb, void* stream) {
    if (!src || !dst) return fail(LM_EINVAL, "NULL field");
    if (Da < 1 || Ha < 1 || Wa < 1 || Db < 1 || Hb < 1 || Wb < 1 || fa < 1 ||
        fb < 1)
        return fail(LM_EINVAL, "sizes and factors must be positive");
    Geom ga{Wa, Ha, Da, (long long)Wa * Ha * Da};
    Geom gb{Wb, Hb, Db, (long long)Wb * Hb * Db};
    resample_field(src, ga, fa, dst, gb, fb, (cudaStream_t)stream);
    LM_CK(cudaGetLastError());
    return LM_OK;
}

extern "C" int lm_downsample(const lm_volume* src, int factor, void* dst,
                             float* tmp, int* dims, void* stream) {
    int rc = check_volume(src, "src");
    if (rc != LM_OK) return rc;
    if (factor != 2 && factor != 4)
        return fail(LM_EINVAL, "factor must be 2 or 4, got %d", factor);
    if (!is_device_ptr(src->data) || !is_device_ptr(dst) ||
        !is_device_ptr(tmp))
        return fail(LM_EINVAL, "src data, dst and tmp must be device pointers");
    const Geom g{src->W, src->H, src->D, (long long)src->W * src->H * src->D};
    int lx, ly, lz;
    level_dims(g.nx, g.ny, g.nz, factor, &lx, &ly, &lz);
    if (downsample_image(src->data, src->dtype, g, factor, dst, tmp,
                         (cudaStream_t)stream))
        return fail(LM_ECUDA, "downsample failed: %s",
                    cudaGetErrorString(cudaGetLastError()));
    if (dims) {
        dims[0] = lz;
        dims[1] = ly;
        dims[2] = lx;
    }
    return LM_OK;
}

extern "C" int lm_batch_set_targets(lm_batch* b, const double* target) {
    if (!b) return fail(LM_EINVAL, "NULL argument");
    Core* k = b->core.get();
    for (int i = 0; i < k->npairs; ++i)
        k->hpd[i].target =
            target ? target[i] : std::numeric_limits<double>::quiet_NaN();
    return k->push_table();
}

extern "C" int lm_batch_register(lm_batch* b, const lm_schedule* s,
                                 float* const* u, lm_report* reps) {
    if (!b || !u) return fail(LM_EINVAL, "NULL argument");
    int rc = check_schedule(s);
    if (rc) return rc;
    Core* top = b->core.get();
    const int n = top->npairs;
    for (int i = 0; i < n; ++i)
        if (!is_device_ptr(u[i]))
            return fail(LM_EINVAL, "u of pair %d is not a device pointer", i);
    auto t0 = std::chrono::steady_clock::now();
    if (b->u_tmp.empty()) {
        b->u_tmp.resize(n);
        for (int i = 0; i < n; ++i)
            if ((rc = top->dalloc(&b->u_tmp[i], 3 * (size_t)top->hpd[i].g.V *
                                                    sizeof(float))) != LM_OK)
                return rc;
    }
    std::vector<lm_report> r(n);
    for (auto& x : r) {
        memset(&x, 0, sizeof(x));
        x.nlevels = s->nlevels;
    }
    std::vector<float*> cur(u, u + n);
    std::vector<Geom> cg(n);
    for (int i = 0; i < n; ++i) cg[i] = top->hpd[i].g;
    int cf = 1;
    for (int l = 0; l < s->nlevels; ++l) {
        const int f = s->factor[l];
        lm_batch* lb = b;
        std::vector<float*> ul(u, u + n);
        if (f != 1) {
            lm_batch::Level* lv = nullptr;
            for (auto& x : b->levels)
                if (x.factor == f) lv = &x;
            if (!lv) {
                lm_batch::Level nl;
                nl.factor = f;
                std::vector<lm_volume> vf(n), vm(n);
                size_t es = top->dtype == LM_BF16 ? 2 : 4;
                nl.Fl.resize(n);
                nl.Ml.resize(n);
                nl.ul.resize(n);
                for (int i = 0; i < n; ++i) {
                    const Geom& G = top->hpd[i].g;
                    int lx, ly, lz;
                    level_dims(G.nx, G.ny, G.nz, f, &lx, &ly, &lz);
                    size_t Vl = (size_t)lx * ly * lz;
                    if ((rc = top->dalloc(&nl.Fl[i], Vl * es)) ||
                        (rc = top->dalloc(&nl.Ml[i], Vl * es)) ||
                        (rc = top->dalloc(&nl.ul[i], 3 * Vl * sizeof(float))))
                        return rc;
                    vf[i] = {lz, ly, lx, top->dtype, nl.Fl[i]};
                    vm[i] = {lz, ly, lx, top->dtype, nl.Ml[i]};
                }
                // the level images must exist before the batch checks them
                for (int i = 0; i < n; ++i) {
                    const PairDesc& d = top->hpd[i];
                    if (downsample_image(d.F, top->dtype, d.g, f, nl.Fl[i],
                                         b->u_tmp[i], top->stream) ||
                        downsample_image(d.M, top->dtype, d.g, f, nl.Ml[i],
                                         b->u_tmp[i], top->stream))
                        return fail(LM_ECUDA, "downsample failed");
                }
                if ((rc = lm_batch_init(&nl.b, n, vf.data(), vm.data(),
                                        &top->p, top->stream)))
                    return rc;
                b->levels.push_back(nl);
                lv = &b->levels.back();
            } else {
                for (int i = 0; i < n; ++i) {
                    const PairDesc& d = top->hpd[i];
                    if (downsample_image(d.F, top->dtype, d.g, f, lv->Fl[i],
                                         b->u_tmp[i], top->stream) ||
                        downsample_image(d.M, top->dtype, d.g, f, lv->Ml[i],
                                         b->u_tmp[i], top->stream))
                        return fail(LM_ECUDA, "downsample failed");
                }
            }
            lb = lv->b;
            ul = lv->ul;
        }
        Core* k = lb->core.get();
        for (int i = 0; i < n; ++i) {
            const Geom lg = k->hpd[i].g;
            if (ul[i] != cur[i] || cf != f) {
                float* src = cur[i];
                if (ul[i] == cur[i]) {
                    LM_CK(cudaMemcpyAsync(b->u_tmp[i], cur[i],
                                          3 * cg[i].V * sizeof(float),
                                          cudaMemcpyDeviceToDevice,
                                          top->stream));
                    src = b->u_tmp[i];
                }
                if (resample_field(src, cg[i], cf, ul[i], lg, f, top->stream))
                    return fail(LM_ECUDA, "field resampling failed");
            }
        }
        if ((rc = core_reset(k, ul.data())) != LM_OK) return rc;
        if ((rc = k->iterate(s->iters[l])) != LM_OK) return rc;
        if ((rc = k->read_states()) != LM_OK) return rc;
        for (int i = 0; i < n; ++i)
            if ((rc = level_report(k, i, &r[i], l)) != LM_OK) return rc;
        for (int i = 0; i < n; ++i) {
            cur[i] = ul[i];
            cg[i] = k->hpd[i].g;
        }
        cf = f;
    }
    for (int i = 0; i < n; ++i)
        if (cur[i] != u[i]) {
            if (resample_field(cur[i], cg[i], cf, u[i], top->hpd[i].g, 1,
                               top->stream))
                return fail(LM_ECUDA, "field resampling failed");
        }
    LM_CK(cudaStreamSynchronize(top->stream));
    auto t1 = std::chrono::steady_clock::now();
    double ms = std::chrono::duration<double, std::milli>(t1 - t0).count();
    for (int i = 0; i < n; ++i) {
        r[i].final_loss = r[i].level_loss[s->nlevels - 1];
        r[i].wall_ms = ms;
        if (reps) reps[i] = r[i];
    }
    return LM_OK;
}

extern "C" int lm_register_batch(int npairs, const lm_volume* fixed,
                                 const lm_volume* moving, float* const* u,
                                 const lm_params* p, const lm_schedule* s,
                                 void* cuda_stream, lm_report* reps) {
    lm_batch* b = nullptr;
    int rc = lm_batch_init(&b, npairs, fixed, moving, p, cuda_stream);
    if (rc != LM_OK) return rc;
    rc = lm_batch_register(b, s, u, reps);
    lm_batch_destroy(b);
    return rc;
}
