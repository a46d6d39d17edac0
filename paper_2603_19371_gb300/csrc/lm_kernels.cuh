// Launch interfaces of the CUDA kernels (internal).
#pragma once

#include "lm_internal.cuh"

namespace lmk {

// Field / gradient routing of one evaluation (see EvalMode).
struct EvalIO {
    const float* u_in;  // EVAL_EXPLICIT field
    float* g_out;       // EVAL_EXPLICIT gradient (may be a scratch buffer)
    float* u0;          // field slot 0 (the caller's field)
    float* u1;          // field slot 1 (context scratch)
    float* g0;          // gradient slots
    float* g1;
    const DevState* st;
    int mode;
    int attempt;        // trial attempt index within an iteration
};

__device__ __forceinline__ bool eval_skip(const EvalIO& io) {
    return io.mode == EVAL_TRIAL && io.attempt > 0 && io.st->done;
}
__device__ __forceinline__ const float* eval_u(const EvalIO& io) {
    if (io.mode == EVAL_EXPLICIT) return io.u_in;
    if (io.mode == EVAL_RESET) return io.u0;
    return io.st->cu ? io.u0 : io.u1;
}
__device__ __forceinline__ float* eval_g(const EvalIO& io) {
    if (io.mode == EVAL_EXPLICIT) return io.g_out;
    if (io.mode == EVAL_RESET) return io.g0;
    return io.st->cg ? io.g0 : io.g1;
}

// Per-CTA partial results of an evaluation, reduced by the finalize kernel.
struct Partials {
    double* loss;     // sum over the CTA's voxels of (1 - cc)
    int n_loss;
    float* g2max;     // max over the CTA's voxels of |g|^2
    int n_g2;
};

// Staged scratch (one full volume per intermediate).
struct StagedScratch {
    float* J;     // V
    float* dJ;    // 3V
    float* S;     // 5V box sums
    float* T;     // 5V separable temp
    float* abc;   // 3V
    float* graw;  // 3V
};

struct EvalLaunch {
    Geom g;
    const void* F;
    const void* M;
    int dtype;
    EvalIO io;
    LnccConsts c;
    Partials part;
    StagedScratch sc;
};

// Launch helpers return the number of kernels they enqueued.

// Pass 1 (steps (a)-(c)), staged form: one kernel per stage.
int eval_staged(const EvalLaunch& a, cudaStream_t s);
int eval_staged_partials(const Geom& g, int* n_loss, int* n_g2);

// Pass 2 (steps (c)-(d)): trial field from the current slot.
struct StepLaunch {
    Geom g;
    float* u0;
    float* u1;
    const float* g0;
    const float* g1;
    const DevState* st;
    float step;
    int attempt;
    // warp smoothing (sigma_warp > 0): composed field goes to tmp first
    Taps wtaps;
    float* tmpA;  // 3V
    float* tmpB;  // 3V
};
int step_compose(const StepLaunch& a, cudaStream_t s);

// Reduction of the partials and the state update.
enum FinMode { FIN_EXPLICIT = 0, FIN_RESET = 1, FIN_DECIDE = 2 };
struct FinLaunch {
    Partials part;
    DevState* st;
    EvalOut* out;       // FIN_EXPLICIT
    LogEntry* log;      // FIN_DECIDE
    DecideConsts d;
    double inv_V;       // 1 / V of the evaluated volume
    int mode;
    int attempt;
};
int finalize(const FinLaunch& a, cudaStream_t s);

// Replace the calling thread's lm_last_error() message.
void set_last_error(const char* msg);

// Copy the current field back into slot 0 when it sits in slot 1.
int sync_back(const Geom& g, float* u0, float* u1, DevState* st,
              cudaStream_t s);

}  // namespace lmk
