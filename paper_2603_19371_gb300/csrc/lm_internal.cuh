// Internal definitions shared by the CUDA translation units of liblmreg.
// Not part of the public ABI (include/lmreg.h is).
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include "lmreg.h"

namespace lmk {

// Volume geometry: x fastest, V = nx * ny * nz.
struct Geom {
    int nx, ny, nz;
    long long V;
};

// Optimiser state kept on the device so that an LM iteration (and its
// rejected retries) runs without a host round trip.  u and g live in two
// ping-pong slots each; cu / cg name the slot holding the current field and
// its gradient, the trial goes to the other slot.
struct DevState {
    double L;          // L_t, loss of the current field
    double L_prev;     // L_{t-1}
    double L_trial;    // loss of the last evaluated trial
    double L_first;    // loss of the first trial of the last iteration
    double lambda;     // damping
    float gmax;        // max |g| of the current gradient
    float gmax_trial;  // max |g| of the last trial gradient
    int has_prev;      // L_prev defined
    int cu, cg;        // current slots
    int retries;       // rejections in the current iteration
    int done;          // current iteration finished (attempts > 0 skip)
    int accepted;      // outcome of the last finished iteration
    int status;        // sticky error bits (STATUS_*)
    int iter;          // finished iterations since reset
    int evals;         // loss evaluations since reset
    int log_pos;       // next log slot
    int stopped;       // reached the pair's target loss: iterations are no-ops
    int att;           // the attempt the next state-driven pass runs (kernels
                       // given -1): 0 starts an iteration, j > 0 retries it
                       // after j rejected trials
    int iter_end;      // > 0: passes are no-ops once iter reaches it (the
                       // end of a replayed run of iterations); 0: no limit
};

// STATUS_TIMEOUT: a bounded device wait ran out (the evaluation's result is
// void); the host reports it as LM_ETIMEOUT ahead of STATUS_NONFINITE.
enum { STATUS_NONFINITE = 1, STATUS_TIMEOUT = 2 };

// One record per finished iteration, written by the decision kernel.
struct LogEntry {
    double loss;
    double lambda;
    float gmax;
    int accepted;
    int retries;
    int pad;
};
constexpr int LOG_CAP = 8192;

// Result of an explicit (stateless) evaluation of one pair.
struct EvalOut {
    double L;
    float gmax;
    int status;
};

// Gaussian taps t_{-R..R}, R <= MAX_R.
constexpr int MAX_R = 6;
struct Taps {
    int R;
    float t[2 * MAX_R + 1];
};

// Where an evaluation reads its field and writes its gradient.
enum EvalMode {
    EVAL_EXPLICIT = 0,  // u = u_in, g -> g_out; result to EvalOut
    EVAL_RESET = 1,     // u = slot 0, g -> slot 0; result initialises state
    EVAL_TRIAL = 2,     // u = trial slot (1 - cu), g -> trial slot (1 - cg)
};

// Scalar LNCC / smoothing constants of one evaluation (shared by all pairs
// of a batch; 1/V is per pair).
struct LnccConsts {
    int win;        // k
    float eps_nr, eps_dr;
    float inv_k3;   // 1 / k^3
    Taps gtaps;     // gradient smoothing taps
};

// Decision parameters (Eq. lambda-update, Eq. rejection), device copy.
struct DecideConsts {
    double lambda0, mu_inc, mu_dec, lambda_max, tau;
    int reject, max_retries;
    int mse;      // loss partials are MSE sums (unit from the pair's QScale)
    int mi;       // the loss is r = log2 B - MI, from the MI table kernel
    int demons;   // every trial is kept (Section 2.3), lambda unused
};

// Image element load as float.
__device__ __forceinline__ float ld_img(const float* p, long long i) {
    return __ldg(p + i);
}
__device__ __forceinline__ float ld_img(const __nv_bfloat16* p, long long i) {
    return __bfloat162float(p[i]);
}

}  // namespace lmk
