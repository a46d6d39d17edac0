// Fused z-streaming evaluation (pass 1) -- internal interface.
#pragma once

#include "lm_kernels.cuh"

namespace lmk {

// Work decomposition of the two evaluation kernels: x-y tiles times z
// chunks; one CTA per item.
struct FusedPlan {
    int e1_tx, e1_ty, e1_tz, e1_zc, e1_items;
    int e2_tx, e2_ty, e2_tz, e2_zc, e2_items;
};

struct FusedLaunch {
    Geom g;
    const void* F;
    const void* M;
    int dtype;
    EvalIO io;
    LnccConsts c;
    FusedPlan plan;
    const float* shift;   // e1_items per-item box-sum shifts
    float* dldj;          // V, dL/dJ between the two kernels
    Partials part;        // n_loss = e1_items, n_g2 = e2_items
};

FusedPlan fused_plan(const Geom& g, int num_sms);
// Opt the kernels in to their dynamic shared memory (once per process).
cudaError_t fused_setup();
// Per-item shifts (mean of F over each E1 tile); returns kernels launched.
int fused_tile_shift(const void* F, int dtype, const Geom& g,
                     const FusedPlan& pl, float* shift, cudaStream_t s);
// Pass 1; returns kernels launched.
int eval_fused(const FusedLaunch& a, cudaStream_t s);

}  // namespace lmk
