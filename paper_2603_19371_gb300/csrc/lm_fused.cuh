// Fused z-streaming evaluation (pass 1) -- internal interface.
#pragma once

#include "lm_kernels.cuh"

namespace lmk {

// Work decomposition of the two evaluation kernels: the volume is cut into
// x-y columns; the (column, slice) units are split into equal contiguous
// shares, one per CTA (a CTA may finish one column and start the next).
struct FusedPlan {
    int e1_cx, e1_cy, e1_ctas;   // E1 columns in x and y, CTAs
    int e2_cx, e2_cy, e2_ctas;   // E2 columns in x and y, CTAs
    int minmax_ctas;             // CTAs of the image range reduction
};

// Fixed-point scale of the exact window moments: Xq = round((X - shift) Q),
// |Xq| <= qlim = 2^qb.
struct QScale {
    float shift;
    float Q;
    float invQ;
    int qlim;
};

struct FusedLaunch {
    Geom g;
    const void* F;
    const void* M;
    int dtype;
    EvalIO io;
    LnccConsts c;
    FusedPlan plan;
    const QScale* qs;     // device
    float* dldj;          // V, dL/dJ between the two kernels
    Partials part;        // n_loss = e1_ctas, n_g2 = e2_ctas
};

FusedPlan fused_plan(const Geom& g, int win, int num_sms);
int quant_bits(int win);
// Opt the kernels in to their dynamic shared memory (once per process).
cudaError_t fused_setup();
// Image range -> QScale (device-side, no host round trip).  part holds
// plan.minmax_ctas float2.  Returns kernels launched.
int fused_qscale(const void* F, const void* M, int dtype, const Geom& g,
                 const FusedPlan& pl, int win, float2* part, QScale* qs,
                 cudaStream_t s);
// Pass 1; returns kernels launched.
int eval_fused(const FusedLaunch& a, cudaStream_t s);

}  // namespace lmk
