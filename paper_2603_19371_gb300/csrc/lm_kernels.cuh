// Launch interfaces of the CUDA kernels (internal).
//
// Every kernel works on a batch of registration pairs described by a
// device-resident table of PairDesc entries (a single-pair context is a
// batch of one).  CTAs are assigned to pairs in contiguous ranges, so each
// CTA works on one pair and the per-CTA partial results reduce per pair in
// a fixed order (deterministic).
#pragma once

#include "lm_internal.cuh"

namespace lmk {

// Fixed-point scale of the exact window moments: Xq = round((X - shift) Q),
// |Xq| <= qlim = 2^qb.
struct QScale {
    float shift;
    float Q;
    float invQ;
    int qlim;
    float lo, hi;   // the range itself: min and max of F, M and 0
};

struct PairDesc {
    Geom g;
    const void* F;
    const void* M;
    float* u0;            // field slot 0 (the caller's field)
    float* u1;            // field slot 1 (library scratch)
    float* g0;            // gradient slots
    float* g1;
    const float* u_in;    // EVAL_EXPLICIT field
    float* g_out;         // EVAL_EXPLICIT gradient
    int* jq;              // J in the moments' fixed point (V), from the J pass
    int* fq;              // F in the moments' fixed point (V), per preparation
    int* fsum;            // exact k^3 window sum of fq (V), per preparation
    float* fvar;          // k^3-window variance B of F (V), per preparation
    float* dj;            // dJ/du (3 x V), from the J pass
    float* graw;          // g_raw [3][nz][ny][gp_w] between the evaluation
                          // kernels (rows padded to gp_w = nx rounded up
                          // to 4, so that TMA can tile it)
    const void* tm_graw;  // CUtensorMap (device memory) of graw for E2
    int gp_w;
    QScale* qs;
    DevState* st;
    LogEntry* log;        // may be NULL
    float* wtmpA;         // warp-smoothing temporaries (sigma_warp > 0)
    float* wtmpB;
    double target;        // stop once the loss is <= target (NaN: never)
    // evaluation kernel 1: columns and CTA range (loss partial slots)
    int e1_cx, e1_cy, e1_cta0, e1_ncta;
    // evaluation kernel 2: columns and CTA range (|g|^2 partial slots)
    int e2_cx, e2_cy, e2_cta0, e2_ncta;
    // step kernel: tiles, z chunks, first block
    int st_tx, st_ty, st_nzc, st_zc, st_blk0;
    // element-wise kernels (warp smoothing, copy-back): first block, count
    int ln_blk0, ln_nblk;
    // pooled curvature (tile side k > 1, Eq. tilen): per tile the mean of
    // g g^T of the current gradient, [th_nz][th_ny][th_nx][8] floats (xx,
    // xy, xz, yy, yz, zz, 2 unused), or NULL; tiles per axis and the first
    // block of the tile kernel (one block per tile row and slice)
    float* tileH;
    int th_nx, th_ny, th_nz, th_blk0;
    // injected fault (LM_FAULT_TIMEOUT, host-side): E2 first waits on a
    // barrier that no copy completes, so that its bounded wait runs out
    int fault_wait;
    // Layout of jq and fq.  qw = 0: plain [nz][ny][nx].  For the LNCC loss
    // a halo-padded volume [nz + 2 qz][qh][qw] whose halo holds the fixed
    // point of 0 (the zero padding of the window sums): voxel (x, y, z)
    // sits at ((z + qz) qh + y + qx) qw + x + qx, with qx = 2W, qz = 2W + 1,
    // qw = 32 ceil(nx / 32) + 4W and qh = 32 ceil(ny / 32) + 4W, so that the
    // moment kernel reads every gather row of every tile as aligned 16-byte
    // vectors without bounds tests.
    int qw, qh, qx, qz;
    // QFLAG_* bits of the pair: a non-finite J (set by the resampling
    // writers, cleared by the decision kernel that reads it) or F (set by
    // the preparation until the next one)
    unsigned* flags;
};
enum { QFLAG_JBAD = 1u, QFLAG_FBAD = 2u };

// Index of voxel (x, y, z) in the pair's jq / fq layout.
__host__ __device__ __forceinline__ long long qidx(const PairDesc& P, int x,
                                                  int y, int z) {
    return P.qw ? ((long long)(z + P.qz) * P.qh + y + P.qx) * P.qw + x + P.qx
                : ((long long)z * P.g.ny + y) * P.g.nx + x;
}
// Sets the jq / fq layout of a pair (halo-padded for the LNCC loss) and
// returns the number of elements each of the two buffers needs.
long long set_q_layout(PairDesc& d, int win, int loss);

// Pointers of an evaluation, routed by mode.
__device__ __forceinline__ const float* eval_u(const PairDesc& p, int mode) {
    if (mode == EVAL_EXPLICIT) return p.u_in;
    if (mode == EVAL_RESET) return p.u0;
    return p.st->cu ? p.u0 : p.u1;
}
__device__ __forceinline__ float* eval_g(const PairDesc& p, int mode) {
    if (mode == EVAL_EXPLICIT) return p.g_out;
    if (mode == EVAL_RESET) return p.g0;
    return p.st->cg ? p.g0 : p.g1;
}
// Later attempts of an iteration are no-ops once the pair's iteration is
// decided, and every attempt is once the pair has reached its target loss
// or the end of its replayed run (iter_end).  attempt < 0: the attempt
// index lives in the pair's device state (the decision sets it), so that
// one captured pass runs whichever attempt each pair is at.
__device__ __forceinline__ int attempt_of(const DevState* st, int attempt) {
    return attempt >= 0 ? attempt : st->att;
}
__device__ __forceinline__ bool attempt_skip(const DevState* st, int attempt) {
    return st->stopped || (st->iter_end > 0 && st->iter >= st->iter_end) ||
           (attempt_of(st, attempt) > 0 && st->done);
}
__device__ __forceinline__ bool trial_skip(const PairDesc& p, int mode,
                                           int attempt) {
    return mode == EVAL_TRIAL && attempt_skip(p.st, attempt);
}

// Pair whose block range starts at or below b (ranges ascend in pair
// order).  WHICH: 1 = E1 CTAs, 2 = E2 CTAs, 3 = step blocks, 4 = line
// blocks, 5 = tile-curvature blocks.
template <int WHICH>
__device__ __forceinline__ int pair_of_block(const PairDesc* pd, int npairs,
                                             int b) {
    int lo = 0, hi = npairs - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        int c0 = WHICH == 1   ? pd[mid].e1_cta0
                 : WHICH == 2 ? pd[mid].e2_cta0
                 : WHICH == 3 ? pd[mid].st_blk0
                 : WHICH == 4 ? pd[mid].ln_blk0
                              : pd[mid].th_blk0;
        if (c0 <= b)
            lo = mid;
        else
            hi = mid - 1;
    }
    return lo;
}

// Loss partials are exact: each voxel's term (1 - cc) is rounded to the
// fixed point 2^-30 and summed in int64, so the loss does not depend on how
// the voxels are split among CTAs (V < 2^31 keeps the sum below 2^63 for
// terms below 2^2 in magnitude, and any term that cc <= max(1, eps_nr /
// eps_dr) allows stays far below 2^32).
constexpr float LOSS_Q = 1073741824.f;            // 2^30
constexpr long long LOSS_BAD = (long long)(1ULL << 63);   // non-finite marker

// MSE partials: per voxel the exact square of the fixed-point difference
// dq = Fq - Jq (|dq| <= 2^(qb + 1)), shifted right by mse_shift(qlim) with
// rounding so that a term stays below 2^32 and a pair's sum (V < 2^30)
// below 2^62.  The loss is sum * 2^shift / (Q^2 V).
__host__ __device__ inline int mse_shift(int qlim) {
    int qb = 0;
    while ((1 << (qb + 1)) <= qlim) ++qb;
    const int sh = 2 * (qb + 1) - 32;
    return sh > 0 ? sh : 0;
}

// The 64-bit integer <-> FP32 conversions share the FP64 pipe, which is
// narrow on this part; the two helpers below use 32-bit conversions only.
//
// int64 -> FP32: v = hi 2^32 + lo with lo the signed low word, so that
// |v| < 2^31 converts exactly as one rounding of lo and larger values with
// at most ~1.3 ulp of error (one fused multiply-add of two converted words).
__device__ __forceinline__ float i64_to_f32(long long v) {
    const int lo = (int)(unsigned)(unsigned long long)v;
    const int hi = (int)((v - (long long)lo) >> 32);
    return fmaf((float)hi, 4294967296.f, (float)lo);
}

// A loss term scaled by LOSS_Q, rounded to the nearest integer (ties to
// even).  |v| < 2^31 takes one 32-bit conversion; a larger finite v is an
// integer already (its ulp is >= 256) and is split exactly at 2^31.  A
// non-finite or out-of-range v sets *bad.
__device__ __forceinline__ long long loss_fixed(float v, bool* bad) {
    if (fabsf(v) < 0x1p31f) return (long long)__float2int_rn(v);
    if (!(fabsf(v) < 0x1p61f)) {
        *bad = true;
        return 0;
    }
    const float h = truncf(v * 0x1p-31f);
    return ((long long)__float2int_rz(h) << 31) +
           (long long)__float2int_rn(fmaf(-h, 0x1p31f, v));
}

// Contiguous share of the (column, slice) work of CTA b out of n: the CTA
// walks segments [col, z0, z1) covering work units [lo, hi).
struct Share {
    long long lo, hi;
};
__device__ __forceinline__ Share share_of(int b, int n, long long total) {
    Share s;
    s.lo = total * b / n;
    s.hi = total * (b + 1) / n;
    return s;
}

// Sum of v[L .. L + N) as a balanced tree (depth ceil(log2 N) instead of
// N - 1 dependent adds); N and L are compile-time, so v stays in registers.
template <int L, int N, typename T>
__device__ __forceinline__ T tree_sum(const T* v) {
    if constexpr (N == 1)
        return v[L];
    else
        return tree_sum<L, N / 2, T>(v) + tree_sum<L + N / 2, N - N / 2, T>(v);
}

// Output tile variants of the LNCC moment kernel (a CTA marches along z
// over a column of such tiles; the autotuner picks one per batch):
//   E1_TILE_32X16: 32 x 16 outputs, 256 threads, two CTAs per SM (k <= 7),
//                  so one CTA's barriers overlap the other's work;
//   E1_TILE_32X32: 32 x 32 outputs, 512 threads, one CTA per SM, a smaller
//                  halo share per output (k <= 7 only).
enum { E1_TILE_32X16 = 0, E1_TILE_32X32 = 1, E1_NTILES = 2 };
constexpr int E1_OX = 32;
__host__ __device__ constexpr int e1_tile_oy(int t) { return t ? 32 : 16; }
__host__ __device__ constexpr int e1_tile_threads(int t) { return t ? 512 : 256; }
// the y granularity of the padded fixed-point layout: a multiple of every
// variant's tile height
constexpr int E1_QY = 32;

struct Partials {
    long long* loss;  // one per E1 CTA, fixed point LOSS_Q (or LOSS_BAD)
    float* g2max;     // one per E2 CTA
    // MI loss only, per pair: the B x B joint histogram (fixed point MI_HQ;
    // the CTAs add to it, the table kernel reads and clears it), the loss
    // r = log2 B - MI and the gradient table log2(p_ij / q_j) (B x B floats)
    unsigned long long* mi_hist;
    double* mi_loss;
    float* mi_table;
};

// Fixed point of one voxel's joint-histogram weight a_i b_j (<= 4/9).
constexpr float MI_HQ = 8388608.f;   // 2^23
constexpr int MI_MAX_BINS = 64;

// Totals of a batch plan.
struct BatchPlan {
    int e1_ctas, e2_ctas, st_blocks, ln_blocks, mm_ctas;
    int e1_tile;      // E1_TILE_* of the LNCC moment kernel
    int min_slices;   // z slices a z-streaming CTA gets at least (where the
                      // pair has that much work): long segments amortise the
                      // pipeline's warm-up, short ones add parallelism
    int st_target;    // step-kernel blocks per pair (z chunks of its tiles)
};

// Everything a launch needs besides the stream.
struct Batch {
    const PairDesc* pd;   // device table
    int npairs;
    int dtype;
    BatchPlan plan;
    LnccConsts c;
    DecideConsts d;
    Taps wtaps;
    float step;
    int tile;             // curvature tile side k (1 = Eq. tile1)
    int th_blocks;        // blocks of the tile-curvature kernel (tile > 1)
    int loss;             // LM_LOSS_LNCC / LM_LOSS_MSE / LM_LOSS_MI
    int method;           // LM_METHOD_LM / LM_METHOD_DEMONS
    float alpha;          // Demons damping weight
    int bins;             // MI histogram bins B
    Partials part;
    float2* mm_part;      // npairs * plan.mm_ctas image-range partials
};

// Fills the column / CTA / tile fields of each host PairDesc and returns the
// totals.  num_sms sizes the grids: E1 and E2 run e1_waves and e2_waves CTAs
// per SM in total, split among the pairs in proportion to their work (0: the
// defaults, 1 and 2 for a single pair, 4 and 8 for a batch).
BatchPlan plan_batch(PairDesc* host_pd, int npairs, int win, int num_sms,
                     int e1_waves = 0, int e2_waves = 0, int e1_tile = -1,
                     int min_slices = 8, int st_target = 2048);
// Whether the LNCC moment kernel has the tile variant t for window win.
bool e1_tile_ok(int t, int win);

// Opt the kernels in to their dynamic shared memory (once per process).
cudaError_t fused_setup();
// Row pitch of g_raw and its size in floats.
int graw_pitch(int nx);
long long graw_floats(const Geom& g);
// Encode the 4-D tensor map (x, y, z, component) E2 reads g_raw through,
// for Gaussian radius R, into the 128-byte host buffer map.
int encode_graw_map(void* map, const float* graw, const Geom& g, int R);
int quant_bits(int win);
// Tiles of side k per axis and the tile kernel's block range of each pair
// (a group of tile_group(k) of a block's TILE_WARPS warps per tile row and
// slice, so that each warp sums a few of the row's k^2 lines); returns the
// total block count.
constexpr int TILE_WARPS = 8;
__host__ __device__ inline int tile_group(int k) {
    return k * k < 8 ? 1 : k * k < 16 ? 2 : k * k < 32 ? 4 : 8;
}
int plan_tiles(PairDesc* host_pd, int npairs, int k);

// Launch helpers; each returns the number of kernels it enqueued.
// Preparation of the fixed image, once per reset or explicit evaluation:
// image range -> QScale per pair, then F in fixed point and its exact
// window sum and variance (device-side, no host round trip).  The J-pass
// scratch (graw, dj) serves as the separable passes' temporaries.
int batch_prepare(const Batch& b, cudaStream_t s);
// Pass 1: loss partials, dL/dJ, smoothed gradient, |g|^2 partials.  With
// jpass = false the J pass is left out (the step kernel already resampled
// the trial).  LNCC runs E1; MSE and Demons run one pointwise kernel in
// its place (MSE: g_raw = dL/dJ dJ/du; Demons: g_raw = the update of
// Eq. demons), both followed by E2.
int batch_eval(const Batch& b, int mode, int attempt, cudaStream_t s,
               bool jpass = true);
// The LNCC moment kernel (loss partials and g_raw) of pass 1 and its
// shared-memory opt-in.
int launch_lncc(const Batch& b, int mode, int attempt, cudaStream_t s);
cudaError_t lncc_setup();
// Pass 2: trial field (Eq. tile1, or Eq. tilen for tile > 1, + Eq.
// compositive, optional smoothing).
int batch_step(const Batch& b, int attempt, cudaStream_t s);
// Whether batch_step also resamples M at the trial (no warp smoothing).
bool step_resamples(const Batch& b);
// MI loss (pass 1's loss stage for LM_LOSS_MI): joint histogram partials,
// per-pair MI, loss and gradient table, then g_raw.  Returns the launches.
int launch_mi(const Batch& b, int mode, int attempt, cudaStream_t s);
// Opt the MI histogram kernel in to its dynamic shared memory.
cudaError_t mi_setup();
// Per-pair reduction and state update.
enum FinMode { FIN_EXPLICIT = 0, FIN_RESET = 1, FIN_DECIDE = 2 };
// attempt -1 with FIN_DECIDE: the state-driven pass (each pair's attempt
// read from and written back to its device state).
int batch_finalize(const Batch& b, int mode, int attempt, EvalOut* out,
                   cudaStream_t s);
// Sets each pair's iter_end to its iter + n (n > 0), or clears it (n = 0).
int batch_set_iter_end(const Batch& b, int n, cudaStream_t s);
// Copy each pair's current field back to slot 0 when it sits in slot 1.
int batch_sync_back(const Batch& b, cudaStream_t s);


// Replace the calling thread's lm_last_error() message.
void set_last_error(const char* msg);

// Host-side argument checks shared by every entry point (lm_api.cu).
// is_device_ptr: p is device or managed memory (no allocation, no sync).
bool is_device_ptr(const void* p);
// Gaussian taps exp(-j^2 / 2 sigma^2), |j| <= ceil(3 sigma), normalised to
// sum 1; sigma <= 0 gives the identity (R = 0).
Taps make_taps(double sigma);
// Every lm_params field in range; LM_EINVAL with lm_last_error() set.
int check_params(const lm_params* p);

}  // namespace lmk
