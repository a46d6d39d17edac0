// Pass 2 (the factored LM step and the compositive update, steps (c)-(d))
// and the device-side decision (step (e)).
//
//   ghat = g / gmax
//   du   = -r ghat / (|ghat|^2 + lambda)             Eq. tile1 (Appendix A)
//   v    = step * du
//   u*   = v + u o (Id + v)                           Eq. compositive
//   u*  <- G_sigma_warp * u*   (edge-extended, optional)
// then, after the trial is evaluated, the damping rule of Eq. lambda-update
// and the rejection rule of Eq. rejection decide on device.
#include <algorithm>

#include "lm_kernels.cuh"

namespace lmk {
namespace {

constexpr int TPB = 256;

__device__ __forceinline__ float safe_floor(float v) {
    return fminf(fmaxf(floorf(v), -1048576.f), 1048576.f);
}

__device__ __forceinline__ bool attempt_skip(const DevState* st, int attempt) {
    return attempt > 0 && st->done;
}

// One thread per voxel.  The trial goes to slot (1 - cu), or to dst when
// the warp is smoothed afterwards.
__global__ void k_step_compose(StepLaunch a, float* __restrict__ dst) {
    if (attempt_skip(a.st, a.attempt)) return;
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const Geom& g = a.g;
    if (i >= g.V) return;
    const int cu = a.st->cu, cg = a.st->cg;
    const float* __restrict__ u = cu ? a.u1 : a.u0;
    float* __restrict__ out = dst ? dst : (cu ? a.u0 : a.u1);
    const float* __restrict__ gg = cg ? a.g1 : a.g0;
    const float r = (float)a.st->L;
    const float lam = (float)a.st->lambda;
    const float gm = a.st->gmax;
    const float inv = gm > 0.f ? 1.f / gm : 0.f;

    float gh[3] = {gg[i] * inv, gg[g.V + i] * inv, gg[2 * g.V + i] * inv};
    float n2 = gh[0] * gh[0] + gh[1] * gh[1] + gh[2] * gh[2];
    float sc = -r / (n2 + lam) * a.step;
    float v[3] = {gh[0] * sc, gh[1] * sc, gh[2] * sc};

    int x = (int)(i % g.nx);
    long long rr = i / g.nx;
    int y = (int)(rr % g.ny), z = (int)(rr / g.ny);
    const int p[3] = {x, y, z};
    const int n[3] = {g.nx, g.ny, g.nz};
    int c0[3], c1[3];
    float f[3];
    for (int k = 0; k < 3; ++k) {
        float fl = safe_floor(v[k]);
        f[k] = v[k] - fl;
        int c = p[k] + (int)fl;
        c0[k] = min(max(c, 0), n[k] - 1);
        c1[k] = min(max(c + 1, 0), n[k] - 1);
    }
    long long sy = g.nx, sz = (long long)g.nx * g.ny;
    long long i000 = c0[2] * sz + c0[1] * sy + c0[0];
    long long dx = c1[0] - c0[0], dy = (c1[1] - c0[1]) * sy,
              dz = (c1[2] - c0[2]) * sz;
    float wx1 = f[0], wx0 = 1.f - f[0];
    float wy1 = f[1], wy0 = 1.f - f[1];
    float wz1 = f[2], wz0 = 1.f - f[2];
#pragma unroll
    for (int q = 0; q < 3; ++q) {
        const float* U = u + q * g.V;
        float m000 = U[i000], m100 = U[i000 + dx];
        float m010 = U[i000 + dy], m110 = U[i000 + dy + dx];
        float m001 = U[i000 + dz], m101 = U[i000 + dz + dx];
        float m011 = U[i000 + dz + dy], m111 = U[i000 + dz + dy + dx];
        float s = wz0 * (wy0 * (wx0 * m000 + wx1 * m100) +
                         wy1 * (wx0 * m010 + wx1 * m110)) +
                  wz1 * (wy0 * (wx0 * m001 + wx1 * m101) +
                         wy1 * (wx0 * m011 + wx1 * m111));
        out[q * g.V + i] = v[q] + s;
    }
}

// 1-D Gaussian along an axis of a 3-component field, edge-extended.  The z
// pass writes the trial slot (1 - cu).
__global__ void k_warp_gauss(const float* __restrict__ in, StepLaunch a,
                             int axis, float* __restrict__ out,
                             int final_pass) {
    if (attempt_skip(a.st, a.attempt)) return;
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const Geom& g = a.g;
    if (i >= g.V) return;
    float* dst = final_pass ? (a.st->cu ? a.u0 : a.u1) : out;
    int x = (int)(i % g.nx);
    long long rr = i / g.nx;
    int y = (int)(rr % g.ny), z = (int)(rr / g.ny);
    int pos = axis == 0 ? x : (axis == 1 ? y : z);
    int n = axis == 0 ? g.nx : (axis == 1 ? g.ny : g.nz);
    long long stride = axis == 0 ? 1 : (axis == 1 ? g.nx : (long long)g.nx * g.ny);
    const Taps& t = a.wtaps;
    float acc[3] = {0.f, 0.f, 0.f};
    for (int j = -t.R; j <= t.R; ++j) {
        int pp = min(max(pos + j, 0), n - 1);
        long long idx = i + (long long)(pp - pos) * stride;
        float w = t.t[j + t.R];
#pragma unroll
        for (int q = 0; q < 3; ++q) acc[q] += w * in[q * g.V + idx];
    }
#pragma unroll
    for (int q = 0; q < 3; ++q) dst[q * g.V + i] = acc[q];
}

__device__ __forceinline__ double block_sum1024(double v, double* sh) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) sh[wid] = v;
    __syncthreads();
    v = (threadIdx.x < (blockDim.x >> 5)) ? sh[threadIdx.x] : 0.0;
    if (wid == 0)
        for (int o = 16; o > 0; o >>= 1)
            v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ float block_max1024(float v, float* sh) {
    for (int o = 16; o > 0; o >>= 1)
        v = fmaxf(v, __shfl_down_sync(0xffffffffu, v, o));
    int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) sh[wid] = v;
    __syncthreads();
    v = (threadIdx.x < (blockDim.x >> 5)) ? sh[threadIdx.x] : 0.f;
    if (wid == 0)
        for (int o = 16; o > 0; o >>= 1)
            v = fmaxf(v, __shfl_down_sync(0xffffffffu, v, o));
    return v;
}

// Fixed-order FP64 reduction of the partials (deterministic), then the
// per-mode state update.  One CTA.
__global__ void k_finalize(FinLaunch a) {
    __shared__ double shd[32];
    __shared__ float shf[32];
    DevState* st = a.st;
    if (a.mode == FIN_DECIDE && attempt_skip(st, a.attempt)) return;
    double s = 0.0;
    for (int i = threadIdx.x; i < a.part.n_loss; i += blockDim.x)
        s += a.part.loss[i];
    s = block_sum1024(s, shd);
    float m = 0.f;
    int nf = 0;
    for (int i = threadIdx.x; i < a.part.n_g2; i += blockDim.x) {
        float v = a.part.g2max[i];
        if (!(v <= 3.0e38f)) nf = 1;   // NaN or overflow
        else m = fmaxf(m, v);
    }
    nf = __syncthreads_or(nf);
    m = block_max1024(m, shf);
    if (threadIdx.x != 0) return;
    double L = s * a.inv_V;
    float gmax = sqrtf(m);
    bool bad = nf || !isfinite(L) || !isfinite(gmax);
    if (a.mode == FIN_EXPLICIT) {
        a.out->L = L;
        a.out->gmax = gmax;
        a.out->status = bad ? STATUS_NONFINITE : 0;
        return;
    }
    if (a.mode == FIN_RESET) {
        st->L = L;
        st->L_prev = 0.0;
        st->L_trial = L;
        st->L_first = L;
        st->lambda = a.d.lambda0;
        st->gmax = gmax;
        st->gmax_trial = gmax;
        st->has_prev = 0;
        st->cu = 0;
        st->cg = 0;
        st->retries = 0;
        st->done = 0;
        st->accepted = 0;
        st->status = bad ? STATUS_NONFINITE : 0;
        st->iter = 0;
        st->evals = 1;
        st->log_pos = 0;
        return;
    }
    // FIN_DECIDE
    const int j = a.attempt;
    st->evals += 1;
    st->L_trial = L;
    st->gmax_trial = gmax;
    if (j == 0) {
        st->L_first = L;
        st->retries = 0;
    }
    const DecideConsts& d = a.d;
    double lam = st->lambda;
    int finished = 0, accepted = 0;
    if (bad) {
        st->status |= STATUS_NONFINITE;
        finished = 1;   // the trial is dropped, the state kept
    } else {
        bool rejected = false;
        if (d.reject) {
            double prev = st->has_prev ? fabs(st->L - st->L_prev) : 0.0;
            if (L - st->L > d.tau * prev) rejected = true;
        }
        if (rejected) {
            lam = fmin(d.mu_inc * lam, d.lambda_max);
            if (j < d.max_retries) {
                st->lambda = lam;
                st->retries = j + 1;
                st->done = 0;
                return;
            }
            finished = 1;   // discard after the last retry
        } else {
            lam = (L > st->L) ? fmin(d.mu_inc * lam, d.lambda_max)
                              : d.mu_dec * lam;
            finished = 1;
            accepted = 1;
        }
    }
    st->lambda = lam;
    st->retries = j;
    if (accepted) {
        st->cu ^= 1;
        st->cg ^= 1;
        st->L_prev = st->L;
        st->L = L;
        st->gmax = gmax;
        st->has_prev = 1;
    }
    st->accepted = accepted;
    st->done = finished;
    st->iter += 1;
    if (a.log) {
        int pos = st->log_pos;
        LogEntry e;
        e.loss = st->L;
        e.lambda = lam;
        e.gmax = st->gmax;
        e.accepted = accepted;
        e.retries = j;
        e.pad = 0;
        a.log[pos % LOG_CAP] = e;
        st->log_pos = pos + 1;
    }
}

__global__ void k_copy_back(const Geom g, float* __restrict__ u0,
                            const float* __restrict__ u1,
                            const DevState* st) {
    if (st->cu == 0) return;
    long long n = 3 * g.V;
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    long long stride = (long long)gridDim.x * blockDim.x;
    for (; i < n; i += stride) u0[i] = u1[i];
}

__global__ void k_flip_slot(DevState* st) { st->cu = 0; }

}  // namespace

int step_compose(const StepLaunch& a, cudaStream_t s) {
    unsigned nb = (unsigned)((a.g.V + TPB - 1) / TPB);
    if (a.wtaps.R > 0) {
        k_step_compose<<<nb, TPB, 0, s>>>(a, a.tmpA);
        k_warp_gauss<<<nb, TPB, 0, s>>>(a.tmpA, a, 0, a.tmpB, 0);
        k_warp_gauss<<<nb, TPB, 0, s>>>(a.tmpB, a, 1, a.tmpA, 0);
        k_warp_gauss<<<nb, TPB, 0, s>>>(a.tmpA, a, 2, nullptr, 1);
        return 4;
    }
    k_step_compose<<<nb, TPB, 0, s>>>(a, nullptr);
    return 1;
}

int finalize(const FinLaunch& a, cudaStream_t s) {
    k_finalize<<<1, 1024, 0, s>>>(a);
    return 1;
}

int sync_back(const Geom& g, float* u0, float* u1, DevState* st,
              cudaStream_t s) {
    long long n = 3 * g.V;
    unsigned nb = (unsigned)std::min<long long>((n + TPB - 1) / TPB, 4096);
    k_copy_back<<<nb, TPB, 0, s>>>(g, u0, u1, st);
    k_flip_slot<<<1, 1, 0, s>>>(st);
    return 2;
}

}  // namespace lmk
