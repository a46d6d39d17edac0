// Pass 1 (loss and smoothed gradient, steps (a)-(c)) in staged form: one
// simple kernel per stage with full-volume intermediates.  This is the
// straightforward schedule of the evaluation; the fused z-streaming kernel
// computes the same quantities in one pass.
//
//  (a) trilinear resampling J = M(p + u), dJ/du        -- Section 2.1
//  (b) LNCC window statistics, per-voxel (1 - cc) and the backward
//      coefficients a = dcc/dS_FJ, b = dcc/dS_JJ, c = dcc/dS_J; box of
//      (a, b, c); dL/dJ and g_raw = dL/dJ * dJ/du   -- Section 2.2
//  (c) separable Gaussian of g_raw, max |g|           -- Section 2.1 / 3
//
// Box sums use a common shift s applied to F and J (padding value -s), so
// the window moments are formed from values near zero (shifted-mean FP32
// accumulation); the moments A, B, C and the gradient are shift-invariant.
#include "lm_kernels.cuh"

namespace lmk {
namespace {

constexpr int TPB = 256;

__device__ __forceinline__ void vox_xyz(long long i, const Geom& g, int& x,
                                        int& y, int& z) {
    x = (int)(i % g.nx);
    long long r = i / g.nx;
    y = (int)(r % g.ny);
    z = (int)(r / g.ny);
}

// Clamp of floor(u) keeps the integer cell arithmetic in range for any
// finite or infinite u; NaN propagates through the fractional weights.
__device__ __forceinline__ float safe_floor(float v) {
    return fminf(fmaxf(floorf(v), -1048576.f), 1048576.f);
}

template <typename T>
__global__ void k_sample(const T* __restrict__ M, EvalIO io, Geom g,
                         float* __restrict__ J, float* __restrict__ dJ) {
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= g.V || eval_skip(io)) return;
    int x, y, z;
    vox_xyz(i, g, x, y, z);
    const float* u = eval_u(io);
    float d[3] = {u[i], u[g.V + i], u[2 * g.V + i]};
    int c[3];
    float f[3];
    const int p[3] = {x, y, z};
    for (int k = 0; k < 3; ++k) {
        float fl = safe_floor(d[k]);
        c[k] = p[k] + (int)fl;
        f[k] = d[k] - fl;
    }
    float val = 0.f, gx = 0.f, gy = 0.f, gz = 0.f;
#pragma unroll
    for (int s = 0; s < 8; ++s) {
        int sx = s & 1, sy = (s >> 1) & 1, sz = s >> 2;
        int qx = c[0] + sx, qy = c[1] + sy, qz = c[2] + sz;
        float m = 0.f;
        if (qx >= 0 && qx < g.nx && qy >= 0 && qy < g.ny && qz >= 0 &&
            qz < g.nz)
            m = ld_img(M, ((long long)qz * g.ny + qy) * g.nx + qx);
        float wx = sx ? f[0] : 1.f - f[0];
        float wy = sy ? f[1] : 1.f - f[1];
        float wz = sz ? f[2] : 1.f - f[2];
        val += wx * wy * wz * m;
        gx += (sx ? 1.f : -1.f) * wy * wz * m;
        gy += (sy ? 1.f : -1.f) * wx * wz * m;
        gz += (sz ? 1.f : -1.f) * wx * wy * m;
    }
    J[i] = val;
    dJ[i] = gx;
    dJ[g.V + i] = gy;
    dJ[2 * g.V + i] = gz;
}

// x-pass of the first box filter: window sums of the five shifted products
// (F', J', F'F', J'J', F'J') with F' = F - s, J' = J - s, and -s outside.
template <typename T>
__global__ void k_box1_x(const T* __restrict__ F, const float* __restrict__ J,
                         EvalIO io, Geom g, int w, float s,
                         float* __restrict__ out) {
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= g.V || eval_skip(io)) return;
    int x, y, z;
    vox_xyz(i, g, x, y, z);
    float a0 = 0.f, a1 = 0.f, a2 = 0.f, a3 = 0.f, a4 = 0.f;
    for (int o = -w; o <= w; ++o) {
        int xx = x + o;
        float fp = -s, jp = -s;
        if (xx >= 0 && xx < g.nx) {
            fp = ld_img(F, i + o) - s;
            jp = J[i + o] - s;
        }
        a0 += fp;
        a1 += jp;
        a2 += fp * fp;
        a3 += jp * jp;
        a4 += fp * jp;
    }
    out[i] = a0;
    out[g.V + i] = a1;
    out[2 * g.V + i] = a2;
    out[3 * g.V + i] = a3;
    out[4 * g.V + i] = a4;
}

struct Pad5 {
    float v[5];
};

// Window sum along axis (1 = y, 2 = z) of NQ fields; out-of-volume entries
// contribute pad[q].
template <int NQ>
__global__ void k_box_line(const float* __restrict__ in, EvalIO io, Geom g,
                           int axis, int w, Pad5 pad, float* __restrict__ out) {
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= g.V || eval_skip(io)) return;
    int x, y, z;
    vox_xyz(i, g, x, y, z);
    int pos = axis == 0 ? x : (axis == 1 ? y : z);
    int n = axis == 0 ? g.nx : (axis == 1 ? g.ny : g.nz);
    long long stride = axis == 0 ? 1 : (axis == 1 ? g.nx : (long long)g.nx * g.ny);
    float acc[NQ];
#pragma unroll
    for (int q = 0; q < NQ; ++q) acc[q] = 0.f;
    for (int o = -w; o <= w; ++o) {
        int pp = pos + o;
        bool in_range = pp >= 0 && pp < n;
#pragma unroll
        for (int q = 0; q < NQ; ++q)
            acc[q] += in_range ? in[q * g.V + i + o * stride] : pad.v[q];
    }
#pragma unroll
    for (int q = 0; q < NQ; ++q) out[q * g.V + i] = acc[q];
}

__device__ __forceinline__ double block_sum(double v) {
    __shared__ double sh[32];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) sh[wid] = v;
    __syncthreads();
    int nw = blockDim.x >> 5;
    v = (threadIdx.x < nw) ? sh[threadIdx.x] : 0.0;
    if (wid == 0)
        for (int o = 16; o > 0; o >>= 1)
            v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ float block_max(float v) {
    __shared__ float sh[32];
    for (int o = 16; o > 0; o >>= 1)
        v = fmaxf(v, __shfl_down_sync(0xffffffffu, v, o));
    int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) sh[wid] = v;
    __syncthreads();
    int nw = blockDim.x >> 5;
    v = (threadIdx.x < nw) ? sh[threadIdx.x] : 0.f;
    if (wid == 0)
        for (int o = 16; o > 0; o >>= 1)
            v = fmaxf(v, __shfl_down_sync(0xffffffffu, v, o));
    return v;
}

// Window moments -> per-voxel (1 - cc) and backward coefficients.
//   A = S_FJ - mF mJ, B = max(S_FF - mF^2, 0), C = max(S_JJ - mJ^2, 0)
//   1 - cc = (B C - A^2 + eps_dr - eps_nr) / (B C + eps_dr)
//   a = 2A/D, b = -(A^2 + eps_nr) B / D^2 (the clamp on C only guards
//   against rounding; its slope is taken as 1),
//   c = -a mF - 2 b mJ  (in shifted coordinates)
// Products are formed with explicit round-to-nearest multiplies so that
// identical F and J windows give bitwise B == C == A and cc == 1.
__global__ void k_coef(const float* __restrict__ S, EvalIO io, Geom g,
                       LnccConsts c, float* __restrict__ abc,
                       double* __restrict__ loss_part) {
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (eval_skip(io)) return;
    float one_m_cc = 0.f;
    if (i < g.V) {
        float mF = S[i] * c.inv_k3;
        float mJ = S[g.V + i] * c.inv_k3;
        float sFF = S[2 * g.V + i] * c.inv_k3;
        float sJJ = S[3 * g.V + i] * c.inv_k3;
        float sFJ = S[4 * g.V + i] * c.inv_k3;
        float A = __fmaf_rn(-mF, mJ, sFJ);
        float Braw = __fmaf_rn(-mF, mF, sFF);
        float Craw = __fmaf_rn(-mJ, mJ, sJJ);
        float B = fmaxf(Braw, 0.f), C = fmaxf(Craw, 0.f);
        float BC = __fmul_rn(B, C), AA = __fmul_rn(A, A);
        float N = AA + c.eps_nr;
        float D = BC + c.eps_dr;
        float rD = 1.f / D;
        one_m_cc = ((BC - AA) + (c.eps_dr - c.eps_nr)) * rD;
        float a = 2.f * A * rD;
        float b = -N * B * rD * rD;
        float cc = -a * mF - 2.f * b * mJ;
        abc[i] = a;
        abc[g.V + i] = b;
        abc[2 * g.V + i] = cc;
    }
    double s = block_sum((double)one_m_cc);
    if (threadIdx.x == 0) loss_part[blockIdx.x] = s;
}

// dL/dJ(y) = -V^-1 [F'(y) Box(a) + 2 J'(y) Box(b) + Box(c)],
// g_raw = dL/dJ * dJ/du.  Box sums arrive unnormalised (x k^3).
template <typename T>
__global__ void k_graw(const T* __restrict__ F, const float* __restrict__ J,
                       const float* __restrict__ dJ,
                       const float* __restrict__ Babc, EvalIO io, Geom g,
                       LnccConsts c, float* __restrict__ graw) {
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= g.V || eval_skip(io)) return;
    float fp = ld_img(F, i) - c.shift;
    float jp = J[i] - c.shift;
    float ba = Babc[i] * c.inv_k3;
    float bb = Babc[g.V + i] * c.inv_k3;
    float bc = Babc[2 * g.V + i] * c.inv_k3;
    float dl = -c.inv_V * (fp * ba + 2.f * jp * bb + bc);
    graw[i] = dl * dJ[i];
    graw[g.V + i] = dl * dJ[g.V + i];
    graw[2 * g.V + i] = dl * dJ[2 * g.V + i];
}

// 1-D Gaussian along an axis of three fields, zero padding.  The z pass
// writes the routed gradient output and the per-CTA max |g|^2.
__global__ void k_gauss_line(const float* __restrict__ in, EvalIO io, Geom g,
                             int axis, Taps t, float* __restrict__ out,
                             int final_pass, float* __restrict__ g2_part) {
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (eval_skip(io)) return;
    float* dst = final_pass ? eval_g(io) : out;
    float n2 = 0.f;
    if (i < g.V) {
        int x, y, z;
        vox_xyz(i, g, x, y, z);
        int pos = axis == 0 ? x : (axis == 1 ? y : z);
        int n = axis == 0 ? g.nx : (axis == 1 ? g.ny : g.nz);
        long long stride =
            axis == 0 ? 1 : (axis == 1 ? g.nx : (long long)g.nx * g.ny);
        float acc[3] = {0.f, 0.f, 0.f};
        for (int j = -t.R; j <= t.R; ++j) {
            int pp = pos + j;
            if (pp < 0 || pp >= n) continue;
            float w = t.t[j + t.R];
#pragma unroll
            for (int q = 0; q < 3; ++q)
                acc[q] += w * in[q * g.V + i + j * stride];
        }
#pragma unroll
        for (int q = 0; q < 3; ++q) dst[q * g.V + i] = acc[q];
        n2 = acc[0] * acc[0] + acc[1] * acc[1] + acc[2] * acc[2];
    }
    if (final_pass) {
        float m = block_max(n2);
        if (threadIdx.x == 0) g2_part[blockIdx.x] = m;
    }
}

// sigma_grad = 0: g = g_raw, still producing the max |g|^2 partials.
__global__ void k_copy3_final(const float* __restrict__ in, EvalIO io,
                              Geom g, float* __restrict__ g2_part) {
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (eval_skip(io)) return;
    float* dst = eval_g(io);
    float n2 = 0.f;
    if (i < g.V) {
        float a = in[i], b = in[g.V + i], cz = in[2 * g.V + i];
        dst[i] = a;
        dst[g.V + i] = b;
        dst[2 * g.V + i] = cz;
        n2 = a * a + b * b + cz * cz;
    }
    float m = block_max(n2);
    if (threadIdx.x == 0) g2_part[blockIdx.x] = m;
}

}  // namespace

int eval_staged_partials(const Geom& g, int* n_loss, int* n_g2) {
    long long nb = (g.V + TPB - 1) / TPB;
    *n_loss = (int)nb;
    *n_g2 = (int)nb;
    return 0;
}

int eval_staged(const EvalLaunch& a, cudaStream_t s) {
    const Geom& g = a.g;
    unsigned nb = (unsigned)((g.V + TPB - 1) / TPB);
    int w = (a.c.win - 1) / 2;
    int k = a.c.win;
    float sh = a.c.shift;
    const StagedScratch& sc = a.sc;
    if (a.dtype == LM_BF16) {
        k_sample<<<nb, TPB, 0, s>>>((const __nv_bfloat16*)a.M, a.io, g, sc.J,
                                    sc.dJ);
        k_box1_x<<<nb, TPB, 0, s>>>((const __nv_bfloat16*)a.F, sc.J, a.io, g,
                                    w, sh, sc.T);
    } else {
        k_sample<<<nb, TPB, 0, s>>>((const float*)a.M, a.io, g, sc.J, sc.dJ);
        k_box1_x<<<nb, TPB, 0, s>>>((const float*)a.F, sc.J, a.io, g, w, sh,
                                    sc.T);
    }
    // padding products of (-s, -s): -s, -s, s^2, s^2, s^2 per cell
    float p1[5] = {-sh, -sh, sh * sh, sh * sh, sh * sh};
    Pad5 py, pz;
    for (int q = 0; q < 5; ++q) {
        py.v[q] = p1[q] * k;       // a row outside holds k padded cells
        pz.v[q] = p1[q] * k * k;   // a slice outside holds k^2
    }
    k_box_line<5><<<nb, TPB, 0, s>>>(sc.T, a.io, g, 1, w, py, sc.S);
    k_box_line<5><<<nb, TPB, 0, s>>>(sc.S, a.io, g, 2, w, pz, sc.T);
    k_coef<<<nb, TPB, 0, s>>>(sc.T, a.io, g, a.c, sc.abc, a.part.loss);
    Pad5 zero = {};
    k_box_line<3><<<nb, TPB, 0, s>>>(sc.abc, a.io, g, 0, w, zero, sc.S);
    k_box_line<3><<<nb, TPB, 0, s>>>(sc.S, a.io, g, 1, w, zero, sc.T);
    k_box_line<3><<<nb, TPB, 0, s>>>(sc.T, a.io, g, 2, w, zero, sc.S);
    if (a.dtype == LM_BF16)
        k_graw<<<nb, TPB, 0, s>>>((const __nv_bfloat16*)a.F, sc.J, sc.dJ,
                                  sc.S, a.io, g, a.c, sc.graw);
    else
        k_graw<<<nb, TPB, 0, s>>>((const float*)a.F, sc.J, sc.dJ, sc.S, a.io,
                                  g, a.c, sc.graw);
    if (a.c.gtaps.R > 0) {
        k_gauss_line<<<nb, TPB, 0, s>>>(sc.graw, a.io, g, 0, a.c.gtaps, sc.T,
                                        0, nullptr);
        k_gauss_line<<<nb, TPB, 0, s>>>(sc.T, a.io, g, 1, a.c.gtaps, sc.S, 0,
                                        nullptr);
        k_gauss_line<<<nb, TPB, 0, s>>>(sc.S, a.io, g, 2, a.c.gtaps, nullptr,
                                        1, a.part.g2max);
    } else {
        k_copy3_final<<<nb, TPB, 0, s>>>(sc.graw, a.io, g, a.part.g2max);
    }
    return a.c.gtaps.R > 0 ? 12 : 10;
}

}  // namespace lmk
