// Pass 1 (loss and smoothed gradient, steps (a)-(c)) as two z-streaming
// kernels.  Each CTA owns an x-y tile and a z-range and marches along z,
// keeping the planes of every stage in shared memory; the separable box and
// Gaussian filters run in x and y on those planes and in z on ring buffers
// of the last k planes.
//
//  E1 (lncc): J = M(p + u) (trilinear, Section 2.1); window moments of the
//     shifted F' = F - s, J' = J - s (box k^3, zero padding); per voxel
//     (1 - cc) and the backward coefficients (a, b, c) of Section 2.2's
//     squared-loss form; their box sums; and
//        dL/dJ(y) = -V^-1 [F'(y) Box(a) + 2 J'(y) Box(b) + Box(c)]
//     written to HBM (4 bytes / voxel), plus the CTA's loss partial.
//     Halo: 2w voxels of J around the tile (w around the moments).
//  E2 (grad): dJ/du at the tile and an R-voxel halo, g_raw = dL/dJ * dJ/du,
//     separable Gaussian (R = ceil(3 sigma)), g to HBM, CTA max |g|^2.
//
// HBM traffic per voxel: E1 reads F, M, u (20 B) and writes dL/dJ (4 B);
// E2 reads dL/dJ, M, u (20 B) and writes g (12 B).  Halo re-reads hit L2.
//
// The shift s is one value per E1 work item (the mean of F over the item's
// tile), so the window moments are formed from values near zero; moments,
// cc and the gradient are exactly shift-invariant in exact arithmetic
// because out-of-volume cells carry -s as well.
#include <algorithm>

#include "lm_fused.cuh"

namespace lmk {
namespace {

constexpr int E1_TX = 32, E1_TY = 8, E1_NT = 256;
constexpr int E2_TX = 32, E2_TY = 16, E2_NT = 256;

__device__ __forceinline__ float safe_floor(float v) {
    return fminf(fmaxf(floorf(v), -1048576.f), 1048576.f);
}

// Trilinear corners of M around p + u(p), zero outside the volume.
template <typename T>
__device__ __forceinline__ void corners(const T* __restrict__ M,
                                        const float* __restrict__ u,
                                        const Geom& g, int x, int y, int z,
                                        long long i, float m[8], float f[3]) {
    float d0 = u[i], d1 = u[g.V + i], d2 = u[2 * g.V + i];
    float l0 = safe_floor(d0), l1 = safe_floor(d1), l2 = safe_floor(d2);
    f[0] = d0 - l0;
    f[1] = d1 - l1;
    f[2] = d2 - l2;
    int cx = x + (int)l0, cy = y + (int)l1, cz = z + (int)l2;
    const long long sxy = (long long)g.nx * g.ny;
    if (cx >= 0 && cx + 1 < g.nx && cy >= 0 && cy + 1 < g.ny && cz >= 0 &&
        cz + 1 < g.nz) {
        long long b = (long long)cz * sxy + (long long)cy * g.nx + cx;
        m[0] = ld_img(M, b);
        m[1] = ld_img(M, b + 1);
        m[2] = ld_img(M, b + g.nx);
        m[3] = ld_img(M, b + g.nx + 1);
        m[4] = ld_img(M, b + sxy);
        m[5] = ld_img(M, b + sxy + 1);
        m[6] = ld_img(M, b + sxy + g.nx);
        m[7] = ld_img(M, b + sxy + g.nx + 1);
    } else {
#pragma unroll
        for (int s = 0; s < 8; ++s) {
            int qx = cx + (s & 1), qy = cy + ((s >> 1) & 1), qz = cz + (s >> 2);
            bool in = qx >= 0 && qx < g.nx && qy >= 0 && qy < g.ny && qz >= 0 &&
                      qz < g.nz;
            m[s] = in ? ld_img(M, (long long)qz * sxy + (long long)qy * g.nx + qx)
                      : 0.f;
        }
    }
}

// J from the corners (m index = x + 2y + 4z).
__device__ __forceinline__ float interp(const float m[8], const float f[3]) {
    float a0 = m[0] + f[0] * (m[1] - m[0]);
    float a1 = m[2] + f[0] * (m[3] - m[2]);
    float a2 = m[4] + f[0] * (m[5] - m[4]);
    float a3 = m[6] + f[0] * (m[7] - m[6]);
    float b0 = a0 + f[1] * (a1 - a0);
    float b1 = a2 + f[1] * (a3 - a2);
    return b0 + f[2] * (b1 - b0);
}

// dJ/du from the corners.
__device__ __forceinline__ void interp_grad(const float m[8], const float f[3],
                                            float d[3]) {
    float ex0 = m[1] - m[0], ex1 = m[3] - m[2], ex2 = m[5] - m[4],
          ex3 = m[7] - m[6];
    float gx0 = ex0 + f[1] * (ex1 - ex0);
    float gx1 = ex2 + f[1] * (ex3 - ex2);
    d[0] = gx0 + f[2] * (gx1 - gx0);
    float a0 = m[0] + f[0] * ex0, a1 = m[2] + f[0] * ex1;
    float a2 = m[4] + f[0] * ex2, a3 = m[6] + f[0] * ex3;
    float ey0 = a1 - a0, ey1 = a3 - a2;
    d[1] = ey0 + f[2] * (ey1 - ey0);
    float b0 = a0 + f[1] * ey0, b1 = a2 + f[1] * ey1;
    d[2] = b1 - b0;
}

template <int W>
struct E1Smem {
    static constexpr int K = 2 * W + 1;
    static constexpr int GX = E1_TX + 4 * W, GY = E1_TY + 4 * W;
    static constexpr int SX = E1_TX + 2 * W, SY = E1_TY + 2 * W;
    static constexpr int P = 5 * GY * GX;            // products, gather plane
    static constexpr int X = 5 * GY * SX;            // x-boxed
    static constexpr int SR = K * 5 * SY * SX;       // xy-boxed ring
    static constexpr int AB = 3 * SY * SX;           // a, b, c
    static constexpr int AX = 3 * SY * E1_TX;        // x-boxed a, b, c
    static constexpr int BR = K * 3 * E1_TY * E1_TX; // xy-boxed ring
    static constexpr int JR = K * E1_TY * E1_TX;     // J' delay line
    static constexpr int floats = P + X + SR + AB + AX + BR + JR;
};

template <int W, typename T>
__global__ void __launch_bounds__(E1_NT)
    k_e1(const T* __restrict__ F, const T* __restrict__ M, EvalIO io, Geom g,
         LnccConsts c, FusedPlan pl, const float* __restrict__ shift,
         float* __restrict__ dldj, double* __restrict__ loss_part) {
    using S = E1Smem<W>;
    constexpr int K = S::K, GX = S::GX, GY = S::GY, SX = S::SX, SY = S::SY;
    constexpr int TX = E1_TX, TY = E1_TY;
    extern __shared__ float sm[];
    float* Pg = sm;
    float* Sx = Pg + S::P;
    float* Sr = Sx + S::X;
    float* Ab = Sr + S::SR;
    float* Ax = Ab + S::AB;
    float* Br = Ax + S::AX;
    float* Jr = Br + S::BR;
    __shared__ double red[E1_NT / 32];

    if (eval_skip(io)) return;
    const int item = blockIdx.x;
    const int tx_ = item % pl.e1_tx;
    const int rest = item / pl.e1_tx;
    const int ty_ = rest % pl.e1_ty;
    const int zi = rest / pl.e1_ty;
    const int x0 = tx_ * TX, y0 = ty_ * TY;
    const int z0 = zi * pl.e1_zc;
    const int z1 = min(z0 + pl.e1_zc, g.nz);
    const float sh = shift[item];
    const float* __restrict__ u = eval_u(io);
    const long long sxy = (long long)g.nx * g.ny;
    const int tid = threadIdx.x;
    double lacc = 0.0;

    const int s_begin = z0 - 2 * W, s_end = z1 + 2 * W;
    for (int s = s_begin, t = 0; s < s_end; ++s, ++t) {
        // (1) gather plane: F', J' and the five products
        const bool zin = s >= 0 && s < g.nz;
        for (int idx = tid; idx < GX * GY; idx += E1_NT) {
            int gy = idx / GX, gx = idx - gy * GX;
            int x = x0 - 2 * W + gx, y = y0 - 2 * W + gy;
            float fp = -sh, jp = -sh;
            if (zin && x >= 0 && x < g.nx && y >= 0 && y < g.ny) {
                long long i = (long long)s * sxy + (long long)y * g.nx + x;
                float m[8], f[3];
                corners(M, u, g, x, y, s, i, m, f);
                fp = ld_img(F, i) - sh;
                jp = interp(m, f) - sh;
            }
            Pg[idx] = fp;
            Pg[GY * GX + idx] = jp;
            Pg[2 * GY * GX + idx] = fp * fp;
            Pg[3 * GY * GX + idx] = jp * jp;
            Pg[4 * GY * GX + idx] = fp * jp;
            int ox = gx - 2 * W, oy = gy - 2 * W;
            if (ox >= 0 && ox < TX && oy >= 0 && oy < TY)
                Jr[(t % K) * TY * TX + oy * TX + ox] = jp;
        }
        __syncthreads();
        // (2) box along x
        for (int idx = tid; idx < 5 * GY * SX; idx += E1_NT) {
            int q = idx / (GY * SX);
            int r2 = idx - q * (GY * SX);
            int gy = r2 / SX, sx = r2 - gy * SX;
            const float* row = Pg + q * GY * GX + gy * GX + sx;
            float v = 0.f;
#pragma unroll
            for (int o = 0; o < K; ++o) v += row[o];
            Sx[idx] = v;
        }
        __syncthreads();
        // (3) box along y into the ring; along z once the ring is full; the
        //     moments give (1 - cc) and (a, b, c) at slice cz = s - W
        const int cz = s - W;
        const bool coef_valid = t >= 2 * W;
        for (int idx = tid; idx < SY * SX; idx += E1_NT) {
            int sy = idx / SX, sx = idx - sy * SX;
#pragma unroll
            for (int q = 0; q < 5; ++q) {
                const float* col = Sx + q * GY * SX + sy * SX + sx;
                float v = 0.f;
#pragma unroll
                for (int o = 0; o < K; ++o) v += col[o * SX];
                Sr[((t % K) * 5 + q) * SY * SX + idx] = v;
            }
            if (!coef_valid) continue;
            float m5[5];
#pragma unroll
            for (int q = 0; q < 5; ++q) {
                float v = 0.f;
#pragma unroll
                for (int j = 0; j < K; ++j)
                    v += Sr[(((t - 2 * W + j) % K) * 5 + q) * SY * SX + idx];
                m5[q] = v * c.inv_k3;
            }
            int x = x0 - W + sx, y = y0 - W + sy;
            float av = 0.f, bv = 0.f, cv = 0.f;
            if (x >= 0 && x < g.nx && y >= 0 && y < g.ny && cz >= 0 &&
                cz < g.nz) {
                float mF = m5[0], mJ = m5[1];
                float A = __fmaf_rn(-mF, mJ, m5[4]);
                float B = fmaxf(__fmaf_rn(-mF, mF, m5[2]), 0.f);
                float C = fmaxf(__fmaf_rn(-mJ, mJ, m5[3]), 0.f);
                float BC = __fmul_rn(B, C), AA = __fmul_rn(A, A);
                float N = AA + c.eps_nr;
                float D = BC + c.eps_dr;
                float rD = 1.f / D;
                av = 2.f * A * rD;
                bv = -N * B * rD * rD;
                cv = -av * mF - 2.f * bv * mJ;
                if (sx >= W && sx < W + TX && sy >= W && sy < W + TY &&
                    cz >= z0 && cz < z1)
                    lacc += (double)(((BC - AA) + (c.eps_dr - c.eps_nr)) * rD);
            }
            Ab[idx] = av;
            Ab[SY * SX + idx] = bv;
            Ab[2 * SY * SX + idx] = cv;
        }
        __syncthreads();
        if (coef_valid) {
            // (4) box of (a, b, c) along x
            for (int idx = tid; idx < 3 * SY * TX; idx += E1_NT) {
                int q = idx / (SY * TX);
                int r2 = idx - q * (SY * TX);
                int sy = r2 / TX, tx = r2 - sy * TX;
                const float* row = Ab + q * SY * SX + sy * SX + tx;
                float v = 0.f;
#pragma unroll
                for (int o = 0; o < K; ++o) v += row[o];
                Ax[idx] = v;
            }
            __syncthreads();
            // (5) along y into the second ring, along z, then dL/dJ at
            //     slice r = s - 2W
            const int tc = t - 2 * W;
            const bool out_valid = tc >= 2 * W;
            const int r = cz - W;
            for (int idx = tid; idx < TY * TX; idx += E1_NT) {
                int ty = idx / TX, tx = idx - ty * TX;
#pragma unroll
                for (int q = 0; q < 3; ++q) {
                    const float* col = Ax + q * SY * TX + ty * TX + tx;
                    float v = 0.f;
#pragma unroll
                    for (int o = 0; o < K; ++o) v += col[o * TX];
                    Br[((tc % K) * 3 + q) * TY * TX + idx] = v;
                }
                if (!out_valid) continue;
                float b3[3];
#pragma unroll
                for (int q = 0; q < 3; ++q) {
                    float v = 0.f;
#pragma unroll
                    for (int j = 0; j < K; ++j)
                        v += Br[(((tc - 2 * W + j) % K) * 3 + q) * TY * TX + idx];
                    b3[q] = v;
                }
                int x = x0 + tx, y = y0 + ty;
                if (x < g.nx && y < g.ny) {
                    long long i = (long long)r * sxy + (long long)y * g.nx + x;
                    float fp = ld_img(F, i) - sh;
                    float jp = Jr[((t - 2 * W) % K) * TY * TX + idx];
                    dldj[i] = -c.inv_V *
                              ((fp * b3[0] + 2.f * jp * b3[1] + b3[2]) * c.inv_k3);
                }
            }
        }
        __syncthreads();
    }
    // CTA loss partial, fixed-order FP64 reduction
    for (int o = 16; o > 0; o >>= 1) lacc += __shfl_down_sync(0xffffffffu, lacc, o);
    if ((tid & 31) == 0) red[tid >> 5] = lacc;
    __syncthreads();
    if (tid == 0) {
        double v = 0.0;
        for (int w = 0; w < E1_NT / 32; ++w) v += red[w];
        loss_part[item] = v;
    }
}

template <int R>
struct E2Smem {
    static constexpr int KG = 2 * R + 1;
    static constexpr int RX = E2_TX + 2 * R, RY = E2_TY + 2 * R;
    static constexpr int GR = 3 * RY * RX;
    static constexpr int GXs = 3 * RY * E2_TX;
    static constexpr int GQ = KG * 3 * E2_TY * E2_TX;
    static constexpr int floats = GR + GXs + GQ;
};

template <int R, typename T>
__global__ void __launch_bounds__(E2_NT)
    k_e2(const T* __restrict__ M, EvalIO io, Geom g, Taps tp, FusedPlan pl,
         const float* __restrict__ dldj, float* __restrict__ g2_part) {
    using S = E2Smem<R>;
    constexpr int KG = S::KG, RX = S::RX, RY = S::RY;
    constexpr int TX = E2_TX, TY = E2_TY;
    extern __shared__ float sm[];
    float* Gr = sm;
    float* Gx = Gr + S::GR;
    float* Gq = Gx + S::GXs;
    __shared__ float red[E2_NT / 32];

    if (eval_skip(io)) return;
    const int item = blockIdx.x;
    const int tx_ = item % pl.e2_tx;
    const int rest = item / pl.e2_tx;
    const int ty_ = rest % pl.e2_ty;
    const int zi = rest / pl.e2_ty;
    const int x0 = tx_ * TX, y0 = ty_ * TY;
    const int z0 = zi * pl.e2_zc;
    const int z1 = min(z0 + pl.e2_zc, g.nz);
    const float* __restrict__ u = eval_u(io);
    float* __restrict__ gout = eval_g(io);
    const long long sxy = (long long)g.nx * g.ny;
    const int tid = threadIdx.x;
    float m2 = 0.f;

    for (int s = z0 - R, t = 0; s < z1 + R; ++s, ++t) {
        const bool zin = s >= 0 && s < g.nz;
        // (1) g_raw = dL/dJ * dJ/du on the tile and its R halo
        for (int idx = tid; idx < RX * RY; idx += E2_NT) {
            int ry = idx / RX, rx = idx - ry * RX;
            int x = x0 - R + rx, y = y0 - R + ry;
            float g0 = 0.f, g1 = 0.f, g2 = 0.f;
            if (zin && x >= 0 && x < g.nx && y >= 0 && y < g.ny) {
                long long i = (long long)s * sxy + (long long)y * g.nx + x;
                float m[8], f[3], d[3];
                corners(M, u, g, x, y, s, i, m, f);
                interp_grad(m, f, d);
                float dl = dldj[i];
                g0 = dl * d[0];
                g1 = dl * d[1];
                g2 = dl * d[2];
            }
            Gr[idx] = g0;
            Gr[RY * RX + idx] = g1;
            Gr[2 * RY * RX + idx] = g2;
        }
        __syncthreads();
        // (2) Gaussian along x
        for (int idx = tid; idx < 3 * RY * TX; idx += E2_NT) {
            int q = idx / (RY * TX);
            int r2 = idx - q * (RY * TX);
            int ry = r2 / TX, tx = r2 - ry * TX;
            const float* row = Gr + q * RY * RX + ry * RX + tx;
            float v = 0.f;
#pragma unroll
            for (int j = 0; j < KG; ++j) v += tp.t[j] * row[j];
            Gx[idx] = v;
        }
        __syncthreads();
        // (3) along y into the ring, along z at slice o = s - R
        const int o = s - R;
        const bool valid = t >= 2 * R;
        for (int idx = tid; idx < TY * TX; idx += E2_NT) {
            int ty = idx / TX, tx = idx - ty * TX;
#pragma unroll
            for (int q = 0; q < 3; ++q) {
                const float* col = Gx + q * RY * TX + ty * TX + tx;
                float v = 0.f;
#pragma unroll
                for (int j = 0; j < KG; ++j) v += tp.t[j] * col[j * TX];
                Gq[((t % KG) * 3 + q) * TY * TX + idx] = v;
            }
            if (!valid) continue;
            int x = x0 + tx, y = y0 + ty;
            if (x >= g.nx || y >= g.ny) continue;
            long long i = (long long)o * sxy + (long long)y * g.nx + x;
            float n2 = 0.f;
#pragma unroll
            for (int q = 0; q < 3; ++q) {
                float v = 0.f;
#pragma unroll
                for (int j = 0; j < KG; ++j)
                    v += tp.t[j] * Gq[(((t - 2 * R + j) % KG) * 3 + q) * TY * TX + idx];
                gout[q * g.V + i] = v;
                n2 += v * v;
            }
            m2 = (n2 != n2) ? INFINITY : fmaxf(m2, n2);
        }
        __syncthreads();
    }
    for (int k = 16; k > 0; k >>= 1)
        m2 = fmaxf(m2, __shfl_down_sync(0xffffffffu, m2, k));
    if ((tid & 31) == 0) red[tid >> 5] = m2;
    __syncthreads();
    if (tid == 0) {
        float v = 0.f;
        for (int w = 0; w < E2_NT / 32; ++w) v = fmaxf(v, red[w]);
        g2_part[item] = v;
    }
}

// Per-item mean of F over the item's E1 tile (the box-sum shift).
template <typename T>
__global__ void k_tile_shift(const T* __restrict__ F, Geom g, FusedPlan pl,
                             float* __restrict__ shift) {
    __shared__ double red[256 / 32];
    const int item = blockIdx.x;
    const int tx_ = item % pl.e1_tx;
    const int rest = item / pl.e1_tx;
    const int ty_ = rest % pl.e1_ty;
    const int zi = rest / pl.e1_ty;
    const int x0 = tx_ * E1_TX, y0 = ty_ * E1_TY;
    const int z0 = zi * pl.e1_zc, z1 = min(z0 + pl.e1_zc, g.nz);
    const int nxl = min(E1_TX, g.nx - x0), nyl = min(E1_TY, g.ny - y0);
    const long long n = (long long)nxl * nyl * (z1 - z0);
    double s = 0.0;
    for (long long k = threadIdx.x; k < n; k += blockDim.x) {
        int x = (int)(k % nxl);
        long long r = k / nxl;
        int y = (int)(r % nyl);
        int z = (int)(r / nyl);
        s += (double)ld_img(F, ((long long)(z0 + z) * g.ny + (y0 + y)) * g.nx +
                                   (x0 + x));
    }
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double v = 0.0;
        for (int w = 0; w < 256 / 32; ++w) v += red[w];
        shift[item] = n > 0 ? (float)(v / (double)n) : 0.f;
    }
}

template <int W, typename T>
int launch_e1(const FusedLaunch& a, cudaStream_t s) {
    size_t bytes = (size_t)E1Smem<W>::floats * sizeof(float);
    k_e1<W, T><<<a.plan.e1_items, E1_NT, bytes, s>>>(
        (const T*)a.F, (const T*)a.M, a.io, a.g, a.c, a.plan, a.shift, a.dldj,
        a.part.loss);
    return 1;
}

template <int R, typename T>
int launch_e2(const FusedLaunch& a, cudaStream_t s) {
    size_t bytes = (size_t)E2Smem<R>::floats * sizeof(float);
    k_e2<R, T><<<a.plan.e2_items, E2_NT, bytes, s>>>(
        (const T*)a.M, a.io, a.g, a.c.gtaps, a.plan, a.dldj, a.part.g2max);
    return 1;
}

template <typename T>
int launch_e1_w(const FusedLaunch& a, cudaStream_t s) {
    switch ((a.c.win - 1) / 2) {
        case 1: return launch_e1<1, T>(a, s);
        case 2: return launch_e1<2, T>(a, s);
        case 3: return launch_e1<3, T>(a, s);
        default: return launch_e1<4, T>(a, s);
    }
}

template <typename T>
int launch_e2_r(const FusedLaunch& a, cudaStream_t s) {
    switch (a.c.gtaps.R) {
        case 0: return launch_e2<0, T>(a, s);
        case 1: return launch_e2<1, T>(a, s);
        case 2: return launch_e2<2, T>(a, s);
        case 3: return launch_e2<3, T>(a, s);
        case 4: return launch_e2<4, T>(a, s);
        case 5: return launch_e2<5, T>(a, s);
        default: return launch_e2<6, T>(a, s);
    }
}

template <int W, typename T>
cudaError_t attr_e1() {
    return cudaFuncSetAttribute(k_e1<W, T>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)(E1Smem<W>::floats * sizeof(float)));
}
template <int R, typename T>
cudaError_t attr_e2() {
    return cudaFuncSetAttribute(k_e2<R, T>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)(E2Smem<R>::floats * sizeof(float)));
}

template <typename T>
cudaError_t attrs_all() {
    cudaError_t e = cudaSuccess;
    cudaError_t r;
    if ((r = attr_e1<1, T>()) != cudaSuccess) e = r;
    if ((r = attr_e1<2, T>()) != cudaSuccess) e = r;
    if ((r = attr_e1<3, T>()) != cudaSuccess) e = r;
    if ((r = attr_e1<4, T>()) != cudaSuccess) e = r;
    if ((r = attr_e2<0, T>()) != cudaSuccess) e = r;
    if ((r = attr_e2<1, T>()) != cudaSuccess) e = r;
    if ((r = attr_e2<2, T>()) != cudaSuccess) e = r;
    if ((r = attr_e2<3, T>()) != cudaSuccess) e = r;
    if ((r = attr_e2<4, T>()) != cudaSuccess) e = r;
    if ((r = attr_e2<5, T>()) != cudaSuccess) e = r;
    if ((r = attr_e2<6, T>()) != cudaSuccess) e = r;
    return e;
}

int ceil_div(long long a, long long b) { return (int)((a + b - 1) / b); }

}  // namespace

FusedPlan fused_plan(const Geom& g, int num_sms) {
    FusedPlan p;
    const int target = 4 * num_sms;
    p.e1_tx = ceil_div(g.nx, E1_TX);
    p.e1_ty = ceil_div(g.ny, E1_TY);
    int cols1 = p.e1_tx * p.e1_ty;
    int nzc1 = std::min(std::max(1, ceil_div(target, cols1)),
                        std::max(1, ceil_div(g.nz, 8)));
    p.e1_zc = ceil_div(g.nz, nzc1);
    p.e1_tz = ceil_div(g.nz, p.e1_zc);
    p.e1_items = cols1 * p.e1_tz;
    p.e2_tx = ceil_div(g.nx, E2_TX);
    p.e2_ty = ceil_div(g.ny, E2_TY);
    int cols2 = p.e2_tx * p.e2_ty;
    int nzc2 = std::min(std::max(1, ceil_div(target, cols2)),
                        std::max(1, ceil_div(g.nz, 8)));
    p.e2_zc = ceil_div(g.nz, nzc2);
    p.e2_tz = ceil_div(g.nz, p.e2_zc);
    p.e2_items = cols2 * p.e2_tz;
    return p;
}

cudaError_t fused_setup() {
    cudaError_t e = attrs_all<float>();
    cudaError_t e2 = attrs_all<__nv_bfloat16>();
    return e != cudaSuccess ? e : e2;
}

int fused_tile_shift(const void* F, int dtype, const Geom& g,
                     const FusedPlan& pl, float* shift, cudaStream_t s) {
    if (dtype == LM_BF16)
        k_tile_shift<<<pl.e1_items, 256, 0, s>>>((const __nv_bfloat16*)F, g,
                                                  pl, shift);
    else
        k_tile_shift<<<pl.e1_items, 256, 0, s>>>((const float*)F, g, pl,
                                                  shift);
    return 1;
}

int eval_fused(const FusedLaunch& a, cudaStream_t s) {
    int n = 0;
    if (a.dtype == LM_BF16) {
        n += launch_e1_w<__nv_bfloat16>(a, s);
        n += launch_e2_r<__nv_bfloat16>(a, s);
    } else {
        n += launch_e1_w<float>(a, s);
        n += launch_e2_r<float>(a, s);
    }
    return n;
}

}  // namespace lmk
