// Pass 2 (the factored LM step and the compositive update, steps (c)-(d))
// and the device-side decision (step (e)), for every pair of a batch.
//
//   ghat = g / gmax
//   du   = -r ghat / (|ghat|^2 + lambda)             Eq. tile1 (Appendix A)
//   du   = -(H_tile + lambda I)^-1 r ghat            Eq. tilen (tile side k > 1)
//   v    = step * g  (Demons: g is the smoothed update of Eq. demons)
//   v    = step * du
//   u*   = v + u o (Id + v)                           Eq. compositive
//   u*  <- G_sigma_warp * u*   (edge-extended, optional)
// then, after the trial is evaluated, the damping rule of Eq. lambda-update
// and the rejection rule of Eq. rejection decide on device, per pair.
#include <algorithm>

#include "lm_kernels.cuh"
#include "lm_sample.cuh"

namespace lmk {
namespace {

constexpr int TPB = 256;

// Pooled curvature of Eq. tilen (tile side k > 1).  For every
// non-overlapping k x k x k tile T of the current gradient the kernel
// forms H_T = |T|^-1 sum_T g g^T and stores the inverse of
// A_T = H_T / gmax^2 + lambda I (the damped pooled curvature of ghat), so
// that the step kernel's solve is one 3 x 3 product per voxel.  A group
// of G = tile_group(k) warps owns one tile row and slice (ty, tz) (a
// block holds 8 / G of them) and walks it two strips of 32 / k whole
// tiles along x at a time: lane i of warp j sums g g^T of voxel columns
// x0 + i and x0 + cw + i over the (y, z) lines j, j + G, ... of the k x k
// lines of the strips (coalesced loads, several lines and both strips in
// flight); then one lane per tile adds the G partials of its k columns
// in a fixed order (deterministic) and inverts A_T by Cholesky,
// A^-1 = L^-T L^-1 (reciprocal square roots of the pivots, about 2 ulp
// each).  Every pivot of H + lambda I is >= lambda
// (each Schur complement of a matrix >= lambda I is >= lambda I), so a
// pivot that rounding pushes below lambda is raised back to it.  Runs
// before the step kernel of every attempt, as lambda changes between
// retries.
constexpr int TH_W = TILE_WARPS;

__device__ __forceinline__ void spd3_inverse(float a00, float a01, float a02,
                                             float a11, float a12, float a22,
                                             float lam, float inv[6]) {
    // M = L^-1 from the reciprocal square roots of the pivots (the
    // factor L itself is never needed: l_ij = a_ij m_jj - ...)
    const float m00 = rsqrtf(fmaxf(a00, lam));
    const float l10 = a01 * m00, l20 = a02 * m00;
    const float m11 = rsqrtf(fmaxf(a11 - l10 * l10, lam));
    const float l21 = (a12 - l20 * l10) * m11;
    const float m22 = rsqrtf(fmaxf(a22 - l20 * l20 - l21 * l21, lam));
    const float m10 = -l10 * m00 * m11;
    const float m21 = -l21 * m11 * m22;
    const float m20 = -(l20 * m00 + l21 * m10) * m22;
    // A^-1 = M^T M: xx, xy, xz, yy, yz, zz
    inv[0] = m00 * m00 + m10 * m10 + m20 * m20;
    inv[1] = m10 * m11 + m20 * m21;
    inv[2] = m20 * m22;
    inv[3] = m11 * m11 + m21 * m21;
    inv[4] = m21 * m22;
    inv[5] = m22 * m22;
}

__global__ void __launch_bounds__(TH_W * 32)
    k_tile_hess(const PairDesc* __restrict__ pd, int npairs, int attempt,
                int k) {
    __shared__ float part[TH_W][6][64];
    const PairDesc& P = pd[pair_of_block<5>(pd, npairs, blockIdx.x)];
    const DevState* st = P.st;
    if (attempt_skip(st, attempt)) return;   // block-uniform
    const Geom g = P.g;
    const int G = tile_group(k);             // warps per tile row
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int lead = warp / G * G, j = warp - lead;
    const int row = (blockIdx.x - P.th_blk0) * (TH_W / G) + warp / G;
    const bool has_row = row < P.th_ny * P.th_nz;
    const int ty = row % P.th_ny, tz = row / P.th_ny;
    const int y0 = ty * k, y1 = min(y0 + k, g.ny);
    const int z0 = tz * k, z1 = min(z0 + k, g.nz);
    const int ky = y1 - y0, nlines = ky * (z1 - z0);
    const float* __restrict__ gg = st->cg ? P.g1 : P.g0;
    const int sxy = g.nx * g.ny;
    // this warp's lines j, j + G, ... (at most 32): lane i holds the
    // offset of line j + i G, broadcast to the warp in the sum loop
    const int nl = has_row ? (nlines - j + G - 1) / G : 0;
    int my_off = 0;
    if (lane < nl) {
        const int l = j + lane * G, dz = l / ky;
        my_off = (z0 + dz) * sxy + (y0 + l - dz * ky) * g.nx;
    }
    // |T|^-1 gmax^-2 of a full tile along x and of the cut last one, and
    // lambda
    const float gm = st->gmax;
    const float ig = gm > 0.f ? 1.f / gm : 0.f;
    const float lam = (float)st->lambda;
    const float sc_full = ig * ig / (float)(nlines * k);
    const int w_last = g.nx - (g.nx - 1) / k * k;
    const float sc_last = ig * ig / (float)(nlines * w_last);
    // two strips of cw columns (whole tiles) per pass: lane i takes
    // columns x0 + i and x0 + cw + i
    const int cw = 32 / k * k;
    for (int x0 = 0; x0 < g.nx; x0 += 2 * cw) {
        const int xa = x0 + lane, xb = xa + cw;
        const bool aa = lane < cw && xa < g.nx;
        const bool ab = lane < cw && xb < g.nx;
        const float* pa = gg + (aa ? xa : 0);
        const float* pb = gg + (ab ? xb : 0);
        float h[12];
#pragma unroll
        for (int e = 0; e < 12; ++e) h[e] = 0.f;
#pragma unroll 4
        for (int it = 0; it < nl; ++it) {
            const int i = __shfl_sync(0xffffffffu, my_off, it);
            if (aa) {
                const float a0 = __ldg(pa + i);
                const float a1 = __ldg(pa + g.V + i);
                const float a2 = __ldg(pa + 2 * g.V + i);
                h[0] = fmaf(a0, a0, h[0]);
                h[1] = fmaf(a0, a1, h[1]);
                h[2] = fmaf(a0, a2, h[2]);
                h[3] = fmaf(a1, a1, h[3]);
                h[4] = fmaf(a1, a2, h[4]);
                h[5] = fmaf(a2, a2, h[5]);
            }
            if (ab) {
                const float b0 = __ldg(pb + i);
                const float b1 = __ldg(pb + g.V + i);
                const float b2 = __ldg(pb + 2 * g.V + i);
                h[6] = fmaf(b0, b0, h[6]);
                h[7] = fmaf(b0, b1, h[7]);
                h[8] = fmaf(b0, b2, h[8]);
                h[9] = fmaf(b1, b1, h[9]);
                h[10] = fmaf(b1, b2, h[10]);
                h[11] = fmaf(b2, b2, h[11]);
            }
        }
#pragma unroll
        for (int e = 0; e < 6; ++e) {
            part[warp][e][lane] = h[e];
            part[warp][e][32 + lane] = h[6 + e];
        }
        __syncthreads();
        // one lane per tile of the two strips (at most 2 x 16)
        const int ntile = cw / k;
        const int sb = lane >= ntile;           // strip of this lane's tile
        const int tl = lane - sb * ntile;       // tile within the strip
        const int xt0 = x0 + sb * cw + tl * k;
        if (has_row && j == 0 && lane < 2 * ntile && xt0 < g.nx) {
            const int w = min(k, g.nx - xt0);
            const int c0 = sb * 32 + tl * k;
            float sum[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
            for (int q = 0; q < G; ++q)
                for (int c = 0; c < w; ++c)
#pragma unroll
                    for (int e = 0; e < 6; ++e)
                        sum[e] += part[lead + q][e][c0 + c];
            const float sc = w == k ? sc_full : sc_last;
            float inv[6];
            spd3_inverse(fmaf(sum[0], sc, lam), sum[1] * sc, sum[2] * sc,
                         fmaf(sum[3], sc, lam), sum[4] * sc,
                         fmaf(sum[5], sc, lam), lam, inv);
            float* dst = P.tileH +
                         ((size_t)(tz * P.th_ny + ty) * P.th_nx + xt0 / k) * 8;
            *(float4*)dst = make_float4(inv[0], inv[1], inv[2], inv[3]);
            *(float4*)(dst + 4) = make_float4(inv[4], inv[5], 0.f, 0.f);
        }
        __syncthreads();
    }
}

// Trial field, one voxel per thread.  A block owns a 32 x 8 x-y tile and a
// z range of one pair; the planes z-1, z, z+1 of u (3 components, with a
// one-voxel x-y halo, read at edge-clamped positions) sit in an eight-slot
// shared-memory ring that cp.async fills two planes ahead (the block's g
// tile of each slice rides along three slices ahead of its use, in a
// four-slot ring of its own), so the trilinear
// read of u at p + v comes from shared memory whenever |v| < 1 along each
// axis and from global memory otherwise.  The trial goes to slot (1 - cu),
// or to the pair's warp-smoothing buffer.  Without warp smoothing the
// kernel also resamples M at the trial (J and dJ/du of the trial's
// evaluation, Section 2.1) while the trial is in registers, so the
// evaluation starts at the moment kernel.
constexpr int ST_X = 32, ST_Y = 8, ST_HX = ST_X + 2, ST_HY = ST_Y + 2;
constexpr int ST_PLANE = ST_HX * ST_HY;

// How the step kernel forms v from the current g.
enum StepMode {
    STEP_POINT = 0,   // Eq. tile1
    STEP_TILE = 1,    // Eq. tilen with the tile kernel's inverses
    STEP_DIRECT = 2,  // v = step * g (Demons)
};

__device__ __forceinline__ void cp_async4(float* dst, const float* src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(
                     (unsigned)__cvta_generic_to_shared(dst)),
                 "l"(src)
                 : "memory");
}
// zero-filled where !pred
__device__ __forceinline__ void cp_async4_zf(float* dst, const float* src, bool pred) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(
                     (unsigned)__cvta_generic_to_shared(dst)),
                 "l"(src), "r"(pred ? 4 : 0)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit_wait_all() {
    asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;\n" ::: "memory");
}
__device__ __forceinline__ void cp_async_commit() {
    asm volatile("cp.async.commit_group;\n" ::: "memory");
}

template <typename T, bool RESAMPLE, int MODE>
__global__ void __launch_bounds__(ST_X * ST_Y, 3)
    k_step_compose(const PairDesc* __restrict__ pd, int npairs, int attempt,
                   float step, int smooth, int tile) {
    __shared__ __align__(16) float ring[8][3][ST_PLANE];   // [slot][comp][y][x]
    __shared__ __align__(16) float gring[4][3][ST_X * ST_Y];   // g tiles
    const PairDesc& P = pd[pair_of_block<3>(pd, npairs, blockIdx.x)];
    const DevState* st = P.st;
    if (attempt_skip(st, attempt)) return;
    const Geom g = P.g;
    const int cu = st->cu, cg = st->cg;
    const float* __restrict__ u = cu ? P.u1 : P.u0;
    float* __restrict__ out = smooth ? P.wtmpA : (cu ? P.u0 : P.u1);
    const float* __restrict__ gg = cg ? P.g1 : P.g0;
    const T* __restrict__ M = (const T*)P.M;
    const float r = (float)st->L;
    const float lam = (float)st->lambda;
    const float gm = st->gmax;
    const float inv = gm > 0.f ? 1.f / gm : 0.f;
    const float scale = -r * step;
    JOut jo;
    if (RESAMPLE) jo = jout_of(P);

    const int b = blockIdx.x - P.st_blk0;
    const int bx = b % P.st_tx;
    const int rest = b / P.st_tx;
    const int by = rest % P.st_ty;
    const int bz = rest / P.st_ty;
    const int tid = threadIdx.y * ST_X + threadIdx.x;
    const int x0 = bx * ST_X, y0 = by * ST_Y;
    const int z0 = bz * P.st_zc;
    const int z1 = min(z0 + P.st_zc, g.nz);
    const int x = x0 + threadIdx.x, y = y0 + threadIdx.y;
    const int sxy = g.nx * g.ny;
    const int V = (int)g.V;
    // Tile-mode pair fields (read once)
    const float* __restrict__ tileH = MODE == STEP_TILE ? P.tileH : nullptr;

    // Each thread copies fixed halo positions of every plane; their clamped
    // in-plane sources (offsets from u, component included) and ring
    // offsets are computed once.
    constexpr int NLD = (3 * ST_PLANE + ST_X * ST_Y - 1) / (ST_X * ST_Y);
    int ld_src[NLD], ld_dst[NLD];
#pragma unroll
    for (int k = 0; k < NLD; ++k) {
        const int e = tid + k * ST_X * ST_Y;
        ld_dst[k] = -1;
        ld_src[k] = 0;
        if (e < 3 * ST_PLANE) {
            const int q = e / ST_PLANE, rem = e - q * ST_PLANE;
            const int hy = rem / ST_HX, hx = rem - hy * ST_HX;
            const int gx = min(max(x0 - 1 + hx, 0), g.nx - 1);
            const int gy = min(max(y0 - 1 + hy, 0), g.ny - 1);
            ld_src[k] = q * V + gy * g.nx + gx;
            ld_dst[k] = q * ST_PLANE + rem;
        }
    }
    // plane zp (edge-clamped) into ring slot zp mod 8
    auto issue_plane = [&](int zp) {
        const float* src = u + min(max(zp, 0), g.nz - 1) * sxy;
        float* dst = &ring[zp & 7][0][0];
#pragma unroll
        for (int k = 0; k < NLD; ++k)
            if (ld_dst[k] >= 0) cp_async4(dst + ld_dst[k], src + ld_src[k]);
    };
    const bool in_xy = x < g.nx && y < g.ny;
    // this thread's g at slice zp into g slot zp mod 4 (zero outside the
    // volume or past the block's range; only this thread reads it back)
    const int gxy = in_xy ? y * g.nx + x : 0;
    auto issue_g = [&](int zp) {
        const bool on = in_xy && zp < z1;
        const float* src = gg + (on ? zp * sxy + gxy : 0);
        float* dst = &gring[zp & 3][0][tid];
#pragma unroll
        for (int q = 0; q < 3; ++q)
            cp_async4_zf(dst + q * ST_X * ST_Y, src + (on ? q * V : 0), on);
    };
    issue_plane(z0 - 1);
    issue_plane(z0);
    issue_plane(z0 + 1);
    issue_g(z0);
    issue_g(z0 + 1);
    cp_async_commit_wait_all();
    // the first group in flight: plane z0 + 2 and g at z0 + 2
    if (z0 + 2 <= z1) issue_plane(z0 + 2);
    issue_g(z0 + 2);
    cp_async_commit();
    // Eq. tilen: this column's tiles (x / k, y / k fixed; z / k counted),
    // as tile indices of the pair's table
    int tile_col = 0, tile_slice = 0, tz_ = 0, tzr = 0;
    if (MODE == STEP_TILE) {
        tile_col = (y / tile) * P.th_nx + x / tile;
        tile_slice = P.th_nx * P.th_ny;
        tz_ = z0 / tile;
        tzr = z0 - tz_ * tile;
    }
    int i = z0 * sxy + y * g.nx + x;
    __syncthreads();
    // resampling is pipelined by one voxel: the corners of M at the trial of
    // voxel z are requested at step z and consumed at step z + 1
    float pm[8], pf[3];
    bool have = false;
    for (int z = z0; z < z1; ++z, i += sxy) {
        // plane z + 3 (read from step z + 2 on) and g at z + 3 stream into
        // their slots, the ones plane z - 5 and g at z - 1 left
        if (z + 3 <= z1) issue_plane(z + 3);
        issue_g(z + 3);
        cp_async_commit();
        const float cg0 = gring[z & 3][0][tid], cg1 = gring[z & 3][1][tid],
                    cg2 = gring[z & 3][2][tid];
        if (in_xy) {
            float v[3];
            if (MODE == STEP_DIRECT) {
                v[0] = cg0 * step;
                v[1] = cg1 * step;
                v[2] = cg2 * step;
            } else {
                const float gh0 = cg0 * inv, gh1 = cg1 * inv, gh2 = cg2 * inv;
                if (MODE == STEP_TILE) {
                    // the tile's (H / gmax^2 + lambda I)^-1, symmetric
                    const float* a8 = tileH + (size_t)(tz_ * tile_slice + tile_col) * 8;
                    const float4 ia = __ldg((const float4*)a8);
                    const float4 ib = __ldg((const float4*)(a8 + 4));
                    v[0] = scale * (ia.x * gh0 + ia.y * gh1 + ia.z * gh2);
                    v[1] = scale * (ia.y * gh0 + ia.w * gh1 + ib.x * gh2);
                    v[2] = scale * (ia.z * gh0 + ib.x * gh1 + ib.y * gh2);
                } else {
                    // n2 + lam >= lam > 0 in every iteration: the
                    // approximate division (about 2 ulp) is safe; a context
                    // timed before its first reset (lambda 0, g 0) steps 0
                    const float n2 = gh0 * gh0 + gh1 * gh1 + gh2 * gh2;
                    const float den = n2 + lam;
                    const float sc = den > 0.f ? __fdividef(scale, den) : 0.f;
                    v[0] = gh0 * sc;
                    v[1] = gh1 * sc;
                    v[2] = gh2 * sc;
                }
            }
            float fl[3], f[3];
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                fl[k] = safe_floor(v[k]);
                f[k] = v[k] - fl[k];
            }
            const int cx = x + (int)fl[0], cy = y + (int)fl[1], cz = z + (int)fl[2];
            const float wx1 = f[0], wx0 = 1.f - f[0];
            const float wy1 = f[1], wy0 = 1.f - f[1];
            const float wz1 = f[2], wz0 = 1.f - f[2];
            float m[3][8];
            if (cx >= x0 - 1 && cx + 1 <= x0 + ST_X && cy >= y0 - 1 &&
                cy + 1 <= y0 + ST_Y && cz >= z - 1 && cz + 1 <= z + 1) {
                const int o = (cy - (y0 - 1)) * ST_HX + cx - (x0 - 1);
                const float* p0 = &ring[cz & 7][0][0] + o;
                const float* p1 = &ring[(cz + 1) & 7][0][0] + o;
#pragma unroll
                for (int q = 0; q < 3; ++q) {
                    m[q][0] = p0[q * ST_PLANE];
                    m[q][1] = p0[q * ST_PLANE + 1];
                    m[q][2] = p0[q * ST_PLANE + ST_HX];
                    m[q][3] = p0[q * ST_PLANE + ST_HX + 1];
                    m[q][4] = p1[q * ST_PLANE];
                    m[q][5] = p1[q * ST_PLANE + 1];
                    m[q][6] = p1[q * ST_PLANE + ST_HX];
                    m[q][7] = p1[q * ST_PLANE + ST_HX + 1];
                }
            } else {
                const int ax = min(max(cx, 0), g.nx - 1), bx2 = min(max(cx + 1, 0), g.nx - 1);
                const int ay = min(max(cy, 0), g.ny - 1), by2 = min(max(cy + 1, 0), g.ny - 1);
                const int az = min(max(cz, 0), g.nz - 1), bz2 = min(max(cz + 1, 0), g.nz - 1);
                const int o000 = az * sxy + ay * g.nx;
                const int o010 = az * sxy + by2 * g.nx;
                const int o001 = bz2 * sxy + ay * g.nx;
                const int o011 = bz2 * sxy + by2 * g.nx;
#pragma unroll
                for (int q = 0; q < 3; ++q) {
                    const float* U = u + q * V;
                    m[q][0] = __ldg(U + o000 + ax);
                    m[q][1] = __ldg(U + o000 + bx2);
                    m[q][2] = __ldg(U + o010 + ax);
                    m[q][3] = __ldg(U + o010 + bx2);
                    m[q][4] = __ldg(U + o001 + ax);
                    m[q][5] = __ldg(U + o001 + bx2);
                    m[q][6] = __ldg(U + o011 + ax);
                    m[q][7] = __ldg(U + o011 + bx2);
                }
            }
            float ut[3];
#pragma unroll
            for (int q = 0; q < 3; ++q) {
                float sv = wz0 * (wy0 * (wx0 * m[q][0] + wx1 * m[q][1]) +
                                  wy1 * (wx0 * m[q][2] + wx1 * m[q][3])) +
                           wz1 * (wy0 * (wx0 * m[q][4] + wx1 * m[q][5]) +
                                  wy1 * (wx0 * m[q][6] + wx1 * m[q][7]));
                ut[q] = v[q] + sv;
                out[q * V + i] = ut[q];
            }
            if (RESAMPLE) {
                float cm[8], cf[3];
                corners(M, g, x, y, z, ut[0], ut[1], ut[2], cm, cf);
                if (have) store_resampled(jo, i - sxy, x, y, z - 1, pm, pf);
#pragma unroll
                for (int k = 0; k < 8; ++k) pm[k] = cm[k];
                pf[0] = cf[0];
                pf[1] = cf[1];
                pf[2] = cf[2];
                have = true;
            }
        }
        if (MODE == STEP_TILE && ++tzr == tile) {
            tzr = 0;
            ++tz_;
        }
        // the group issued at step z - 1 (plane z + 2, g at z + 2) has
        // landed, this step's may still be in flight; the barrier makes the
        // plane's copies of every thread visible before step z + 1
        asm volatile("cp.async.wait_group 1;\n" ::: "memory");
        __syncthreads();
    }
    if (RESAMPLE && have) store_resampled(jo, i - sxy, x, y, z1 - 1, pm, pf);
}

// 1-D Gaussian along an axis of a pair's 3-component field, edge-extended;
// pass 0: wtmpA -> wtmpB (x), 1: wtmpB -> wtmpA (y), 2: wtmpA -> trial
// slot (1 - cu) (z).  One thread per voxel.
__global__ void k_warp_gauss(const PairDesc* __restrict__ pd, int npairs,
                             int attempt, Taps t, int axis) {
    const PairDesc& P = pd[pair_of_block<4>(pd, npairs, blockIdx.x)];
    if (attempt_skip(P.st, attempt)) return;
    const Geom g = P.g;
    long long i = (long long)(blockIdx.x - P.ln_blk0) * blockDim.x + threadIdx.x;
    if (i >= g.V) return;
    const float* in = axis == 1 ? P.wtmpB : P.wtmpA;
    float* dst = axis == 0 ? P.wtmpB
                           : (axis == 1 ? P.wtmpA : (P.st->cu ? P.u0 : P.u1));
    int x = (int)(i % g.nx);
    long long rr = i / g.nx;
    int y = (int)(rr % g.ny), z = (int)(rr / g.ny);
    int pos = axis == 0 ? x : (axis == 1 ? y : z);
    int n = axis == 0 ? g.nx : (axis == 1 ? g.ny : g.nz);
    long long stride = axis == 0 ? 1 : (axis == 1 ? g.nx : (long long)g.nx * g.ny);
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

__device__ __forceinline__ long long block_sum1024_ll(long long v, long long* sh) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) sh[wid] = v;
    __syncthreads();
    v = (threadIdx.x < (blockDim.x >> 5)) ? sh[threadIdx.x] : 0;
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

// One CTA per pair: fixed-order FP64 reduction of the pair's partials
// (deterministic), then the per-mode state update.
__device__ __forceinline__ void finalize_pair(const PairDesc* __restrict__ pd,
                                              const Partials& part,
                                              const DecideConsts& d, int mode,
                                              int attempt,
                                              EvalOut* __restrict__ outs) {
    __shared__ long long shl[32];
    __shared__ float shf[32];
    const PairDesc& P = pd[blockIdx.x];
    DevState* st = P.st;
    if (mode == FIN_DECIDE && attempt_skip(st, attempt)) return;
    // exact: integer partials in fixed point LOSS_Q
    long long s = 0;
    int lbad = 0;
    for (int i = threadIdx.x; i < P.e1_ncta; i += blockDim.x) {
        const long long v = part.loss[P.e1_cta0 + i];
        if (v == LOSS_BAD) lbad = 1;
        else s += v;
    }
    lbad = __syncthreads_or(lbad);
    s = block_sum1024_ll(s, shl);
    float m = 0.f;
    int nf = 0, to = 0;
    for (int i = threadIdx.x; i < P.e2_ncta; i += blockDim.x) {
        float v = part.g2max[P.e2_cta0 + i];
        if (v < 0.f) to = 1;                 // E2's bounded wait ran out
        else if (!(v <= 3.0e38f)) nf = 1;    // NaN or overflow
        else m = fmaxf(m, v);
    }
    nf = __syncthreads_or(nf);
    to = __syncthreads_or(to);
    m = block_max1024(m, shf);
    if (threadIdx.x != 0) return;
    double L;
    if (d.mi) {
        L = part.mi_loss[blockIdx.x];   // r = log2 B - MI, from k_mi_table
    } else if (d.mse) {
        // exact MSE sum in units of 2^shift / Q^2
        const QScale q = *P.qs;
        L = (double)s * ldexp(1.0, mse_shift(q.qlim)) /
            ((double)q.Q * (double)q.Q) / (double)P.g.V;
    } else {
        L = ((double)s / (double)LOSS_Q) / (double)P.g.V;
    }
    float gmax = sqrtf(m);
    // a non-finite J of this evaluation (its flag is cleared here) or F
    const unsigned fl = *P.flags;
    if (fl & QFLAG_JBAD) *P.flags = fl & ~QFLAG_JBAD;
    const bool nonfinite = nf || lbad || fl || !isfinite(L) || !isfinite(gmax);
    const bool bad = nonfinite || to;
    const int bits = (nonfinite ? STATUS_NONFINITE : 0) | (to ? STATUS_TIMEOUT : 0);
    if (mode == FIN_EXPLICIT) {
        EvalOut* o = outs + blockIdx.x;
        o->L = L;
        o->gmax = gmax;
        o->status = bits;
        return;
    }
    if (mode == FIN_RESET) {
        st->L = L;
        st->L_prev = 0.0;
        st->L_trial = L;
        st->L_first = L;
        st->lambda = d.lambda0;
        st->gmax = gmax;
        st->gmax_trial = gmax;
        st->has_prev = 0;
        st->cu = 0;
        st->cg = 0;
        st->retries = 0;
        st->done = 0;
        st->accepted = 0;
        st->status = bits;
        st->iter = 0;
        st->evals = 1;
        st->log_pos = 0;
        st->stopped = 0;
        st->att = 0;
        st->iter_end = 0;
        return;
    }
    // FIN_DECIDE
    const int j = attempt_of(st, attempt);
    st->evals += 1;
    st->L_trial = L;
    st->gmax_trial = gmax;
    if (j == 0) {
        st->L_first = L;
        st->retries = 0;
    }
    double lam = st->lambda;
    int finished = 0, accepted = 0;
    if (bad) {
        st->status |= bits;
        finished = 1;   // the trial is dropped, the state kept
    } else if (d.demons) {
        finished = 1;   // Demons keeps every step; lambda is unused
        accepted = 1;
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
                st->att = j + 1;   // the next state-driven pass retries
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
    st->att = 0;   // the next state-driven pass starts an iteration
    st->iter += 1;
    if (st->L <= P.target) st->stopped = 1;   // false for a NaN target
    if (P.log) {
        int pos = st->log_pos;
        LogEntry e;
        e.loss = st->L;
        e.lambda = lam;
        e.gmax = st->gmax;
        e.accepted = accepted;
        e.retries = j;
        e.pad = 0;
        P.log[pos % LOG_CAP] = e;
        st->log_pos = pos + 1;
    }
}

// One CTA per pair: fixed-order reduction of the pair's partials, then the
// per-mode state update.
__global__ void k_finalize(const PairDesc* __restrict__ pd, Partials part,
                           DecideConsts d, int mode, int attempt,
                           EvalOut* __restrict__ outs) {
    finalize_pair(pd, part, d, mode, attempt, outs);
}

// iter_end of every pair: iter + n, or 0 (no limit) for n = 0.
__global__ void k_iter_end(const PairDesc* __restrict__ pd, int npairs, int n) {
    for (int i = threadIdx.x; i < npairs; i += blockDim.x) {
        DevState* st = pd[i].st;
        st->iter_end = n > 0 ? st->iter + n : 0;
    }
}

__global__ void k_copy_back(const PairDesc* __restrict__ pd, int npairs) {
    const PairDesc& P = pd[pair_of_block<4>(pd, npairs, blockIdx.x)];
    if (P.st->cu == 0) return;
    long long i = (long long)(blockIdx.x - P.ln_blk0) * blockDim.x + threadIdx.x;
    if (i >= P.g.V) return;
    for (int q = 0; q < 3; ++q) P.u0[q * P.g.V + i] = P.u1[q * P.g.V + i];
}

__global__ void k_flip_slot(const PairDesc* __restrict__ pd) {
    if (threadIdx.x == 0) pd[blockIdx.x].st->cu = 0;
}

}  // namespace

bool step_resamples(const Batch& b) { return b.wtaps.R == 0; }

template <int MODE>
int launch_step(const Batch& b, int attempt, cudaStream_t s) {
    const int smooth = b.wtaps.R > 0;
    const dim3 grid(b.plan.st_blocks), block(ST_X, ST_Y);
    if (!smooth) {
        if (b.dtype == LM_BF16)
            k_step_compose<__nv_bfloat16, true, MODE><<<grid, block, 0, s>>>(
                b.pd, b.npairs, attempt, b.step, 0, b.tile);
        else
            k_step_compose<float, true, MODE><<<grid, block, 0, s>>>(
                b.pd, b.npairs, attempt, b.step, 0, b.tile);
        return 1;
    }
    k_step_compose<float, false, MODE><<<grid, block, 0, s>>>(
        b.pd, b.npairs, attempt, b.step, 1, b.tile);
    for (int axis = 0; axis < 3; ++axis)
        k_warp_gauss<<<b.plan.ln_blocks, TPB, 0, s>>>(b.pd, b.npairs, attempt,
                                                      b.wtaps, axis);
    return 4;
}

int batch_step(const Batch& b, int attempt, cudaStream_t s) {
    if (b.method == LM_METHOD_DEMONS)
        return launch_step<STEP_DIRECT>(b, attempt, s);
    if (b.tile <= 1) return launch_step<STEP_POINT>(b, attempt, s);
    k_tile_hess<<<b.th_blocks, TH_W * 32, 0, s>>>(b.pd, b.npairs, attempt,
                                                  b.tile);
    return 1 + launch_step<STEP_TILE>(b, attempt, s);
}

// The decision kernel's CTA: a few hundred partials per pair at most, so
// a small CTA keeps its two reduction barriers short (the sums are exact,
// so the result does not depend on the size).
constexpr int FIN_THREADS = 256;

int batch_finalize(const Batch& b, int mode, int attempt, EvalOut* out,
                   cudaStream_t s) {
    k_finalize<<<b.npairs, FIN_THREADS, 0, s>>>(b.pd, b.part, b.d, mode,
                                                attempt, out);
    return 1;
}

int batch_set_iter_end(const Batch& b, int n, cudaStream_t s) {
    k_iter_end<<<1, 256, 0, s>>>(b.pd, b.npairs, n);
    return 1;
}

int batch_sync_back(const Batch& b, cudaStream_t s) {
    k_copy_back<<<b.plan.ln_blocks, TPB, 0, s>>>(b.pd, b.npairs);
    k_flip_slot<<<b.npairs, 32, 0, s>>>(b.pd);
    return 2;
}

}  // namespace lmk
