// Pass 1 (loss and smoothed gradient, steps (a)-(c)) as a per-voxel
// resampling kernel (J pass) and two z-streaming kernels.  Each CTA owns a column of the volume (an x-y tile) and a range
// of z, marching along z with the planes of every stage in shared memory;
// separable box and Gaussian filters run along x and y on the planes and
// along z on ring buffers of the last k planes.
//
//  J pass: J = M(p + u) and dJ/du (trilinear, Section 2.1), J in the fixed
//     point of the moments (int32) and dJ/du (FP32) to HBM.
//  E1 (lncc): the LNCC window moments of F' and J' (k^3 box, zero padding); per voxel (1 - cc) and the backward
//     coefficients (a, b, c) of the squared-loss form (Section 2.2); their
//     box sums; and
//        dL/dJ(y) = -V^-1 [F'(y) Box(a) + 2 J'(y) Box(b) + Box(c)]
//     plus the CTA's loss partial.
//     E1 writes g_raw = dL/dJ * dJ/du (12 bytes / voxel).
//  E2 (grad): separable Gaussian of g_raw (R = ceil(3 sigma), zero
//     padding), g to HBM, CTA max |g|^2.
//
// Window moments are exact: F' = F - s and J' = J - s are rounded to fixed
// point (Xq = round(X' * Q), |Xq| <= 2^qb) and the window sums of Xq and of
// the products Xq*Yq are int64, so A, B, C come out of exact integer
// differences k^3 S_XY - S_X S_Y; only their final conversion rounds.  The
// variance cancellation that FP32 window sums suffer in flat regions is
// gone.  Everything after the moments is FP32.
//
// The fixed image's share of the moments (F' in fixed point, its exact
// window sum and its window variance) does not change during a
// registration; the preparation kernels compute it once per reset.
//
// HBM traffic per voxel: the J pass reads u, M (16 B) and writes Jq, dJ
// (16 B); E1 reads F', S_F, B, Jq, dJ (28 B) and writes g_raw (12 B); E2
// reads g_raw (12 B) and writes g (12 B).  Halo re-reads hit L2.  For the
// MSE loss and for Demons a pointwise kernel takes E1's place.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <vector>

#include "lm_kernels.cuh"
#include "lm_sample.cuh"

namespace lmk {
namespace {

constexpr int NT = 512;       // threads per CTA (both kernels)
constexpr int PLANE_X = 32;   // E1 moment plane / E2 output tile width
constexpr int PLANE_Y = 16;   // and height


// ----------------------------------------------------------------------
// J pass: per voxel J = M(p + u(p)) and dJ/du (trilinear, Section 2.1), J
// rounded to the fixed point of the window moments (JQ_BAD marks a
// non-finite J), dJ/du kept in FP32.  One thread per x-y column of a 32 x 8
// tile, marching over the tile's z range (the step kernel's tiling).
// ----------------------------------------------------------------------
constexpr int FQ_BAD = JQ_BAD;   // same sentinel for a non-finite F

template <typename T>
__global__ void __launch_bounds__(256)
    k_jpass(const PairDesc* __restrict__ pd, int npairs, int mode, int attempt) {
    const PairDesc& P = pd[pair_of_block<3>(pd, npairs, blockIdx.x)];
    if (trial_skip(P, mode, attempt)) return;
    const Geom g = P.g;
    const int b = blockIdx.x - P.st_blk0;
    const int bx = b % P.st_tx;
    const int rest = b / P.st_tx;
    const int by = rest % P.st_ty;
    const int bz = rest / P.st_ty;
    const int x = bx * 32 + threadIdx.x, y = by * 8 + threadIdx.y;
    if (x >= g.nx || y >= g.ny) return;
    const int z0 = bz * P.st_zc;
    const int z1 = min(z0 + P.st_zc, g.nz);
    const T* __restrict__ M = (const T*)P.M;
    const float* __restrict__ u = eval_u(P, mode);
    const JOut jo = jout_of(P);
    const int sxy = g.nx * g.ny;
    int i = z0 * sxy + y * g.nx + x;
    float nu0 = 0.f, nu1 = 0.f, nu2 = 0.f;
    if (z0 < z1) {
        nu0 = __ldg(u + i);
        nu1 = __ldg(u + g.V + i);
        nu2 = __ldg(u + 2 * g.V + i);
    }
    for (int z = z0; z < z1; ++z, i += sxy) {
        // u of the next slice streams in while this one is resampled
        const float d0 = nu0, d1 = nu1, d2 = nu2;
        if (z + 1 < z1) {
            nu0 = __ldg(u + i + sxy);
            nu1 = __ldg(u + g.V + i + sxy);
            nu2 = __ldg(u + 2 * g.V + i + sxy);
        }
        resample_voxel(jo, g, M, x, y, z, i, d0, d1, d2);
    }
}


// ----------------------------------------------------------------------
// Pointwise evaluation for MSE (Section 2.2) and Demons (Section 2.3), in
// place of E1.  Per voxel: dq = Fq - Jq, the fixed-point F - J (exact);
// the loss term dq^2, rounded to the MSE unit (mse_shift) and summed
// exactly; and g_raw:
//   MSE:    g_raw = dL/dJ dJ/du,  dL/dJ = -2 (F - J) / V
//   Demons: g_raw = r n / (|n|^2 + alpha^2 r^2), r = F - J, n = dJ/du
//           (Eq. demons; 0 where r and n both vanish)
// The CTAs of a pair (its E1 partial slots) split its voxels into
// contiguous ranges.  HBM traffic per voxel: Fq, Jq, dJ/du (20 B) in,
// g_raw (12 B) out.
// ----------------------------------------------------------------------
constexpr int NTP = 1024;   // pointwise kernel threads per CTA (one CTA per slot)

template <bool DEMONS>
__global__ void __launch_bounds__(NTP)
    k_pointwise(const PairDesc* __restrict__ pd, int npairs, int mode,
                int attempt, float alpha, long long* __restrict__ loss_part) {
    __shared__ long long red[NTP / 32];
    const PairDesc& P = pd[pair_of_block<1>(pd, npairs, blockIdx.x)];
    if (trial_skip(P, mode, attempt)) return;
    const Geom g = P.g;
    const int c = blockIdx.x - P.e1_cta0;
    const long long i0 = g.V * c / P.e1_ncta, i1 = g.V * (c + 1) / P.e1_ncta;
    const int* __restrict__ fqv = P.fq;
    const int* __restrict__ jqv = P.jq;
    const float* __restrict__ djv = P.dj;
    float* __restrict__ graw = P.graw;
    const float iQ = P.qs->invQ;
    const int sh = mse_shift(P.qs->qlim);
    const long long half = sh > 0 ? 1LL << (sh - 1) : 0;
    const float coef = -2.f / (float)g.V;
    const float a2 = alpha * alpha;
    const int gpw = P.gp_w;
    const long long gcs = (long long)g.nz * g.ny * gpw;
    const bool dense = gpw == g.nx;
    long long lacc = 0;
    bool bad = false;
    // two voxels per thread and pass, all loads issued before any use
    constexpr int U = 2;
    for (long long base = i0; base < i1; base += (long long)U * NTP) {
        int fq[U], jq[U];
        float d[U][3];
#pragma unroll
        for (int k = 0; k < U; ++k) {
            const long long i = base + threadIdx.x + (long long)k * NTP;
            const bool in = i < i1;
            fq[k] = in ? __ldg(fqv + i) : 0;
            jq[k] = in ? __ldg(jqv + i) : 0;
            d[k][0] = in ? __ldg(djv + i) : 0.f;
            d[k][1] = in ? __ldg(djv + g.V + i) : 0.f;
            d[k][2] = in ? __ldg(djv + 2 * g.V + i) : 0.f;
        }
#pragma unroll
        for (int k = 0; k < U; ++k) {
            const long long i = base + threadIdx.x + (long long)k * NTP;
            if (i >= i1) break;
            float sc = 0.f;
            if (fq[k] == FQ_BAD || jq[k] == JQ_BAD) {
                bad = true;
            } else {
                const int dq = fq[k] - jq[k];
                lacc += ((long long)dq * dq + half) >> sh;
                const float r = (float)dq * iQ;
                if (DEMONS) {
                    const float den = d[k][0] * d[k][0] + d[k][1] * d[k][1] +
                                      d[k][2] * d[k][2] + a2 * r * r;
                    sc = den > 0.f ? r / den : 0.f;
                } else {
                    sc = coef * r;
                }
            }
            const long long gi =
                dense ? i : (i / g.nx) * gpw + (i - (i / g.nx) * g.nx);
            graw[gi] = sc * d[k][0];
            graw[gcs + gi] = sc * d[k][1];
            graw[2 * gcs + gi] = sc * d[k][2];
        }
    }
    for (int o = 16; o > 0; o >>= 1) lacc += __shfl_down_sync(0xffffffffu, lacc, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = lacc;
    const int any_bad = __syncthreads_or(bad);
    if (threadIdx.x == 0) {
        long long v = 0;
        for (int w = 0; w < NTP / 32; ++w) v += red[w];
        loss_part[blockIdx.x] = any_bad ? LOSS_BAD : v;
    }
}

// ----------------------------------------------------------------------
// E2
// ----------------------------------------------------------------------
// 256 threads: in the y and z passes each thread owns two x-adjacent
// outputs of one row with all three components (8-byte shared-memory reads,
// 8-byte global stores), and the z window of those six values sits in a
// register ring.  The g_raw plane of each slice (three components with the
// halo) arrives by one TMA tile load into a ring of E2_NB buffers, issued
// E2_NB slices ahead and tracked by an mbarrier per buffer.
constexpr int NT2 = 256;
constexpr int E2_NB = 4;

template <int R>
struct E2Cfg {
    static constexpr int KG = 2 * R + 1;
    static constexpr int TX = PLANE_X, TY = PLANE_Y;
    // the TMA box starts at x0 - RA, a multiple of 4 floats (16 bytes)
    static constexpr int RA = (R + 3) / 4 * 4;
    static constexpr int BX = TX + 2 * RA, BY = TY + 2 * R;
    static constexpr int NQ = TX / 4;               // quads per row
    static constexpr int NXU = 3 * BY * NQ;         // x-pass units (4 outputs)
    static constexpr int TXB = 3 * BY * BX * 4;     // bytes per TMA tile
    static constexpr int GRF = (3 * BY * BX + 31) / 32 * 32;   // floats/buffer
    static_assert(TX * TY == 2 * NT2, "two outputs per thread");
    // g_raw tiles and the x-smoothed plane (+ alignment)
    static constexpr int bytes = 128 + (E2_NB * GRF + 3 * BY * TX) * 4;
};

__device__ __forceinline__ unsigned smem_u32(const void* p) {
    return (unsigned)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(unsigned long long* b, unsigned n) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(b)),
                 "r"(n)
                 : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(unsigned long long* b,
                                               unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(
                     smem_u32(b)),
                 "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(unsigned long long* b,
                                              unsigned parity) {
    unsigned ok;
    asm volatile(
        "{\n .reg .pred p;\n"
        " mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(b)), "r"(parity)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ unsigned long long globaltimer_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;\n" : "=l"(t));
    return t;
}
// Bounded wait: false if the phase did not complete within 2^20 polls or
// half a second, whichever comes first (a TMA tile lands in microseconds).
constexpr unsigned long long WAIT_NS = 500000000ull;
__device__ __forceinline__ bool mbar_wait(unsigned long long* b, unsigned parity) {
    if (mbar_try_wait(b, parity)) return true;
    const unsigned long long t0 = globaltimer_ns();
    for (int it = 1; it < (1 << 20); ++it) {
        if (mbar_try_wait(b, parity)) return true;
        if ((it & 63) == 0 && globaltimer_ns() - t0 > WAIT_NS) return false;
    }
    return false;
}
__device__ __forceinline__ void tma_load_4d(void* dst, const void* map, int x,
                                            int y, int z, int c,
                                            unsigned long long* bar) {
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_"
        "tx::bytes [%0], [%1, {%2, %3, %4, %5}], [%6];\n" ::"r"(smem_u32(dst)),
        "l"(map), "r"(x), "r"(y), "r"(z), "r"(c), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ float4 f4_fma(float a, float4 x, float4 y) {
    return make_float4(fmaf(a, x.x, y.x), fmaf(a, x.y, y.y), fmaf(a, x.z, y.z),
                       fmaf(a, x.w, y.w));
}
__device__ __forceinline__ float4 f4_add(float4 x, float4 y) {
    return make_float4(x.x + y.x, x.y + y.y, x.z + y.z, x.w + y.w);
}
__device__ __forceinline__ float4 f4_mul(float a, float4 x) {
    return make_float4(a * x.x, a * x.y, a * x.z, a * x.w);
}

template <int R, typename T>
__global__ void __launch_bounds__(NT2, R <= 3 ? 3 : 2)
    k_e2(const PairDesc* __restrict__ pd, int npairs, int mode, int attempt,
         Taps tp, float* __restrict__ g2_part) {
    using C = E2Cfg<R>;
    constexpr int KG = C::KG, BX = C::BX, BY = C::BY, RA = C::RA;
    constexpr int TX = C::TX, TY = C::TY, NQ = C::NQ, GRF = C::GRF;
    constexpr int NXS = (C::NXU + NT2 - 1) / NT2;        // x-pass slots
    extern __shared__ __align__(128) unsigned char smem_raw[];
    float* Gr = (float*)(((size_t)smem_raw + 127) & ~(size_t)127);  // [NB][GRF]
    float* Gx = Gr + E2_NB * GRF;          // [3][BY][TX]
    __shared__ __align__(8) unsigned long long mbar[E2_NB];
    __shared__ float red[NT2 / 32];

    const PairDesc& P = pd[pair_of_block<2>(pd, npairs, blockIdx.x)];
    if (trial_skip(P, mode, attempt)) return;
    const Geom g = P.g;
    const int tid = threadIdx.x;
    float* __restrict__ gout = eval_g(P, mode);
    const int sxy = g.nx * g.ny;
    // taps stay in the kernel-parameter constant bank (no registers)
    const float* tt = tp.t;
    // y/z role: outputs 2 px, 2 px + 1 of row oy, all three components
    const int px = tid % (TX / 2), oy = tid / (TX / 2);
    int x_in[NXS], x_out[NXS];
#pragma unroll
    for (int k = 0; k < NXS; ++k) {
        const int u = tid + k * NT2;
        const int row = u / NQ, p = u - row * NQ;   // row over 3 BY rows
        x_in[k] = u < C::NXU ? row * BX + 4 * p : -1;
        x_out[k] = row * TX + 4 * p;
    }
    if (tid == 0) {
        for (int b = 0; b < E2_NB; ++b) mbar_init(&mbar[b], 1);
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
        asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;\n" ::"l"(
                         P.tm_graw)
                     : "memory");
    }
    __syncthreads();
    unsigned phase = 0;          // bit b: parity of buffer b's next phase
    bool failed = false;
    if (P.fault_wait) {
        // injected: no copy is issued for buffer 0 yet, so its phase 0
        // never completes and the bounded wait runs out (nothing in flight)
        failed = __syncthreads_or(!mbar_wait(&mbar[0], 0)) != 0;
    }
    float m2 = 0.f;
    const bool pair_store = (g.nx & 1) == 0;   // 8-byte aligned pairs

    const int e2_cx = P.e2_cx;
    const long long total = (long long)P.e2_cx * P.e2_cy * g.nz;
    const Share sh_ = share_of(blockIdx.x - P.e2_cta0, P.e2_ncta, total);
    long long w0 = sh_.lo;
    while (w0 < sh_.hi && !failed) {
        const long long col = w0 / g.nz;
        const int z0 = (int)(w0 - col * g.nz);
        const long long zl = z0 + (sh_.hi - w0);
        const int z1 = zl < g.nz ? (int)zl : g.nz;
        w0 += z1 - z0;
        const int x0 = (int)(col % e2_cx) * TX;
        const int y0 = (int)(col / e2_cx) * TY;
        const int ox = x0 + 2 * px, oyy = y0 + oy;
        const bool in0 = oyy < g.ny && ox < g.nx;
        const bool in1 = oyy < g.ny && ox + 1 < g.nx;
        const int o_off = oyy * g.nx + ox;
        const int s_begin = z0 - R, s_end = z1 + R;
        // slices outside the volume and the halo outside it read as zero
        if (tid == 0) {
            for (int b = 0; b < E2_NB && s_begin + b < s_end; ++b) {
                mbar_expect_tx(&mbar[b], C::TXB);
                tma_load_4d(Gr + b * GRF, P.tm_graw, x0 - RA, y0 - R, s_begin + b,
                            0, &mbar[b]);
            }
        }
        float2 ring[KG][3];
#pragma unroll
        for (int k = 0; k < KG; ++k)
#pragma unroll
            for (int q = 0; q < 3; ++q) ring[k][q] = make_float2(0.f, 0.f);
        for (int base = s_begin; base < s_end && !failed; base += KG) {
#pragma unroll
            for (int j = 0; j < KG; ++j) {
                const int s = base + j;
                if (s >= s_end) break;
                const int t = s - s_begin;
                const int b = t % E2_NB;
                const float* gr = Gr + b * GRF;
                // (1) this slice's g_raw tile (TMA, issued E2_NB slices ago);
                //     the barrier also frees the x-smoothed plane
                const bool ok = mbar_wait(&mbar[b], (phase >> b) & 1u);
                phase ^= 1u << b;
                if (__syncthreads_or(!ok)) {
                    // give the copies still in flight a bounded wait
                    for (int d = 1; d < E2_NB && s + d < s_end; ++d) {
                        const int bb = (b + d) % E2_NB;
                        mbar_wait(&mbar[bb], (phase >> bb) & 1u);
                    }
                    failed = true;
                    break;
                }
                // (2) Gaussian along x: four outputs per unit
#pragma unroll
                for (int k = 0; k < NXS; ++k) {
                    if (x_in[k] < 0) continue;
                    // the unit's 4 + 2R inputs start DOFF floats into a
                    // 16-byte-aligned run of NV4 float4 (inside the row:
                    // 4 (NQ - 1) + 4 NV4 <= BX for every R)
                    constexpr int DOFF = RA - R;
                    constexpr int NV4 = (DOFF + 4 + 2 * R + 3) / 4;
                    static_assert(4 * (NQ - 1) + 4 * NV4 <= BX, "x-pass read in row");
                    const float4* rr4 = (const float4*)(gr + x_in[k]);
                    float w4[4 * NV4];
#pragma unroll
                    for (int q4 = 0; q4 < NV4; ++q4) {
                        const float4 t4 = rr4[q4];
                        w4[4 * q4] = t4.x;
                        w4[4 * q4 + 1] = t4.y;
                        w4[4 * q4 + 2] = t4.z;
                        w4[4 * q4 + 3] = t4.w;
                    }
                    float out[4];
#pragma unroll
                    for (int e = 0; e < 4; ++e) {
                        float a = tt[R] * w4[DOFF + e + R];
#pragma unroll
                        for (int m = 1; m <= R; ++m)
                            a += tt[R + m] * (w4[DOFF + e + R - m] + w4[DOFF + e + R + m]);
                        out[e] = a;
                    }
                    *(float4*)(Gx + x_out[k]) = make_float4(out[0], out[1], out[2], out[3]);
                }
                __syncthreads();
                // the tile is consumed: refill this buffer E2_NB slices ahead
                if (tid == 0 && s + E2_NB < s_end) {
                    mbar_expect_tx(&mbar[b], C::TXB);
                    tma_load_4d(Gr + b * GRF, P.tm_graw, x0 - RA, y0 - R, s + E2_NB,
                                0, &mbar[b]);
                }
                // (3) along y for this thread's pair, all components, into
                //     the ring; along z at slice o = s - R
#pragma unroll
                for (int q = 0; q < 3; ++q) {
                    const float* c2 = Gx + (q * BY + oy) * TX + 2 * px;
                    const float2 mid = *(const float2*)(c2 + R * TX);
                    float2 a = make_float2(tt[R] * mid.x, tt[R] * mid.y);
#pragma unroll
                    for (int m = 1; m <= R; ++m) {
                        const float2 lo = *(const float2*)(c2 + (R - m) * TX);
                        const float2 hi = *(const float2*)(c2 + (R + m) * TX);
                        a.x = fmaf(tt[R + m], lo.x + hi.x, a.x);
                        a.y = fmaf(tt[R + m], lo.y + hi.y, a.y);
                    }
                    ring[j][q] = a;
                }
                if (t >= 2 * R) {
                    // slice o + d sits in slot (j + 1 + R + d) mod KG
                    float2 zv[3];
#pragma unroll
                    for (int q = 0; q < 3; ++q) {
                        const float2 mid = ring[(j + 1 + R) % KG][q];
                        float2 a = make_float2(tt[R] * mid.x, tt[R] * mid.y);
#pragma unroll
                        for (int m = 1; m <= R; ++m) {
                            const float2 lo = ring[(j + 1 + R - m) % KG][q];
                            const float2 hi = ring[(j + 1 + R + m) % KG][q];
                            a.x = fmaf(tt[R + m], lo.x + hi.x, a.x);
                            a.y = fmaf(tt[R + m], lo.y + hi.y, a.y);
                        }
                        zv[q] = a;
                    }
                    float* dst = gout + (s - R) * sxy + o_off;
                    if (in1 && pair_store) {
#pragma unroll
                        for (int q = 0; q < 3; ++q)
                            *(float2*)(dst + (long long)q * g.V) = zv[q];
                    } else {
#pragma unroll
                        for (int q = 0; q < 3; ++q) {
                            if (in0) dst[(long long)q * g.V] = zv[q].x;
                            if (in1) dst[(long long)q * g.V + 1] = zv[q].y;
                        }
                    }
                    const float n0 = zv[0].x * zv[0].x + zv[1].x * zv[1].x +
                                     zv[2].x * zv[2].x;
                    const float n1 = zv[0].y * zv[0].y + zv[1].y * zv[1].y +
                                     zv[2].y * zv[2].y;
                    if (in0) m2 = (n0 != n0) ? INFINITY : fmaxf(m2, n0);
                    if (in1) m2 = (n1 != n1) ? INFINITY : fmaxf(m2, n1);
                }
            }
        }
        __syncthreads();   // Gx is rewritten by the next segment
    }
    for (int k = 16; k > 0; k >>= 1)
        m2 = fmaxf(m2, __shfl_down_sync(0xffffffffu, m2, k));
    if ((tid & 31) == 0) red[tid >> 5] = m2;
    __syncthreads();
    if (tid == 0) {
        float v = 0.f;
        for (int w = 0; w < NT2 / 32; ++w) v = fmaxf(v, red[w]);
        // a wait that ran out leaves the marker -1 (|g|^2 is never negative)
        g2_part[blockIdx.x] = failed ? -1.f : v;
    }
}

// ----------------------------------------------------------------------
// Quantisation scale per pair: shift s = (lo + hi) / 2 and Q = 2^qb / h with
// h = (hi - lo) / 2, lo = min(0, F, M), hi = max(0, F, M) (0 is the padding
// value and J is a convex combination of M values and 0).
// ----------------------------------------------------------------------
template <typename T>
__global__ void k_minmax(const PairDesc* __restrict__ pd,
                         float2* __restrict__ part) {
    __shared__ float smin[NT / 32], smax[NT / 32];
    const PairDesc& P = pd[blockIdx.y];
    const T* __restrict__ F = (const T*)P.F;
    const T* __restrict__ M = (const T*)P.M;
    const long long V = P.g.V;
    float lo = 0.f, hi = 0.f;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < V;
         i += (long long)gridDim.x * blockDim.x) {
        float a = ld_img(F, i), b = ld_img(M, i);
        lo = fminf(lo, fminf(a, b));
        hi = fmaxf(hi, fmaxf(a, b));
    }
    for (int o = 16; o > 0; o >>= 1) {
        lo = fminf(lo, __shfl_down_sync(0xffffffffu, lo, o));
        hi = fmaxf(hi, __shfl_down_sync(0xffffffffu, hi, o));
    }
    if ((threadIdx.x & 31) == 0) {
        smin[threadIdx.x >> 5] = lo;
        smax[threadIdx.x >> 5] = hi;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < (int)(blockDim.x / 32); ++w) {
            lo = fminf(lo, smin[w]);
            hi = fmaxf(hi, smax[w]);
        }
        part[blockIdx.y * gridDim.x + blockIdx.x] = make_float2(lo, hi);
    }
}

__global__ void k_qscale(const PairDesc* __restrict__ pd,
                         const float2* __restrict__ part, int n, int qb) {
    if (threadIdx.x != 0) return;
    const int p = blockIdx.x;
    float lo = 0.f, hi = 0.f;
    for (int i = 0; i < n; ++i) {
        lo = fminf(lo, part[p * n + i].x);
        hi = fmaxf(hi, part[p * n + i].y);
    }
    double h = 0.5 * ((double)hi - (double)lo);
    if (!(h > 1e-30)) h = 1.0;       // constant images: any scale is exact
    double sft = 0.5 * ((double)hi + (double)lo);
    double lim = ldexp(1.0, qb);
    QScale* qs = pd[p].qs;
    qs->shift = (float)sft;
    // a little headroom so that rounding never leaves [-lim, lim]
    float Q = (float)(lim / (h * (1.0 + 1e-6)));
    qs->Q = Q;
    qs->invQ = (float)(1.0 / (double)Q);
    qs->qlim = (int)lim;
    qs->lo = lo;
    qs->hi = hi;
}

// ----------------------------------------------------------------------
// Fixed-image moments.  F does not change during a registration, so its
// share of the window moments is computed once per preparation: F' = F - s
// in the fixed point (FQ_BAD marks a non-finite F), and at every voxel the
// exact k^3 window sum S_F of those values and the variance
// B = (k^3 S_FF - S_F^2) / (k^6 Q^2), converted to FP32 exactly as the
// moment stage converts A and C.  Zero padding: points outside the volume
// hold the fixed point of 0.  Three separable passes (x, y, z) through
// int32 / int64 temporaries laid out in a 12-byte-per-voxel scratch.
// ----------------------------------------------------------------------
struct MomTmp {
    long long* ss;   // V sums of squares
    int* s;          // V sums
};
__device__ __forceinline__ MomTmp mom_tmp(float* base, long long V) {
    MomTmp t;
    t.ss = (long long*)base;
    t.s = (int*)((char*)base + 8 * V);
    return t;
}

// Fills the halo-padded jq and fq of each pair with the fixed point of 0
// (the interior is written later: fq by k_fmom_x, jq by every resampling)
// and clears the pair's non-finite flags.  Grid (blocks per pair, pairs).
__global__ void k_qfill(const PairDesc* __restrict__ pd) {
    const PairDesc& P = pd[blockIdx.y];
    if (blockIdx.x == 0 && threadIdx.x == 0) *P.flags = 0u;
    if (!P.qw) return;
    const int qpad = __float2int_rn(-P.qs->shift * P.qs->Q);
    const long long n = (long long)P.qw * P.qh * (P.g.nz + 2 * P.qz);
    const int4 v = make_int4(qpad, qpad, qpad, qpad);
    int4* jq4 = (int4*)P.jq;
    int4* fq4 = (int4*)P.fq;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
         i < n / 4; i += (long long)gridDim.x * blockDim.x) {
        jq4[i] = v;
        fq4[i] = v;
    }
}

template <typename T>
__global__ void __launch_bounds__(256)
    k_fmom_x(const PairDesc* __restrict__ pd, int npairs, int W) {
    const PairDesc& P = pd[pair_of_block<4>(pd, npairs, blockIdx.x)];
    const Geom g = P.g;
    const int i = (blockIdx.x - P.ln_blk0) * 256 + threadIdx.x;
    if (i >= g.V) return;
    const int x = i % g.nx;
    const T* __restrict__ F = (const T*)P.F;
    const float sh = P.qs->shift, Q = P.qs->Q;
    const int qlim = P.qs->qlim;
    const int qpad = __float2int_rn(-sh * Q);
    int s = 0;
    long long ss = 0;
    for (int d = -W; d <= W; ++d) {
        int q = qpad;
        if (x + d >= 0 && x + d < g.nx) {
            const float f = ld_img(F, i + d);
            const bool fin = fabsf(f) <= 3.0e38f;
            if (fin) q = min(max(__float2int_rn((f - sh) * Q), -qlim), qlim);
            if (d == 0) {
                const int r = i / g.nx;
                P.fq[qidx(P, x, r % g.ny, r / g.ny)] = fin ? q : FQ_BAD;
                if (!fin) atomicOr(P.flags, QFLAG_FBAD);
            }
        }
        s += q;
        ss += (long long)q * q;
    }
    MomTmp t = mom_tmp(P.graw, g.V);
    t.s[i] = s;
    t.ss[i] = ss;
}

template <int AXIS>
__global__ void __launch_bounds__(256)
    k_fmom_yz(const PairDesc* __restrict__ pd, int npairs, int W,
              float inv_k3) {
    const PairDesc& P = pd[pair_of_block<4>(pd, npairs, blockIdx.x)];
    const Geom g = P.g;
    const int i = (blockIdx.x - P.ln_blk0) * 256 + threadIdx.x;
    if (i >= g.V) return;
    const int K = 2 * W + 1;
    const int sxy = g.nx * g.ny;
    const int c = AXIS == 1 ? (i / g.nx) % g.ny : i / sxy;
    const int n = AXIS == 1 ? g.ny : g.nz;
    const int stride = AXIS == 1 ? g.nx : sxy;
    const float sh = P.qs->shift, Q = P.qs->Q;
    const long long qpad = __float2int_rn(-sh * Q);
    // a line of the previous passes that lies outside the volume is padding
    const long long pad_n = AXIS == 1 ? K : (long long)K * K;
    const MomTmp a = mom_tmp(AXIS == 1 ? P.graw : P.dj, g.V);
    int s = 0;
    long long ss = 0;
    for (int d = -W; d <= W; ++d) {
        if (c + d >= 0 && c + d < n) {
            s += a.s[i + d * stride];
            ss += a.ss[i + d * stride];
        } else {
            s += (int)(pad_n * qpad);
            ss += pad_n * qpad * qpad;
        }
    }
    if (AXIS == 1) {
        MomTmp t = mom_tmp(P.dj, g.V);
        t.s[i] = s;
        t.ss[i] = ss;
    } else {
        const long long k3 = (long long)K * K * K;
        const float iQ = P.qs->invQ;
        const float mscale = inv_k3 * inv_k3 * iQ * iQ;
        P.fsum[i] = s;
        P.fvar[i] = i64_to_f32(k3 * ss - (long long)s * s) * mscale;
    }
}

template <int R, typename T>
int launch_e2(const Batch& b, int mode, int attempt, cudaStream_t s) {
    k_e2<R, T><<<b.plan.e2_ctas, NT2, E2Cfg<R>::bytes, s>>>(
        b.pd, b.npairs, mode, attempt, b.c.gtaps, b.part.g2max);
    return 1;
}

template <typename T>
int launch_e2_r(const Batch& b, int mode, int attempt, cudaStream_t s) {
    switch (b.c.gtaps.R) {
        case 0: return launch_e2<0, T>(b, mode, attempt, s);
        case 1: return launch_e2<1, T>(b, mode, attempt, s);
        case 2: return launch_e2<2, T>(b, mode, attempt, s);
        case 3: return launch_e2<3, T>(b, mode, attempt, s);
        case 4: return launch_e2<4, T>(b, mode, attempt, s);
        case 5: return launch_e2<5, T>(b, mode, attempt, s);
        default: return launch_e2<6, T>(b, mode, attempt, s);
    }
}

template <int R, typename T>
cudaError_t attr_e2() {
    return cudaFuncSetAttribute(k_e2<R, T>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize,
                                E2Cfg<R>::bytes);
}

template <typename T>
cudaError_t attrs_all() {
    cudaError_t e = cudaSuccess, r;
    if ((r = attr_e2<0, T>()) != cudaSuccess) e = r;
    if ((r = attr_e2<1, T>()) != cudaSuccess) e = r;
    if ((r = attr_e2<2, T>()) != cudaSuccess) e = r;
    if ((r = attr_e2<3, T>()) != cudaSuccess) e = r;
    if ((r = attr_e2<4, T>()) != cudaSuccess) e = r;
    if ((r = attr_e2<5, T>()) != cudaSuccess) e = r;
    if ((r = attr_e2<6, T>()) != cudaSuccess) e = r;
    return e;
}

long long ceil_div(long long a, long long b) { return (a + b - 1) / b; }

}  // namespace

// Quantisation bits per window: the largest qb with k^3 2^qb < 2^31 (int32
// first-moment sums) and k^6 2^(2 qb) < 2^63 (int64 moment differences).
int quant_bits(int win) {
    switch (win) {
        case 3: return 26;
        case 5: return 24;
        case 7: return 22;
        default: return 21;
    }
}

// CTA ranges per pair: by default a single pair takes the whole grid (one
// CTA per SM for E1, two for E2); a batch shares a grid of several waves among its
// pairs in proportion to their work, at least one CTA each, so that every
// CTA works on one pair.
static void split_ctas(const long long* work, int npairs, long long target,
                       int min_work, int* c0, int* n) {
    long long tot = 0;
    for (int p = 0; p < npairs; ++p) tot += work[p];
    int acc = 0;
    for (int p = 0; p < npairs; ++p) {
        long long k = tot > 0 ? (target * work[p] + tot / 2) / tot : 1;
        k = std::max<long long>(
            1, std::min<long long>(k, std::max<long long>(1, work[p] / min_work)));
        c0[p] = acc;
        n[p] = (int)k;
        acc += (int)k;
    }
}

bool e1_tile_ok(int t, int win) {
    // the 32 x 32 variant's shared memory does not fit k = 9
    return t == E1_TILE_32X16 || (t == E1_TILE_32X32 && win <= 7);
}

BatchPlan plan_batch(PairDesc* pd, int npairs, int win, int num_sms,
                     int e1_waves, int e2_waves, int e1_tile, int min_slices,
                     int st_target) {
    BatchPlan bp{};
    if (min_slices < 1) min_slices = 8;
    if (st_target < 1) st_target = 2048;
    bp.min_slices = min_slices;
    bp.st_target = st_target;
    // default: the 32 x 32 tile for k = 5 and 7 (a smaller share of halo
    // rows, and the pipelined schedule at k = 5)
    if (e1_tile < 0 || !e1_tile_ok(e1_tile, win))
        e1_tile = win == 5 || win == 7 ? E1_TILE_32X32 : E1_TILE_32X16;
    bp.e1_tile = e1_tile;
    const int tx1 = E1_OX, ty1 = e1_tile_oy(e1_tile);
    std::vector<long long> w1(npairs), w2(npairs);
    std::vector<int> c0(npairs), n(npairs);
    for (int p = 0; p < npairs; ++p) {
        Geom& g = pd[p].g;
        pd[p].e1_cx = (int)ceil_div(g.nx, tx1);
        pd[p].e1_cy = (int)ceil_div(g.ny, ty1);
        w1[p] = (long long)pd[p].e1_cx * pd[p].e1_cy * g.nz;
        pd[p].e2_cx = (int)ceil_div(g.nx, PLANE_X);
        pd[p].e2_cy = (int)ceil_div(g.ny, PLANE_Y);
        w2[p] = (long long)pd[p].e2_cx * pd[p].e2_cy * g.nz;
    }
    // one wave is one CTA per SM (the 32 x 16 variant runs two at a time)
    if (e1_waves < 1)
        e1_waves = npairs == 1 ? (e1_tile == E1_TILE_32X16 ? 2 : 1) : 4;
    if (e2_waves < 1) e2_waves = npairs == 1 ? 2 : 8;
    const long long t1 = (long long)e1_waves * num_sms;
    const long long t2 = (long long)e2_waves * num_sms;
    split_ctas(w1.data(), npairs, t1, min_slices, c0.data(), n.data());
    for (int p = 0; p < npairs; ++p) {
        pd[p].e1_cta0 = c0[p];
        pd[p].e1_ncta = n[p];
    }
    bp.e1_ctas = c0[npairs - 1] + n[npairs - 1];
    split_ctas(w2.data(), npairs, t2, min_slices, c0.data(), n.data());
    for (int p = 0; p < npairs; ++p) {
        pd[p].e2_cta0 = c0[p];
        pd[p].e2_ncta = n[p];
    }
    bp.e2_ctas = c0[npairs - 1] + n[npairs - 1];
    // step kernel: 32 x 8 tiles, z chunks with ~st_target blocks per pair
    int blk = 0, lnb = 0;
    for (int p = 0; p < npairs; ++p) {
        Geom& g = pd[p].g;
        pd[p].st_tx = (int)ceil_div(g.nx, 32);
        pd[p].st_ty = (int)ceil_div(g.ny, 8);
        long long cols = (long long)pd[p].st_tx * pd[p].st_ty;
        long long nzc = std::max<long long>(
            1, std::min<long long>(g.nz, ceil_div(st_target, cols)));
        pd[p].st_zc = (int)ceil_div(g.nz, nzc);
        pd[p].st_nzc = (int)ceil_div(g.nz, pd[p].st_zc);
        pd[p].st_blk0 = blk;
        blk += pd[p].st_tx * pd[p].st_ty * pd[p].st_nzc;
        pd[p].ln_blk0 = lnb;
        pd[p].ln_nblk = (int)ceil_div(g.V, 256);
        lnb += pd[p].ln_nblk;
    }
    bp.st_blocks = blk;
    bp.ln_blocks = lnb;
    bp.mm_ctas = std::max(2, num_sms / npairs);
    return bp;
}

int plan_tiles(PairDesc* pd, int npairs, int k) {
    // TILE_WARPS / tile_group(k) tile rows and slices per block, blocks
    // never shared between pairs
    const int rows_per_block = TILE_WARPS / tile_group(k);
    int blk = 0;
    for (int p = 0; p < npairs; ++p) {
        const Geom& g = pd[p].g;
        pd[p].th_nx = (int)ceil_div(g.nx, k);
        pd[p].th_ny = (int)ceil_div(g.ny, k);
        pd[p].th_nz = (int)ceil_div(g.nz, k);
        pd[p].th_blk0 = blk;
        blk += (int)ceil_div((long long)pd[p].th_ny * pd[p].th_nz,
                             rows_per_block);
    }
    return blk;
}

long long set_q_layout(PairDesc& d, int win, int loss) {
    if (loss != LM_LOSS_LNCC) {
        d.qw = d.qh = d.qx = d.qz = 0;
        return d.g.V;
    }
    const int W = (win - 1) / 2;
    d.qx = 2 * W;
    d.qz = 2 * W + 1;
    d.qw = (int)ceil_div(d.g.nx, E1_OX) * E1_OX + 4 * W;
    d.qh = (int)ceil_div(d.g.ny, E1_QY) * E1_QY + 4 * W;
    return (long long)d.qw * d.qh * (d.g.nz + 2 * d.qz);
}

int graw_pitch(int nx) { return (nx + 3) / 4 * 4; }

long long graw_floats(const Geom& g) {
    return 3LL * g.nz * g.ny * graw_pitch(g.nx);
}

int encode_graw_map(void* map, const float* graw, const Geom& g, int R) {
    static PFN_cuTensorMapEncodeTiled_v12000 encode = [] {
        void* f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000,
                                             cudaEnableDefault, &q) != cudaSuccess ||
            q != cudaDriverEntryPointSuccess) {
            cudaGetLastError();
            f = nullptr;
        }
        return (PFN_cuTensorMapEncodeTiled_v12000)f;
    }();
    if (!encode) {
        set_last_error("cuTensorMapEncodeTiled is not available from the driver");
        return LM_EUNSUPPORTED;
    }
    const int RA = (R + 3) / 4 * 4;
    const cuuint64_t pw = (cuuint64_t)graw_pitch(g.nx);
    cuuint64_t dims[4] = {(cuuint64_t)g.nx, (cuuint64_t)g.ny, (cuuint64_t)g.nz, 3};
    cuuint64_t strides[3] = {pw * 4, pw * g.ny * 4, pw * g.ny * g.nz * 4};
    cuuint32_t box[4] = {(cuuint32_t)(PLANE_X + 2 * RA), (cuuint32_t)(PLANE_Y + 2 * R),
                         1, 3};
    cuuint32_t estr[4] = {1, 1, 1, 1};
    CUresult r = encode((CUtensorMap*)map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4,
                        (void*)graw, dims, strides, box, estr,
                        CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                        CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) {
        set_last_error("cuTensorMapEncodeTiled rejected the g_raw tensor map");
        return LM_ECUDA;
    }
    return LM_OK;
}

cudaError_t fused_setup() {
    cudaError_t e = attrs_all<float>();
    cudaError_t e2 = attrs_all<__nv_bfloat16>();
    cudaError_t e3 = mi_setup();
    cudaError_t e4 = lncc_setup();
    return e != cudaSuccess ? e : e2 != cudaSuccess ? e2
                                 : e3 != cudaSuccess ? e3 : e4;
}

int batch_prepare(const Batch& b, cudaStream_t s) {
    dim3 grid(b.plan.mm_ctas, b.npairs);
    const int W = (b.c.win - 1) / 2;
    if (b.dtype == LM_BF16)
        k_minmax<__nv_bfloat16><<<grid, NT, 0, s>>>(b.pd, b.mm_part);
    else
        k_minmax<float><<<grid, NT, 0, s>>>(b.pd, b.mm_part);
    k_qscale<<<b.npairs, 32, 0, s>>>(b.pd, b.mm_part, b.plan.mm_ctas,
                                     quant_bits(b.c.win));
    k_qfill<<<grid, 256, 0, s>>>(b.pd);
    if (b.dtype == LM_BF16)
        k_fmom_x<__nv_bfloat16><<<b.plan.ln_blocks, 256, 0, s>>>(b.pd, b.npairs, W);
    else
        k_fmom_x<float><<<b.plan.ln_blocks, 256, 0, s>>>(b.pd, b.npairs, W);
    k_fmom_yz<1><<<b.plan.ln_blocks, 256, 0, s>>>(b.pd, b.npairs, W, b.c.inv_k3);
    k_fmom_yz<2><<<b.plan.ln_blocks, 256, 0, s>>>(b.pd, b.npairs, W, b.c.inv_k3);
    return 6;
}

// The loss kernel of pass 1: E1 for LNCC, the pointwise kernel otherwise.
static int launch_loss(const Batch& b, int mode, int attempt, cudaStream_t s) {
    if (b.method == LM_METHOD_DEMONS) {
        k_pointwise<true><<<b.plan.e1_ctas, NTP, 0, s>>>(
            b.pd, b.npairs, mode, attempt, b.alpha, b.part.loss);
        return 1;
    }
    if (b.loss == LM_LOSS_MSE) {
        k_pointwise<false><<<b.plan.e1_ctas, NTP, 0, s>>>(
            b.pd, b.npairs, mode, attempt, b.alpha, b.part.loss);
        return 1;
    }
    if (b.loss == LM_LOSS_MI) return launch_mi(b, mode, attempt, s);
    return launch_lncc(b, mode, attempt, s);
}

int batch_eval(const Batch& b, int mode, int attempt, cudaStream_t s,
               bool jpass) {
    int n = 0;
    if (b.dtype == LM_BF16) {
        if (jpass) {
            k_jpass<__nv_bfloat16><<<b.plan.st_blocks, dim3(32, 8), 0, s>>>(
                b.pd, b.npairs, mode, attempt);
            n += 1;
        }
        n += launch_loss(b, mode, attempt, s);
        n += launch_e2_r<__nv_bfloat16>(b, mode, attempt, s);
    } else {
        if (jpass) {
            k_jpass<float><<<b.plan.st_blocks, dim3(32, 8), 0, s>>>(
                b.pd, b.npairs, mode, attempt);
            n += 1;
        }
        n += launch_loss(b, mode, attempt, s);
        n += launch_e2_r<float>(b, mode, attempt, s);
    }
    return n;
}

}  // namespace lmk
