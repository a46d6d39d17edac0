// LNCC loss and backward pass of pass 1 (Section 2.2), as one z-streaming
// kernel per pair.  A CTA owns a column of 32 x OY output voxels (OY = 16
// or 32, the tile variant) and a range of z slices and walks it one moment
// slice at a time.  For moment slice m (window k = 2W + 1, zero padding,
// fixed divisor k^3):
//
//  Z  running sums along z over the slices m - W .. m + W of J', J'J' and
//     F'J' at every point of the (32 + 4W) x (OY + 4W) gather plane, kept in shared
//     memory; each step adds slice m + W and subtracts slice m - W - 1,
//     whose values are read again (they are in L2) rather than kept.  J'
//     and F' come from a halo-padded layout whose halo holds the fixed
//     point of 0, so every gather row is read as aligned 16-byte vectors
//     with no bounds tests;
//  X  sums along x of those, over the (32 + 2W) moment columns;
//  Y  sums along y, which completes the exact window sums S_J, S_JJ, S_FJ
//     at every point of the (32 + 2W) x (OY + 2W) moment plane, and per point the
//     squared local correlation cc = (A^2 + eps_nr) / (B C + eps_dr), its
//     loss term (1 - cc) and the backward coefficients (a, b, c) with
//     A = S_FJ - S_F S_J / k^3, C = S_JJ - S_J^2 / k^3 (B, S_F precomputed
//     per preparation, the fixed image does not change);
//  B  box of (a, b, c) along x, then along y into a ring of the last k
//     slices (shared memory, private to each thread), and along z at
//     output slice m - W:
//        dL/dJ(y) = -V^-1 [F'(y) Box(a) + 2 J'(y) Box(b) + Box(c)],
//        g_raw = dL/dJ dJ/du.
//
// The stages of a slice are separated by four barriers or, where the x-sum
// and x-box planes fit twice in shared memory, software-pipelined over three
// slices with two barriers per slice.
//
// Window moments are exact: F' = F - s and J' = J - s are held in fixed
// point (Xq = round(X' Q), |Xq| <= 2^qb), the sums of Xq are int32 and those
// of the products int64, so A, B, C come out of exact integer differences
// k^3 S_XY - S_X S_Y; only their conversion to FP32 rounds.  Each voxel's
// loss term is rounded to the fixed point 2^-30 and summed in int64, so the
// loss does not depend on the launch plan.  A non-finite J or F reaches
// the decision kernel through the pair's flags (set by the writers), not
// through the values, so this kernel tests none.
//
// HBM traffic per voxel: J', F' (8 B, plus the gather plane's halo where a
// neighbouring column's CTA has not brought it into L2), S_F and B (8 B),
// dJ/du (12 B) in; g_raw (12 B) out.
#include "lm_kernels.cuh"
#include "lm_sample.cuh"

namespace lmk {
namespace {

template <int W, int TILE>
struct E1Z {
    static constexpr int NT = e1_tile_threads(TILE);
    static constexpr int K = 2 * W + 1;
    static constexpr int OX = E1_OX, OY = e1_tile_oy(TILE);   // output tile
    static constexpr int MX = OX + 2 * W, MY = OY + 2 * W;   // moment plane
    static constexpr int GX = OX + 4 * W, GY = OY + 4 * W;   // gather plane
    static constexpr int MXP = (MX + 3) / 4 * 4;       // padded row stride
    static constexpr int GU = GX / 4;                  // 4-point units / row
    static constexpr int NZU = GY * GU;
    static constexpr int NZS = (NZU + NT - 1) / NT;    // z-sum slots / thread
    static constexpr int XW = MX % 4 == 0 ? 4 : 2;     // x-pass outputs / unit
    static constexpr int NXU = GY * (MX / XW);
    static constexpr int NXS = (NXU + NT - 1) / NT;
    // y outputs per unit: the divisor of MY = OY + 2W among 4, 3, 2 that
    // gives the busiest thread the fewest moment points (ties: the larger,
    // whose sliding sums share more loads)
    static constexpr int ypts(int yw) {
        return MY % yw ? 1 << 30 : (MX * (MY / yw) + NT - 1) / NT * yw;
    }
    static constexpr int YW = ypts(4) <= ypts(3) && ypts(4) <= ypts(2)
                                  ? 4
                                  : (ypts(3) <= ypts(2) ? 3 : 2);
    static constexpr int NYU = MX * (MY / YW);
    static constexpr int NYS = (NYU + NT - 1) / NT;
    static constexpr int NBU = 3 * MY * (OX / 4);      // coefficient x box
    static constexpr int NBS = (NBU + NT - 1) / NT;
    static_assert(GX % 4 == 0, "gather rows are whole 16-byte vectors");
    static_assert(MY % YW == 0, "y units tile the moment plane");
    static_assert(OX * OY == 2 * NT, "two outputs per thread");
    // Row strides of the z- and x-sum planes chosen so that eight
    // consecutive rows start in eight distinct 4-bank groups (the x pass
    // maps consecutive lanes to consecutive rows): int32 rows of 4 (odd)
    // words mod 32, int64 rows of 2 x 2 (odd) words mod 32.
    static constexpr int s4(int n) {
        int s = (n + 3) / 4 * 4;
        while ((s % 32) / 4 % 2 == 0) s += 4;
        return s;
    }
    static constexpr int s8(int n) {
        int s = (n + 1) / 2 * 2;
        while ((2 * s % 32) / 4 % 2 == 0) s += 2;
        return s;
    }
    static constexpr int SZJ = s4(GX), SZL = s8(GX);   // z-sum planes
    static constexpr int SXJ = s4(MX), SXL = s8(MX);   // x-sum planes
    static constexpr int NG = MY / YW;                 // y row groups
    static constexpr int r16(int b) { return (b + 15) / 16 * 16; }
    static constexpr int B_ZJ = r16(GY * SZJ * 4);
    static constexpr int B_ZL = r16(GY * SZL * 8);
    static constexpr int B_XJ = r16(GY * SXJ * 4);
    static constexpr int B_XL = r16(GY * SXL * 8);
    static constexpr int B_C = r16(MY * MXP * 4);
    static constexpr int B_B = r16(MY * OX * 4);
    // Pipelined schedule (two barriers per slice, the x-sum and x-box
    // planes double-buffered) where its shared memory still lets the
    // variant keep its CTAs per SM
    static constexpr int bytes_for(int nb) {
        return B_ZJ + 2 * B_ZL + nb * (B_XJ + 2 * B_XL) + 3 * B_C +
               nb * 3 * B_B + K * 3 * NT * 8;
    }
    // (the 32 x 16 tile runs two CTAs per SM: past 96 KB each, the L1 left
    // beside them throttles the gathers more than the barriers cost)
    static constexpr bool PIPE = bytes_for(2) <= (TILE == 0 ? 96 : 226) * 1024;
    static constexpr int NXB = PIPE ? 2 : 1;
    static constexpr int O_ZJ = 0;
    static constexpr int O_ZJJ = O_ZJ + B_ZJ;
    static constexpr int O_ZFJ = O_ZJJ + B_ZL;
    static constexpr int O_XJ = O_ZFJ + B_ZL;            // [NXB] x-sum planes
    static constexpr int O_XJJ = O_XJ + NXB * B_XJ;
    static constexpr int O_XFJ = O_XJJ + NXB * B_XL;
    static constexpr int O_C = O_XFJ + NXB * B_XL;       // a, b, c planes
    static constexpr int O_B = O_C + 3 * B_C;            // [NXB] their x boxes
    static constexpr int O_R = O_B + NXB * 3 * B_B;      // coefficient ring
    static constexpr int bytes = O_R + K * 3 * NT * 8;
    static_assert(bytes == bytes_for(NXB), "layout");
};

// The int64 z-sum rows are held as 16-byte pairs of columns with the even
// pairs in the first half of the row and the odd ones in the second (GU
// pairs each), so that lanes reading pair 2p + o of consecutive units p
// touch consecutive 16-byte words (no bank conflicts).
template <int GU>
__device__ __forceinline__ int zpair(int pr) {
    return (pr & 1) ? GU + (pr >> 1) : (pr >> 1);
}

// XW window sums along x of one row, out[e] = sum_{o < K} in[e + o]; in
// starts 16-byte aligned when XW == 4, 8-byte aligned when XW == 2.
template <int K, int XW>
__device__ __forceinline__ void xsum_i32(const int* in, int* out) {
    constexpr int NV = XW + K - 1;
    static_assert(NV % 4 == 0, "whole vectors");
    int v[NV];
    if constexpr (XW == 4) {
#pragma unroll
        for (int o = 0; o < NV / 4; ++o) {
            const int4 a = ((const int4*)in)[o];
            v[4 * o] = a.x;
            v[4 * o + 1] = a.y;
            v[4 * o + 2] = a.z;
            v[4 * o + 3] = a.w;
        }
    } else {
#pragma unroll
        for (int o = 0; o < NV / 2; ++o) {
            const int2 a = ((const int2*)in)[o];
            v[2 * o] = a.x;
            v[2 * o + 1] = a.y;
        }
    }
    int sm[XW];
    sm[0] = tree_sum<0, K>(v);
#pragma unroll
    for (int e = 1; e < XW; ++e) sm[e] = sm[e - 1] + (v[e + K - 1] - v[e - 1]);
    if constexpr (XW == 4)
        *(int4*)out = make_int4(sm[0], sm[1], sm[2], sm[3]);
    else
        *(int2*)out = make_int2(sm[0], sm[1]);
}
// As xsum_i32 for an int64 z-sum row (pair-swizzled, see zpair) whose
// window starts at column c0 (even).
template <int K, int XW, int GU>
__device__ __forceinline__ void xsum_i64(const longlong2* row, int c0,
                                         long long* out) {
    constexpr int NV = XW + K - 1;
    long long v[NV];
#pragma unroll
    for (int o = 0; o < NV / 2; ++o) {
        const longlong2 a = row[zpair<GU>((c0 >> 1) + o)];
        v[2 * o] = a.x;
        v[2 * o + 1] = a.y;
    }
    long long sm[XW];
    sm[0] = tree_sum<0, K>(v);
#pragma unroll
    for (int e = 1; e < XW; ++e) sm[e] = sm[e - 1] + (v[e + K - 1] - v[e - 1]);
#pragma unroll
    for (int e = 0; e < XW; e += 2)
        *(longlong2*)(out + e) = make_longlong2(sm[e], sm[e + 1]);
}
// YW window sums along y down one column (row stride S): out[e] =
// sum_{o < K} in[(e + o) S].
template <int K, int YW, int S, typename T>
__device__ __forceinline__ void ysum(const T* in, T* out) {
    T v[YW + K - 1];
#pragma unroll
    for (int o = 0; o < YW + K - 1; ++o) v[o] = in[o * S];
    out[0] = tree_sum<0, K>(v);
#pragma unroll
    for (int e = 1; e < YW; ++e) out[e] = out[e - 1] + (v[e + K - 1] - v[e - 1]);
}

// z-sum update of unit g4 (four gather points) of a row: Z += (new terms)
// - (old terms), the terms being J', J'J' and F'J'.  zj points at the
// unit's four int32, zjj / zfj at the row's int64 pairs.
template <int GU>
__device__ __forceinline__ void zupdate(int* zj, longlong2* zjj,
                                        longlong2* zfj, int g4, int4 jn,
                                        int4 fn, int4 jo, int4 fo) {
    int4 a = *(int4*)zj;
    a.x += jn.x - jo.x;
    a.y += jn.y - jo.y;
    a.z += jn.z - jo.z;
    a.w += jn.w - jo.w;
    *(int4*)zj = a;
    longlong2 p = zjj[g4], q = zjj[GU + g4];
    p.x += (long long)jn.x * jn.x - (long long)jo.x * jo.x;
    p.y += (long long)jn.y * jn.y - (long long)jo.y * jo.y;
    q.x += (long long)jn.z * jn.z - (long long)jo.z * jo.z;
    q.y += (long long)jn.w * jn.w - (long long)jo.w * jo.w;
    zjj[g4] = p;
    zjj[GU + g4] = q;
    p = zfj[g4];
    q = zfj[GU + g4];
    p.x += (long long)fn.x * jn.x - (long long)fo.x * jo.x;
    p.y += (long long)fn.y * jn.y - (long long)fo.y * jo.y;
    q.x += (long long)fn.z * jn.z - (long long)fo.z * jo.z;
    q.y += (long long)fn.w * jn.w - (long long)fo.w * jo.w;
    zfj[g4] = p;
    zfj[GU + g4] = q;
}

// Moment column and first row of y unit u: the first 32 NG units cover
// columns 0..31 of the NG row groups one warp per group, the rest the
// last MX - 32 columns, so that no warp's lanes straddle two row groups.
template <typename C>
__device__ __forceinline__ void ymap(int u, int* mx, int* my0) {
    if (u < 32 * C::NG) {
        *mx = u & 31;
        *my0 = (u >> 5) * C::YW;
    } else {
        constexpr int T = C::MX - 32;
        const int v = u - 32 * C::NG;
        *mx = 32 + v % T;
        *my0 = (v / T) * C::YW;
    }
}

template <int W, int TILE>
__global__ void __launch_bounds__(e1_tile_threads(TILE),
                                  TILE == E1_TILE_32X16 ? 2 : 1)
    k_lncc(const PairDesc* __restrict__ pd, int npairs, int mode, int attempt,
           LnccConsts c, long long* __restrict__ loss_part) {
    using C = E1Z<W, TILE>;
    constexpr int NT = C::NT;
    constexpr int K = C::K, OX = C::OX, OY = C::OY, MX = C::MX, MY = C::MY;
    constexpr int MXP = C::MXP, GU = C::GU;
    constexpr int NZS = C::NZS, XW = C::XW, YW = C::YW;
    extern __shared__ __align__(16) unsigned char smem[];
    int* ZJ = (int*)(smem + C::O_ZJ);                 // [GY][SZJ] z sums
    long long* ZJJ = (long long*)(smem + C::O_ZJJ);
    long long* ZFJ = (long long*)(smem + C::O_ZFJ);
    int* XJ = (int*)(smem + C::O_XJ);                 // [GY][SXJ] x sums
    long long* XJJ = (long long*)(smem + C::O_XJJ);
    long long* XFJ = (long long*)(smem + C::O_XFJ);
    float* CP = (float*)(smem + C::O_C);              // [3][MY][MXP]
    float* BP = (float*)(smem + C::O_B);              // [3][MY][OX]
    float2* RG = (float2*)(smem + C::O_R);            // [K][3][NT]
    constexpr int CPS = C::B_C / 4, BPS = C::B_B / 4;  // plane strides
    __shared__ long long red[NT / 32];

    const PairDesc& P = pd[pair_of_block<1>(pd, npairs, blockIdx.x)];
    if (trial_skip(P, mode, attempt)) return;
    const Geom g = P.g;
    const int* __restrict__ fqv = P.fq;               // halo-padded layout
    const int* __restrict__ jqv = P.jq;
    const int* __restrict__ fsv = P.fsum;
    const float* __restrict__ fbv = P.fvar;
    const float* __restrict__ djv = P.dj;
    float* __restrict__ graw = P.graw;
    const int gpw = P.gp_w;
    const long long gcs = (long long)g.nz * g.ny * gpw;
    const QScale* __restrict__ qs = P.qs;
    const float inv_V = (float)(1.0 / (double)g.V);
    const int tid = threadIdx.x;
    const int sxy = g.nx * g.ny;
    const int qw = P.qw, qplane = P.qh * P.qw;
    const float iQ = qs->invQ;
    const long long k3 = (long long)K * K * K;
    const float mscale = c.inv_k3 * c.inv_k3 * iQ * iQ;
    const float m1scale = c.inv_k3 * iQ;
    // slice z of the padded layout starts at (z + qz) qplane
    const int* __restrict__ jq0 = jqv + (long long)P.qz * qplane;
    const int* __restrict__ fq0 = fqv + (long long)P.qz * qplane;

    // out stage role: column ox, rows oy and oy + 1 of the output tile
    const int ox = tid % OX, oy = 2 * (tid / OX);
    // y units: in the pipelined schedule they run beside the x units, which
    // take the low threads, so they start from the high ones (whole warps
    // keep whole groups of 32 units)
    const int yunit = C::PIPE ? NT - 1 - tid : tid;

    long long lacc = 0;
    bool bad = false;
    const long long total = (long long)P.e1_cx * P.e1_cy * g.nz;
    const Share sh_ = share_of(blockIdx.x - P.e1_cta0, P.e1_ncta, total);
    long long w0 = sh_.lo;
    while (w0 < sh_.hi) {
        const long long col = w0 / g.nz;
        const int z0 = (int)(w0 - col * g.nz);
        const long long zl = z0 + (sh_.hi - w0);
        const int z1 = zl < g.nz ? (int)zl : g.nz;
        w0 += z1 - z0;
        const int x0 = (int)(col % P.e1_cx) * OX;
        const int y0 = (int)(col / P.e1_cx) * OY;

        // z-sum units: four gather points of one row; gather point (gx, gy)
        // is the padded voxel (x0 + gx, y0 + gy), 16-byte aligned for gx % 4
        // == 0 (the halo is 2W wide and the pitch a multiple of 4)
        int zoff[NZS], zsm[NZS], zg4[NZS];
#pragma unroll
        for (int k = 0; k < NZS; ++k) {
            const int u = tid + k * NT;
            const int gy = u / GU, g4 = u - gy * GU;
            zsm[k] = u < C::NZU ? gy : -1;   // the unit's row
            zg4[k] = g4;
            zoff[k] = (y0 + gy) * qw + x0 + 4 * g4;
        }
        auto ld4 = [&](const int* base, int z, int k) -> int4 {
            return __ldg((const int4*)(base + z * qplane + zoff[k]));
        };
        // moment slices m0 .. m1 - 1 feed the outputs z0 .. z1 - 1
        const int m0 = z0 - W, m1 = z1 + W;
        int4 pjn[NZS], pfn[NZS], pjo[NZS], pfo[NZS];
        const int4 zero4 = make_int4(0, 0, 0, 0);
#pragma unroll
        for (int k = 0; k < NZS; ++k) {
            if (zsm[k] < 0) continue;
            // zero exactly the words this thread's unit updates (its two
            // swizzled int64 pairs): no other thread touches them before
            // the first barrier
            const int gy = zsm[k];
            *(int4*)(ZJ + gy * C::SZJ + 4 * zg4[k]) = zero4;
            ((longlong2*)(ZJJ + gy * C::SZL))[zg4[k]] = make_longlong2(0, 0);
            ((longlong2*)(ZJJ + gy * C::SZL))[GU + zg4[k]] = make_longlong2(0, 0);
            ((longlong2*)(ZFJ + gy * C::SZL))[zg4[k]] = make_longlong2(0, 0);
            ((longlong2*)(ZFJ + gy * C::SZL))[GU + zg4[k]] = make_longlong2(0, 0);
        }
        // the window of slice m0 - 1 (J slices m0 - W - 1 .. m0 + W - 1)
        // into the z sums, three slices' loads in flight at a time
        for (int c0 = 0; c0 < K; c0 += 3) {
            int4 wj[3][NZS], wf[3][NZS];
#pragma unroll
            for (int e = 0; e < 3; ++e)
#pragma unroll
                for (int k = 0; k < NZS; ++k) {
                    const bool on = c0 + e < K && zsm[k] >= 0;
                    wj[e][k] = on ? ld4(jq0, m0 - W - 1 + c0 + e, k) : zero4;
                    wf[e][k] = on ? ld4(fq0, m0 - W - 1 + c0 + e, k) : zero4;
                }
#pragma unroll
            for (int e = 0; e < 3; ++e)
#pragma unroll
                for (int k = 0; k < NZS; ++k) {
                    if (c0 + e >= K || zsm[k] < 0) continue;
                    const int gy = zsm[k];
                    zupdate<GU>(ZJ + gy * C::SZJ + 4 * zg4[k],
                                (longlong2*)(ZJJ + gy * C::SZL),
                                (longlong2*)(ZFJ + gy * C::SZL), zg4[k],
                                wj[e][k], wf[e][k], zero4, zero4);
                }
        }
        // slice m0's entering and leaving J slices
#pragma unroll
        for (int k = 0; k < NZS; ++k) {
            if (zsm[k] < 0) continue;
            pjn[k] = ld4(jq0, m0 + W, k);
            pfn[k] = ld4(fq0, m0 + W, k);
            pjo[k] = ld4(jq0, m0 - W - 1, k);
            pfo[k] = ld4(fq0, m0 - W - 1, k);
        }

        // F's share of the moments at this thread's y units, one slice ahead
        int pSF[C::NYS][YW];
        float pB[C::NYS][YW];
        auto ld_mom = [&](int m) {
#pragma unroll
            for (int s = 0; s < C::NYS; ++s) {
                const int u = yunit + s * NT;
                int mx, my0;
                ymap<C>(u, &mx, &my0);
                const int x = x0 - W + mx;
#pragma unroll
                for (int e = 0; e < YW; ++e) {
                    const int y = y0 - W + my0 + e;
                    const bool in = u < C::NYU && x >= 0 && x < g.nx &&
                                    y >= 0 && y < g.ny && m >= 0 && m < g.nz;
                    const int i = m * sxy + y * g.nx + x;
                    pSF[s][e] = in ? __ldg(fsv + i) : 0;
                    pB[s][e] = in ? __ldg(fbv + i) : 0.f;
                }
            }
        };
        ld_mom(m0);
        // the output voxels' F', J' (padded layout) and dJ/du, one slice
        // ahead of their use
        const int opad = (y0 + oy + P.qx) * qw + x0 + ox + P.qx;
        const int olin = (y0 + oy) * g.nx + x0 + ox;
        bool ov[2];
        ov[0] = x0 + ox < g.nx && y0 + oy < g.ny;
        ov[1] = x0 + ox < g.nx && y0 + oy + 1 < g.ny;
        int pFq[2] = {0, 0}, pJq[2] = {0, 0};
        float pdj[2][3] = {{0.f, 0.f, 0.f}, {0.f, 0.f, 0.f}};
        auto ld_out = [&](int zo) {
#pragma unroll
            for (int e = 0; e < 2; ++e) {
                const int ip = zo * qplane + opad + e * qw;
                pFq[e] = __ldg(fq0 + ip);
                pJq[e] = __ldg(jq0 + ip);
                const int i = zo * sxy + olin + e * g.nx;
                pdj[e][0] = ov[e] ? __ldg(djv + i) : 0.f;
                pdj[e][1] = ov[e] ? __ldg(djv + g.V + i) : 0.f;
                pdj[e][2] = ov[e] ? __ldg(djv + 2 * g.V + i) : 0.f;
            }
        };

        int j = 0;   // ring slot of the next out stage's slice
        // ---- Z: slide the z sums to the window of slice m, then request
        //      the next slice's values ----
        auto stage_z = [&](int m) {
#pragma unroll
            for (int k = 0; k < NZS; ++k) {
                if (zsm[k] < 0) continue;
                const int gy = zsm[k];
                zupdate<GU>(ZJ + gy * C::SZJ + 4 * zg4[k],
                            (longlong2*)(ZJJ + gy * C::SZL),
                            (longlong2*)(ZFJ + gy * C::SZL), zg4[k], pjn[k],
                            pfn[k], pjo[k], pfo[k]);
                if (m + 1 < m1) {
                    pjn[k] = ld4(jq0, m + 1 + W, k);
                    pfn[k] = ld4(fq0, m + 1 + W, k);
                    pjo[k] = ld4(jq0, m - W, k);
                    pfo[k] = ld4(fq0, m - W, k);
                }
            }
        };
        // ---- X: sums along x over the moment columns (x-sum buffer xb) ----
        auto stage_x = [&](int xb) {
            int* xj = XJ + xb * (C::B_XJ / 4);
            long long* xjj = XJJ + xb * (C::B_XL / 8);
            long long* xfj = XFJ + xb * (C::B_XL / 8);
#pragma unroll
            for (int s = 0; s < C::NXS; ++s) {
                const int u = tid + s * NT;
                if (u >= C::NXU) break;
                // consecutive lanes take consecutive rows (see the strides)
                const int gy = u % C::GY, c0 = (u / C::GY) * XW;
                xsum_i32<K, XW>(ZJ + gy * C::SZJ + c0, xj + gy * C::SXJ + c0);
                xsum_i64<K, XW, GU>((const longlong2*)(ZJJ + gy * C::SZL), c0,
                                    xjj + gy * C::SXL + c0);
                xsum_i64<K, XW, GU>((const longlong2*)(ZFJ + gy * C::SZL), c0,
                                    xfj + gy * C::SXL + c0);
            }
        };
        // ---- Y: sums along y, cc, loss term, (a, b, c) of slice m ----
        auto stage_y = [&](int m, int xb) {
            const int* xj = XJ + xb * (C::B_XJ / 4);
            const long long* xjj = XJJ + xb * (C::B_XL / 8);
            const long long* xfj = XFJ + xb * (C::B_XL / 8);
#pragma unroll
            for (int s = 0; s < C::NYS; ++s) {
                const int u = yunit + s * NT;
                if (u >= C::NYU) break;
                int mx, my0;
                ymap<C>(u, &mx, &my0);
                int SJv[YW];
                long long SJJv[YW], SFJv[YW];
                ysum<K, YW, C::SXJ>(xj + my0 * C::SXJ + mx, SJv);
                ysum<K, YW, C::SXL>(xjj + my0 * C::SXL + mx, SJJv);
                ysum<K, YW, C::SXL>(xfj + my0 * C::SXL + mx, SFJv);
                const int x = x0 - W + mx;
                const bool xin = x >= 0 && x < g.nx;
                const bool xout = mx >= W && mx < W + OX;
                const bool zin = m >= 0 && m < g.nz;
                const bool zout = m >= z0 && m < z1;
#pragma unroll
                for (int e = 0; e < YW; ++e) {
                    const int SJ = SJv[e];
                    const long long SJJ = SJJv[e], SFJ = SFJv[e];
                    const int my = my0 + e;
                    const int y = y0 - W + my;
                    float av = 0.f, bv = 0.f, cv = 0.f;
                    if (xin && zin && y >= 0 && y < g.ny) {
                        const int sf = pSF[s][e];
                        const long long Ai = k3 * SFJ - (long long)sf * SJ;
                        const long long Ci = k3 * SJJ - (long long)SJ * SJ;
                        const float A = i64_to_f32(Ai) * mscale;
                        const float B = pB[s][e];
                        const float Cm = i64_to_f32(Ci) * mscale;
                        const float mF = (float)sf * m1scale;
                        const float mJ = (float)SJ * m1scale;
                        const float BC = __fmul_rn(B, Cm), AA = __fmul_rn(A, A);
                        const float N = AA + c.eps_nr;
                        const float D = BC + c.eps_dr;
                        // D >= eps_dr > 0: the approximate reciprocal (about
                        // 1 ulp) is safe
                        const float rD = __fdividef(1.f, D);
                        av = 2.f * A * rD;
                        bv = -N * B * rD * rD;
                        cv = -av * mF - 2.f * bv * mJ;
                        if (xout && zout && my >= W && my < W + OY)
                            lacc += loss_fixed(
                                ((BC - AA) + (c.eps_dr - c.eps_nr)) * rD * LOSS_Q,
                                &bad);
                    }
                    const int a = my * MXP + mx;
                    CP[a] = av;
                    CP[CPS + a] = bv;
                    CP[2 * CPS + a] = cv;
                }
            }
            // F's share of the next slice's moments
            if (m + 1 < m1) ld_mom(m + 1);
        };
        // ---- B: box of (a, b, c) along x, four outputs per unit (box
        //      buffer bb) ----
        auto stage_b = [&](int bb) {
            float* bp = BP + bb * 3 * BPS;
#pragma unroll
            for (int s = 0; s < C::NBS; ++s) {
                const int u = tid + s * NT;
                if (u >= C::NBU) break;
                constexpr int NU = OX / 4;
                const int row = u / NU;               // q * MY + my
                const int c0 = (u - row * NU) * 4;
                const int q = row / MY, my = row - q * MY;
                const float* r = CP + q * CPS + my * MXP + c0;
                constexpr int NV4 = (K + 3 + 3) / 4;  // float4 reads
                static_assert(OX - 4 + 4 * NV4 <= MXP, "x box reads in row");
                float v[4 * NV4];
#pragma unroll
                for (int o = 0; o < NV4; ++o) {
                    const float4 a = *(const float4*)(r + 4 * o);
                    v[4 * o] = a.x;
                    v[4 * o + 1] = a.y;
                    v[4 * o + 2] = a.z;
                    v[4 * o + 3] = a.w;
                }
                const float s0 = tree_sum<0, K>(v);
                const float s1 = (s0 - v[0]) + v[K];
                const float s2 = (s1 - v[1]) + v[K + 1];
                const float s3 = (s2 - v[2]) + v[K + 2];
                *(float4*)(bp + q * BPS + my * OX + c0) = make_float4(s0, s1, s2, s3);
            }
        };
        // ---- out: box along y of slice m into the ring, along z, dL/dJ ----
        auto stage_out = [&](int m, int bb) {
            const float* bp = BP + bb * 3 * BPS;
#pragma unroll
            for (int q = 0; q < 3; ++q) {
                float v[K + 1];
#pragma unroll
                for (int o = 0; o <= K; ++o)
                    v[o] = bp[q * BPS + (oy + o) * OX + ox];
                const float t0 = tree_sum<0, K>(v);
                RG[(j * 3 + q) * NT + tid] = make_float2(t0, (t0 - v[0]) + v[K]);
            }
            // output slice zo = m - W once the ring holds the slices
            // zo - W .. zo + W: slice zo - W + d sits in slot
            // (j + 1 + d) mod K
            const int zo = m - W;
            if (zo >= z0) {
                float cF[2], cJ[2], cd[2][3];
#pragma unroll
                for (int e = 0; e < 2; ++e) {
                    cF[e] = (float)pFq[e] * iQ;
                    cJ[e] = (float)pJq[e] * iQ;
                    cd[e][0] = pdj[e][0];
                    cd[e][1] = pdj[e][1];
                    cd[e][2] = pdj[e][2];
                }
                if (zo + 1 < z1) ld_out(zo + 1);
                float b3[3][2];
#pragma unroll
                for (int q = 0; q < 3; ++q) {
                    float v0[K], v1[K];
#pragma unroll
                    for (int d = 0; d < K; ++d) {
                        int sl = j + 1 + d;
                        sl = sl >= K ? sl - K : sl;
                        const float2 t = RG[(sl * 3 + q) * NT + tid];
                        v0[d] = t.x;
                        v1[d] = t.y;
                    }
                    b3[q][0] = tree_sum<0, K>(v0);
                    b3[q][1] = tree_sum<0, K>(v1);
                }
#pragma unroll
                for (int e = 0; e < 2; ++e) {
                    if (!ov[e]) continue;
                    const float dLdJ =
                        -inv_V * ((cF[e] * b3[0][e] + 2.f * cJ[e] * b3[1][e] +
                                   b3[2][e]) *
                                  c.inv_k3);
                    const long long gi =
                        (long long)(zo * g.ny + y0 + oy + e) * gpw + x0 + ox;
                    graw[gi] = dLdJ * cd[e][0];
                    graw[gcs + gi] = dLdJ * cd[e][1];
                    graw[2 * gcs + gi] = dLdJ * cd[e][2];
                }
            } else if (zo + 1 == z0) {
                ld_out(z0);
            }
            j = j + 1 == K ? 0 : j + 1;
        };

        if constexpr (C::PIPE) {
            // Round t: Z(t) | X(t) and Y(t - 1) | B(t - 1) and out(t - 2).
            // The x sums of consecutive slices and the x boxes alternate
            // between two buffers, so every hazard is crossed by one of the
            // two barriers: X(t) reads Z(t) after the first, Z(t + 1)
            // rewrites the z sums after the second; Y(t - 1) reads X(t - 1)
            // and rewrites the (a, b, c) planes after B(t - 2) read them;
            // B(t - 1) reads them after the second; out(t - 2) reads the box
            // B(t - 2) wrote a round earlier.
            for (int t = m0; t < m1 + 2; ++t) {
                if (t < m1) stage_z(t);
                __syncthreads();
                if (t < m1) stage_x(t & 1);
                if (t > m0 && t <= m1) stage_y(t - 1, (t - 1) & 1);
                __syncthreads();
                if (t > m0 && t <= m1) stage_b((t - 1) & 1);
                if (t >= m0 + 2) stage_out(t - 2, t & 1);
            }
        } else {
            for (int m = m0; m < m1; ++m) {
                stage_z(m);
                __syncthreads();
                stage_x(0);
                __syncthreads();
                stage_y(m, 0);
                __syncthreads();
                stage_b(0);
                __syncthreads();
                stage_out(m, 0);
            }
        }
        __syncthreads();   // the planes are rewritten by the next segment
    }
    for (int o = 16; o > 0; o >>= 1) lacc += __shfl_down_sync(0xffffffffu, lacc, o);
    if ((tid & 31) == 0) red[tid >> 5] = lacc;
    const int any_bad = __syncthreads_or(bad);
    if (tid == 0) {
        long long v = 0;
        for (int w = 0; w < NT / 32; ++w) v += red[w];
        loss_part[blockIdx.x] = any_bad ? LOSS_BAD : v;
    }
}

template <int W, int TILE>
int launch_w(const Batch& b, int mode, int attempt, cudaStream_t s) {
    using C = E1Z<W, TILE>;
    k_lncc<W, TILE><<<b.plan.e1_ctas, C::NT, C::bytes, s>>>(
        b.pd, b.npairs, mode, attempt, b.c, b.part.loss);
    return 1;
}

template <int W, int TILE>
cudaError_t attr_w() {
    return cudaFuncSetAttribute(k_lncc<W, TILE>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize,
                                E1Z<W, TILE>::bytes);
}

template <int TILE>
int launch_t(const Batch& b, int mode, int attempt, cudaStream_t s) {
    switch ((b.c.win - 1) / 2) {
        case 1: return launch_w<1, TILE>(b, mode, attempt, s);
        case 2: return launch_w<2, TILE>(b, mode, attempt, s);
        default: return launch_w<3, TILE>(b, mode, attempt, s);
    }
}

}  // namespace

int launch_lncc(const Batch& b, int mode, int attempt, cudaStream_t s) {
    if (b.c.win == 9) return launch_w<4, E1_TILE_32X16>(b, mode, attempt, s);
    if (b.plan.e1_tile == E1_TILE_32X32)
        return launch_t<E1_TILE_32X32>(b, mode, attempt, s);
    return launch_t<E1_TILE_32X16>(b, mode, attempt, s);
}

cudaError_t lncc_setup() {
    cudaError_t e = cudaSuccess, r;
    if ((r = attr_w<1, E1_TILE_32X16>()) != cudaSuccess) e = r;
    if ((r = attr_w<2, E1_TILE_32X16>()) != cudaSuccess) e = r;
    if ((r = attr_w<3, E1_TILE_32X16>()) != cudaSuccess) e = r;
    if ((r = attr_w<4, E1_TILE_32X16>()) != cudaSuccess) e = r;
    if ((r = attr_w<1, E1_TILE_32X32>()) != cudaSuccess) e = r;
    if ((r = attr_w<2, E1_TILE_32X32>()) != cudaSuccess) e = r;
    if ((r = attr_w<3, E1_TILE_32X32>()) != cudaSuccess) e = r;
    return e;
}

}  // namespace lmk
