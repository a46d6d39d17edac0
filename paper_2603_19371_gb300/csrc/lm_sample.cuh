// Trilinear sampling of an image at displaced points (Section 2.1): the
// cell split is taken on the displacement (c = p + floor(d), f = d -
// floor(d)), the image reads as zero outside the volume.  Shared by the J
// pass and the fused step kernel.
#pragma once

#include "lm_kernels.cuh"

namespace lmk {

__device__ __forceinline__ float safe_floor(float v) {
    return fminf(fmaxf(floorf(v), -1048576.f), 1048576.f);
}

// Trilinear corners of M around p + d (d = u(p) already loaded), zero
// outside the volume.  Offsets are 32-bit.
template <typename T>
__device__ __forceinline__ void corners(const T* __restrict__ M, const Geom& g,
                                        int x, int y, int z, float d0,
                                        float d1, float d2, float m[8],
                                        float f[3]) {
    float l0 = safe_floor(d0), l1 = safe_floor(d1), l2 = safe_floor(d2);
    f[0] = d0 - l0;
    f[1] = d1 - l1;
    f[2] = d2 - l2;
    int cx = x + (int)l0, cy = y + (int)l1, cz = z + (int)l2;
    const int sxy = g.nx * g.ny;
    if (cx >= 0 && cx + 1 < g.nx && cy >= 0 && cy + 1 < g.ny && cz >= 0 &&
        cz + 1 < g.nz) {
        int b = cz * sxy + cy * g.nx + cx;
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
            m[s] = in ? ld_img(M, qz * sxy + qy * g.nx + qx) : 0.f;
        }
    }
}

// J from the corners (corner index = x + 2y + 4z).
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

// Fixed-point value of a non-finite J (never a valid code).
constexpr int JQ_BAD = (int)0x80000000;

// Where the resampling writes go, loaded once per kernel from the pair's
// table (a store through jq could alias the table, so reading the fields
// at every store would reload them).
struct JOut {
    int* jq;
    float* dj;
    unsigned* flags;
    int V;                    // dj component stride
    int qw, qh, qx, qz;       // jq layout (qw = 0: plain)
    int nx, ny;
    float sh, Q;
    int qlim;
};
__device__ __forceinline__ JOut jout_of(const PairDesc& P) {
    JOut o;
    o.jq = P.jq;
    o.dj = P.dj;
    o.flags = P.flags;
    o.V = (int)P.g.V;
    o.qw = P.qw;
    o.qh = P.qh;
    o.qx = P.qx;
    o.qz = P.qz;
    o.nx = P.g.nx;
    o.ny = P.g.ny;
    o.sh = P.qs->shift;
    o.Q = P.qs->Q;
    o.qlim = P.qs->qlim;
    return o;
}

// J and dJ/du of voxel (x, y, z) (linear index i) from its corners: J in
// the moments' fixed point at the pair's jq layout (JQ_BAD, and the pair's
// QFLAG_JBAD, if not finite) and dJ/du to dj (3 x V).
__device__ __forceinline__ void store_resampled(const JOut& o, int i, int x,
                                                int y, int z, const float m[8],
                                                const float f[3]) {
    float d[3];
    const float J = interp(m, f);
    interp_grad(m, f, d);
    const bool fin = fabsf(J) <= 3.0e38f;
    if (!fin) atomicOr(o.flags, QFLAG_JBAD);
    const int qi = o.qw ? ((z + o.qz) * o.qh + y + o.qx) * o.qw + x + o.qx
                        : i;
    o.jq[qi] = fin ? min(max(__float2int_rn((J - o.sh) * o.Q), -o.qlim), o.qlim)
                   : JQ_BAD;
    o.dj[i] = d[0];
    o.dj[o.V + i] = d[1];
    o.dj[2 * o.V + i] = d[2];
}

// J and dJ/du of voxel (x, y, z) under displacement (d0, d1, d2).
template <typename T>
__device__ __forceinline__ void resample_voxel(const JOut& o, const Geom& g,
                                               const T* M, int x, int y, int z,
                                               int i, float d0, float d1,
                                               float d2) {
    float m[8], f[3];
    corners(M, g, x, y, z, d0, d1, d2, m, f);
    store_resampled(o, i, x, y, z, m, f);
}

}  // namespace lmk
