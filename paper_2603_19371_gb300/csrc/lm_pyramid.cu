// Pyramid kernels: anti-aliased downsampling of the images and resampling
// of the displacement field between levels (Section 2.1, coarse-to-fine).
#include <cmath>

#include "lm_pyramid.cuh"

namespace lmk {
namespace {


template <typename T>
__device__ __forceinline__ void store_img(T* p, long long i, float v);
template <>
__device__ __forceinline__ void store_img(float* p, long long i, float v) {
    p[i] = v;
}
template <>
__device__ __forceinline__ void store_img(__nv_bfloat16* p, long long i,
                                          float v) {
    p[i] = __float2bfloat16_rn(v);
}

// One axis of a level's anti-aliased sampling.  Blurring with the taps t
// (zero outside the volume) and then reading linearly at f p + (f - 1) / 2
// (a corner outside the volume weighs nothing) are both linear and
// separable, so each axis is filtered and sampled in one pass that computes
// only the level's points along it: x first (full y, z), then y, then z.
// The input has extents (ix, iy, iz); the output replaces the axis' extent
// by n_out.  One thread per output point, the other two coordinates from
// the grid (no divisions).
template <typename TI, typename TO>
__global__ void k_level_axis(const TI* __restrict__ in, int ix, int iy, int iz,
                             int axis, int f, int n_out, Taps t,
                             TO* __restrict__ out) {
    const int ox = axis == 0 ? n_out : ix;
    const int oy = axis == 1 ? n_out : iy;
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= ox) return;
    const int y = blockIdx.y, z = blockIdx.z;
    const int p = axis == 0 ? x : (axis == 1 ? y : z);
    const int n = axis == 0 ? ix : (axis == 1 ? iy : iz);
    const long long stride = axis == 0 ? 1 : (axis == 1 ? ix : (long long)ix * iy);
    const long long base = ((long long)(axis == 2 ? 0 : z) * iy + (axis == 1 ? 0 : y)) * ix +
                           (axis == 0 ? 0 : x);
    const float q = f * p + 0.5f * (f - 1);
    const float fl = floorf(q);
    const int c = (int)fl;
    const float w = q - fl;
    float v = 0.f;
#pragma unroll
    for (int o = 0; o < 2; ++o) {
        const int pos = c + o;
        if (pos < 0 || pos >= n) continue;
        float b = 0.f;
        for (int j = -t.R; j <= t.R; ++j) {
            const int pp = pos + j;
            if (pp < 0 || pp >= n) continue;
            b += t.t[j + t.R] * ld_img(in, base + pp * stride);
        }
        v += (o ? w : 1.f - w) * b;
    }
    store_img(out, ((long long)z * oy + y) * ox + x, v);
}

__global__ void k_resample_field(const float* __restrict__ src, Geom ga,
                                 int fa, float* __restrict__ dst, Geom gb,
                                 int fb) {
    // one thread per destination voxel; y and z from the grid
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= gb.nx) return;
    const int y = blockIdx.y, z = blockIdx.z;
    const long long i = ((long long)z * gb.ny + y) * gb.nx + x;
    const int p[3] = {x, y, z};
    const int n[3] = {ga.nx, ga.ny, ga.nz};
    int c0[3], c1[3];
    float w[3];
    for (int k = 0; k < 3; ++k) {
        float fine = fb * p[k] + 0.5f * (fb - 1);
        float q = (fine - 0.5f * (fa - 1)) / fa;
        float fl = floorf(q);
        w[k] = q - fl;
        int c = (int)fl;
        c0[k] = min(max(c, 0), n[k] - 1);
        c1[k] = min(max(c + 1, 0), n[k] - 1);
    }
    float scale = (float)fa / (float)fb;
    for (int comp = 0; comp < 3; ++comp) {
        const float* U = src + comp * ga.V;
        float acc = 0.f;
        for (int s = 0; s < 8; ++s) {
            int o[3] = {s & 1, (s >> 1) & 1, s >> 2};
            int qx = o[0] ? c1[0] : c0[0];
            int qy = o[1] ? c1[1] : c0[1];
            int qz = o[2] ? c1[2] : c0[2];
            float wt = (o[0] ? w[0] : 1.f - w[0]) * (o[1] ? w[1] : 1.f - w[1]) *
                       (o[2] ? w[2] : 1.f - w[2]);
            acc += wt * U[((long long)qz * ga.ny + qy) * ga.nx + qx];
        }
        dst[comp * gb.V + i] = scale * acc;
    }
}

Taps blur_taps(double sigma) {
    Taps t{};
    int R = (int)std::ceil(3.0 * sigma);
    double w[2 * MAX_R + 1], s = 0;
    for (int j = -R; j <= R; ++j) {
        w[j + R] = std::exp(-(double)j * j / (2.0 * sigma * sigma));
        s += w[j + R];
    }
    t.R = R;
    for (int j = 0; j <= 2 * R; ++j) t.t[j] = (float)(w[j] / s);
    return t;
}

}  // namespace

void level_dims(int nx, int ny, int nz, int f, int* ox, int* oy, int* oz) {
    *ox = nx / f > 0 ? nx / f : 1;
    *oy = ny / f > 0 ? ny / f : 1;
    *oz = nz / f > 0 ? nz / f : 1;
}

int downsample_image(const void* src, int dtype, const Geom& g, int f,
                     void* dst, float* tmp, cudaStream_t s) {
    Taps t = blur_taps(0.5 * f);
    if (t.R > MAX_R) return -1;
    Geom go;
    level_dims(g.nx, g.ny, g.nz, f, &go.nx, &go.ny, &go.nz);
    // x: (nx, ny, nz) -> (lx, ny, nz); y: -> (lx, ly, nz); z: -> (lx, ly, lz)
    float* A = tmp;
    float* B = tmp + (long long)go.nx * g.ny * g.nz;
    const int TB = 128;
    const dim3 gx((go.nx + TB - 1) / TB, g.ny, g.nz);
    const dim3 gy((go.nx + TB - 1) / TB, go.ny, g.nz);
    const dim3 gz((go.nx + TB - 1) / TB, go.ny, go.nz);
    if (dtype == LM_BF16)
        k_level_axis<__nv_bfloat16, float><<<gx, TB, 0, s>>>(
            (const __nv_bfloat16*)src, g.nx, g.ny, g.nz, 0, f, go.nx, t, A);
    else
        k_level_axis<float, float><<<gx, TB, 0, s>>>(
            (const float*)src, g.nx, g.ny, g.nz, 0, f, go.nx, t, A);
    k_level_axis<float, float><<<gy, TB, 0, s>>>(A, go.nx, g.ny, g.nz, 1, f,
                                                 go.ny, t, B);
    if (dtype == LM_BF16)
        k_level_axis<float, __nv_bfloat16><<<gz, TB, 0, s>>>(
            B, go.nx, go.ny, g.nz, 2, f, go.nz, t, (__nv_bfloat16*)dst);
    else
        k_level_axis<float, float><<<gz, TB, 0, s>>>(B, go.nx, go.ny, g.nz, 2, f,
                                                     go.nz, t, (float*)dst);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

int resample_field(const float* src, const Geom& ga, int fa, float* dst,
                   const Geom& gb, int fb, cudaStream_t s) {
    const dim3 grid((gb.nx + 127) / 128, gb.ny, gb.nz);
    k_resample_field<<<grid, 128, 0, s>>>(src, ga, fa, dst, gb, fb);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

}  // namespace lmk
