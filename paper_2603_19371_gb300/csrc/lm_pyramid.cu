// Pyramid kernels: anti-aliased downsampling of the images and resampling
// of the displacement field between levels (Section 2.1, coarse-to-fine).
#include <cmath>

#include "lm_pyramid.cuh"

namespace lmk {
namespace {

constexpr int TPB = 256;

template <typename T>
__global__ void k_blur_line(const T* __restrict__ in, Geom g, int axis,
                            Taps t, float* __restrict__ out) {
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= g.V) return;
    int x = (int)(i % g.nx);
    long long r = i / g.nx;
    int y = (int)(r % g.ny), z = (int)(r / g.ny);
    int pos = axis == 0 ? x : (axis == 1 ? y : z);
    int n = axis == 0 ? g.nx : (axis == 1 ? g.ny : g.nz);
    long long stride = axis == 0 ? 1 : (axis == 1 ? g.nx : (long long)g.nx * g.ny);
    float acc = 0.f;
    for (int j = -t.R; j <= t.R; ++j) {
        int pp = pos + j;
        if (pp < 0 || pp >= n) continue;
        acc += t.t[j + t.R] * ld_img(in, i + j * stride);
    }
    out[i] = acc;
}

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

template <typename T>
__global__ void k_level_sample(const float* __restrict__ bl, Geom g, int f,
                               Geom go, T* __restrict__ dst) {
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= go.V) return;
    int x = (int)(i % go.nx);
    long long r = i / go.nx;
    int y = (int)(r % go.ny), z = (int)(r / go.ny);
    float off = 0.5f * (f - 1);
    float q[3] = {f * x + off, f * y + off, f * z + off};
    int c[3];
    float w[3];
    for (int k = 0; k < 3; ++k) {
        float fl = floorf(q[k]);
        c[k] = (int)fl;
        w[k] = q[k] - fl;
    }
    const int n[3] = {g.nx, g.ny, g.nz};
    float acc = 0.f;
    for (int s = 0; s < 8; ++s) {
        int o[3] = {s & 1, (s >> 1) & 1, s >> 2};
        int qq[3];
        bool in = true;
        float wt = 1.f;
        for (int k = 0; k < 3; ++k) {
            qq[k] = c[k] + o[k];
            in = in && qq[k] >= 0 && qq[k] < n[k];
            wt *= o[k] ? w[k] : 1.f - w[k];
        }
        if (in)
            acc += wt * bl[((long long)qq[2] * g.ny + qq[1]) * g.nx + qq[0]];
    }
    store_img(dst, i, acc);
}

__global__ void k_resample_field(const float* __restrict__ src, Geom ga,
                                 int fa, float* __restrict__ dst, Geom gb,
                                 int fb) {
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= gb.V) return;
    int x = (int)(i % gb.nx);
    long long r = i / gb.nx;
    int y = (int)(r % gb.ny), z = (int)(r / gb.ny);
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
    unsigned nb = (unsigned)((g.V + TPB - 1) / TPB);
    float* A = tmp;
    float* B = tmp + g.V;
    if (dtype == LM_BF16)
        k_blur_line<<<nb, TPB, 0, s>>>((const __nv_bfloat16*)src, g, 0, t, A);
    else
        k_blur_line<<<nb, TPB, 0, s>>>((const float*)src, g, 0, t, A);
    k_blur_line<<<nb, TPB, 0, s>>>((const float*)A, g, 1, t, B);
    k_blur_line<<<nb, TPB, 0, s>>>((const float*)B, g, 2, t, A);
    Geom go;
    level_dims(g.nx, g.ny, g.nz, f, &go.nx, &go.ny, &go.nz);
    go.V = (long long)go.nx * go.ny * go.nz;
    unsigned nbo = (unsigned)((go.V + TPB - 1) / TPB);
    if (dtype == LM_BF16)
        k_level_sample<<<nbo, TPB, 0, s>>>(A, g, f, go, (__nv_bfloat16*)dst);
    else
        k_level_sample<<<nbo, TPB, 0, s>>>(A, g, f, go, (float*)dst);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

int resample_field(const float* src, const Geom& ga, int fa, float* dst,
                   const Geom& gb, int fb, cudaStream_t s) {
    unsigned nb = (unsigned)((gb.V + TPB - 1) / TPB);
    k_resample_field<<<nb, TPB, 0, s>>>(src, ga, fa, dst, gb, fb);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

}  // namespace lmk
