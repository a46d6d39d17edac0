// Pyramid helpers (internal): level sizes, image downsampling and field
// resampling between levels (Section 2.1, coarse-to-fine optimisation).
#pragma once

#include "lm_internal.cuh"

namespace lmk {

// Level size: max(1, n / f) per axis.
void level_dims(int nx, int ny, int nz, int f, int* ox, int* oy, int* oz);

// dst = level image of factor f: Gaussian blur (sigma = f / 2, zero
// padding), then trilinear samples at f p + (f - 1) / 2.  tmp: 2V floats.
int downsample_image(const void* src, int dtype, const Geom& g, int f,
                     void* dst, float* tmp, cudaStream_t s);

// dst (level b, factor fb) = src (level a, factor fa) read trilinearly with
// edge clamping at the level-a coordinate of each level-b voxel centre,
// times fa / fb.
int resample_field(const float* src, const Geom& ga, int fa, float* dst,
                   const Geom& gb, int fb, cudaStream_t s);

}  // namespace lmk
