// Mutual-information loss for the LM iteration (Section 2.2: the
// squared-loss form (log2 B - MI)^2 with B Parzen bins), in pass 1's loss
// stage in place of E1:
//
//   t(v)     = 1 + (B - 3) (v - lo) / (hi - lo)   bin coordinate; [lo, hi]
//                                                  is the range of F, M, 0
//   a_i(x)   = beta3(t(F(x)) - i),  b_j(x) = beta3(t(J(x)) - j)
//              cubic B-spline Parzen windows: four bins per value, sum 1
//   p_ij     = V^-1 sum_x a_i(x) b_j(x),  p_i = sum_j p_ij,  q_j = sum_i p_ij
//   MI       = sum_ij p_ij log2(p_ij / (p_i q_j))            (bits)
//   r = L    = log2 B - MI
//   dL/dJ(x) = -V^-1 t' sum_ij a_i(x) b_j'(x) log2(p_ij / q_j)
//
// Three kernels:
//   k_mi_hist   each CTA of a pair's E1 slots accumulates the joint
//               histogram of its voxel range exactly: a voxel's 16 weights
//               a_i b_j are rounded to 2^-23 and added to 32-bit
//               shared-memory bins, each lane starting at a different one
//               of its 16 (rows padded so that they fall in 16 banks);
//               after every pass of the
//               CTA (before a 32-bit bin can overflow) the bins move to
//               64-bit ones, and at the end
//               the CTA adds them to the pair's global histogram (64-bit
//               integer atomics: the sum does not depend on order or split).
//   k_mi_table  one CTA per pair reads (and clears) the histogram, then the
//               marginals and MI (sums in FP64, ratios and logs in FP32), the
//               loss r and the gradient table G_ij = log2(p_ij / q_j) (0
//               where p_ij = 0).
//   k_mi_grad   per voxel, g_raw = dL/dJ dJ/du with the table in shared
//               memory.
// F and J enter through their fixed-point codes (Fq, Jq) and the pair's
// QScale, which also holds the exact range [lo, hi].
#include "lm_kernels.cuh"
#include "lm_sample.cuh"

namespace lmk {
namespace {

constexpr int NTM = 1024;   // threads per CTA of the voxel kernels
constexpr int FQ_BAD_MI = JQ_BAD;

// Cubic B-spline and its derivative, without branches (both pieces are
// evaluated and one is selected; the outer piece is 0 beyond |x| = 2).
__device__ __forceinline__ float bsp3(float x) {
    const float a = fabsf(x);
    const float inner = fmaf(a * a, fmaf(0.5f, a, -1.f), 2.f / 3.f);
    const float b = fmaxf(2.f - a, 0.f);
    const float outer = b * b * b * (1.f / 6.f);
    return a < 1.f ? inner : outer;
}
__device__ __forceinline__ float bsp3d(float x) {
    const float a = fabsf(x);
    const float inner = a * fmaf(1.5f, a, -2.f);
    const float b = fmaxf(2.f - a, 0.f);
    const float outer = -0.5f * b * b;
    const float sg = x < 0.f ? -1.f : 1.f;
    return sg * (a < 1.f ? inner : outer);
}

// t = c0 + c1 Xq for a fixed-point code Xq (X = Xq / Q + shift); sc = t'.
struct MiCoords {
    float c0, c1, sc;
};
__device__ __forceinline__ MiCoords mi_coords(const PairDesc& P, int B) {
    const QScale q = *P.qs;
    float lo = q.lo, hi = q.hi;
    if (!(hi > lo)) hi = lo + 1.f;   // constant images: any width
    MiCoords m;
    m.sc = (float)(B - 3) / (hi - lo);
    m.c0 = fmaf(m.sc, q.shift - lo, 1.f);
    m.c1 = m.sc * q.invQ;
    return m;
}
// First of the four bins a coordinate spreads over (the top bin is cut
// off at t = B - 2, where its weight is 0).
__device__ __forceinline__ int mi_base(float t, int B) {
    return min(max((int)floorf(t) - 1, 0), B - 4);
}

// Passes between moves of the 32-bit bins: MI_FLUSH * NTM voxels of
// weight <= 4/9 at MI_HQ stay below 2^32.
constexpr int MI_FLUSH = 1;
static_assert((double)MI_FLUSH * NTM * (4.0 / 9.0) * (double)MI_HQ <
                  4294967296.0,
              "32-bit histogram bins would overflow");

// Row stride of the 32-bit shared bins: = 4 (mod 32), so that the 4 x 4
// bins around one base (offsets 4 p + q in banks) fall in 16 banks.
__host__ __device__ inline int mi_stride(int B) {
    return B + ((4 - B % 32) + 32) % 32;
}

// v[k] for a run-time k without indexing the register array
__device__ __forceinline__ float pick4(const float (&v)[4], int k) {
    return k == 0 ? v[0] : k == 1 ? v[1] : k == 2 ? v[2] : v[3];
}

__global__ void __launch_bounds__(NTM)
    k_mi_hist(const PairDesc* __restrict__ pd, int npairs, int mode,
              int attempt, int B, long long* __restrict__ loss_part,
              unsigned long long* __restrict__ mi_hist) {
    extern __shared__ unsigned long long h64[];   // B x B, then h32
    const int pi = pair_of_block<1>(pd, npairs, blockIdx.x);
    const PairDesc& P = pd[pi];
    if (trial_skip(P, mode, attempt)) return;     // block-uniform
    const int BB = B * B, S = mi_stride(B);
    unsigned* h32 = (unsigned*)(h64 + BB);        // B rows of stride S
    for (int e = threadIdx.x; e < BB; e += NTM) h64[e] = 0ull;
    for (int e = threadIdx.x; e < B * S; e += NTM) h32[e] = 0u;
    __syncthreads();
    const Geom g = P.g;
    const MiCoords mc = mi_coords(P, B);
    const int c = blockIdx.x - P.e1_cta0;
    const long long i0 = g.V * c / P.e1_ncta, i1 = g.V * (c + 1) / P.e1_ncta;
    const int* __restrict__ fqv = P.fq;
    const int* __restrict__ jqv = P.jq;
    const int rot = threadIdx.x & 15;   // this lane's first of the 16 bins
    bool bad = false;
    // CTA-uniform passes (the moves of the 32-bit bins need the whole CTA)
    int pass = 0;
    for (long long b0 = i0; b0 < i1; b0 += NTM) {
        const long long i = b0 + threadIdx.x;
        bool ok = i < i1;
        const int fq = ok ? __ldg(fqv + i) : 0;
        const int jq = ok ? __ldg(jqv + i) : 0;
        if (ok && (fq == FQ_BAD_MI || jq == JQ_BAD)) {
            bad = true;
            ok = false;
        }
        if (ok) {
            const float tf = fmaf(mc.c1, (float)fq, mc.c0);
            const float tj = fmaf(mc.c1, (float)jq, mc.c0);
            const int bf = mi_base(tf, B), bj = mi_base(tj, B);
            float a[4], w[4];
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                a[k] = bsp3(tf - (float)(bf + k));
                w[k] = bsp3(tj - (float)(bj + k));
            }
            unsigned* base = h32 + bf * S + bj;
            // lanes that share a base start at different bins of it, so an
            // atomic instruction of the warp rarely hits one address twice
#pragma unroll
            for (int t = 0; t < 16; ++t) {
                const int cc = (t + rot) & 15, p = cc >> 2, q = cc & 3;
                const unsigned v =
                    __float2uint_rn(pick4(a, p) * pick4(w, q) * MI_HQ);
                atomicAdd(base + p * S + q, v);
            }
        }
        if (++pass == MI_FLUSH) {
            pass = 0;
            __syncthreads();
            for (int e = threadIdx.x; e < BB; e += NTM) {
                const int r = e / B, col = e - r * B;
                h64[e] += h32[r * S + col];
                h32[r * S + col] = 0u;
            }
            __syncthreads();
        }
    }
    const int any_bad = __syncthreads_or(bad);
    unsigned long long* dst = mi_hist + (size_t)pi * BB;
    for (int e = threadIdx.x; e < BB; e += NTM) {
        const int r = e / B, col = e - r * B;
        const unsigned long long v = h64[e] + h32[r * S + col];
        if (v) atomicAdd(dst + e, v);
    }
    if (threadIdx.x == 0) loss_part[blockIdx.x] = any_bad ? LOSS_BAD : 0;
}

__global__ void __launch_bounds__(1024)
    k_mi_table(const PairDesc* __restrict__ pd, int mode, int attempt, int B,
               unsigned long long* __restrict__ mi_hist,
               double* __restrict__ mi_loss, float* __restrict__ mi_table) {
    __shared__ double pj[MI_MAX_BINS * MI_MAX_BINS];
    __shared__ double pf[MI_MAX_BINS], qm[MI_MAX_BINS];
    __shared__ double red[32];
    const PairDesc& P = pd[blockIdx.x];
    if (trial_skip(P, mode, attempt)) return;
    const int BB = B * B, tid = threadIdx.x;
    const double inv = 1.0 / ((double)MI_HQ * (double)P.g.V);
    unsigned long long* h = mi_hist + (size_t)blockIdx.x * BB;
    for (int e = tid; e < BB; e += blockDim.x) {
        pj[e] = (double)h[e] * inv;
        h[e] = 0ull;   // ready for the next evaluation
    }
    __syncthreads();
    if (tid < B) {
        double a = 0.0, b = 0.0;
        for (int k = 0; k < B; ++k) {
            a += pj[tid * B + k];
            b += pj[k * B + tid];
        }
        pf[tid] = a;
        qm[tid] = b;
    }
    __syncthreads();
    float* G = mi_table + (size_t)blockIdx.x * BB;
    double m = 0.0;
    // the ratios and their logs in FP32 (about 1e-7 relative): FP64
    // division and log2 would run on the narrow FP64 pipe
    for (int e = tid; e < BB; e += blockDim.x) {
        const int i = e / B, j = e - i * B;
        const double v = pj[e];
        float gv = 0.f;
        if (v > 0.0) {
            const float vf = (float)v, qf = (float)qm[j];
            m += v * (double)log2f(vf / ((float)pf[i] * qf));
            gv = log2f(vf / qf);
        }
        G[e] = gv;
    }
    for (int o = 16; o > 0; o >>= 1) m += __shfl_down_sync(0xffffffffu, m, o);
    if ((tid & 31) == 0) red[tid >> 5] = m;
    __syncthreads();
    if (tid == 0) {
        double s = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
        mi_loss[blockIdx.x] = log2((double)B) - s;
    }
}

__global__ void __launch_bounds__(NTM)
    k_mi_grad(const PairDesc* __restrict__ pd, int npairs, int mode,
              int attempt, int B, const float* __restrict__ mi_table) {
    extern __shared__ float G[];   // B x B
    const int pi = pair_of_block<1>(pd, npairs, blockIdx.x);
    const PairDesc& P = pd[pi];
    if (trial_skip(P, mode, attempt)) return;
    const int BB = B * B;
    for (int e = threadIdx.x; e < BB; e += NTM)
        G[e] = __ldg(mi_table + (size_t)pi * BB + e);
    __syncthreads();
    const Geom g = P.g;
    const MiCoords mc = mi_coords(P, B);
    const float coef = -mc.sc / (float)g.V;
    const int c = blockIdx.x - P.e1_cta0;
    const long long i0 = g.V * c / P.e1_ncta, i1 = g.V * (c + 1) / P.e1_ncta;
    const int* __restrict__ fqv = P.fq;
    const int* __restrict__ jqv = P.jq;
    const float* __restrict__ djv = P.dj;
    float* __restrict__ graw = P.graw;
    const int gpw = P.gp_w;
    const long long gcs = (long long)g.nz * g.ny * gpw;
    const bool dense = gpw == g.nx;
    // two voxels per thread and pass, their loads issued before any use
    constexpr int U = 2;
    for (long long b0 = i0; b0 < i1; b0 += (long long)U * NTM) {
      int fqk[U], jqk[U];
      float dk[U][3];
#pragma unroll
      for (int k = 0; k < U; ++k) {
        const long long i = b0 + threadIdx.x + (long long)k * NTM;
        const bool in = i < i1;
        fqk[k] = in ? __ldg(fqv + i) : FQ_BAD_MI;
        jqk[k] = in ? __ldg(jqv + i) : 0;
        dk[k][0] = in ? __ldg(djv + i) : 0.f;
        dk[k][1] = in ? __ldg(djv + g.V + i) : 0.f;
        dk[k][2] = in ? __ldg(djv + 2 * g.V + i) : 0.f;
      }
#pragma unroll
      for (int k = 0; k < U; ++k) {
        const long long i = b0 + threadIdx.x + (long long)k * NTM;
        if (i >= i1) break;
        const int fq = fqk[k], jq = jqk[k];
        const float d0 = dk[k][0], d1 = dk[k][1], d2 = dk[k][2];
        float dl = 0.f;
        if (fq != FQ_BAD_MI && jq != JQ_BAD) {
            const float tf = fmaf(mc.c1, (float)fq, mc.c0);
            const float tj = fmaf(mc.c1, (float)jq, mc.c0);
            const int bf = mi_base(tf, B), bj = mi_base(tj, B);
            float a[4], db[4];
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                a[k] = bsp3(tf - (float)(bf + k));
                db[k] = bsp3d(tj - (float)(bj + k));
            }
            float s = 0.f;
#pragma unroll
            for (int p = 0; p < 4; ++p) {
                const float* row = G + (bf + p) * B + bj;
                const float r = db[0] * row[0] + db[1] * row[1] +
                                db[2] * row[2] + db[3] * row[3];
                s = fmaf(a[p], r, s);
            }
            dl = coef * s;
        }
        const long long gi =
            dense ? i : (i / g.nx) * gpw + (i - (i / g.nx) * g.nx);
        graw[gi] = dl * d0;
        graw[gcs + gi] = dl * d1;
        graw[2 * gcs + gi] = dl * d2;
      }
    }
}

}  // namespace

static size_t mi_hist_smem(int B) {
    return (size_t)B * B * sizeof(unsigned long long) +
           (size_t)B * mi_stride(B) * sizeof(unsigned);
}

cudaError_t mi_setup() {
    return cudaFuncSetAttribute(k_mi_hist,
                                cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)mi_hist_smem(MI_MAX_BINS));
}

int launch_mi(const Batch& b, int mode, int attempt, cudaStream_t s) {
    const int BB = b.bins * b.bins;
    k_mi_hist<<<b.plan.e1_ctas, NTM, mi_hist_smem(b.bins), s>>>(
        b.pd, b.npairs, mode, attempt, b.bins, b.part.loss, b.part.mi_hist);
    k_mi_table<<<b.npairs, 1024, 0, s>>>(b.pd, mode, attempt, b.bins,
                                         b.part.mi_hist, b.part.mi_loss,
                                         b.part.mi_table);
    k_mi_grad<<<b.plan.e1_ctas, NTM, BB * sizeof(float), s>>>(
        b.pd, b.npairs, mode, attempt, b.bins, b.part.mi_table);
    return 3;
}

}  // namespace lmk
