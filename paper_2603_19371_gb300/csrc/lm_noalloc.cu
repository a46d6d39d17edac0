// lm_eval_noalloc: the loss / gradient evaluation without any allocation.
//
// Some callers cannot allocate device memory at the time they evaluate:
// code running inside another framework's memory pool or allocator hooks,
// real-time loops that forbid cudaMalloc/cudaFree (both synchronise the
// device), or a process that has handed all free memory to another
// component.  For them this entry point takes only the caller's inputs and
// outputs and keeps its scratch (J, dJ/du and g_raw between the evaluation
// kernels, the fixed image's fixed point, window sum and variance,
// per-CTA partials, the fixed-point scale and the reduced result) in one
// file-scope static device array, sized for volumes up to
// LM_NOALLOC_MAX_VOXELS voxels.  Every GPU that loads the library holds that
// array until the process exits.
#include <cmath>
#include <cstring>
#include <mutex>

#include "lm_kernels.cuh"

namespace {

// Scratch layout (bytes, each section 256-byte aligned):
//   g_raw               3 x LM_NOALLOC_MAX_VOXELS floats (rows padded to 4)
//   J (fixed point)     MAX_Q int32 (the LNCC kernel's halo-padded layout)
//   dJ/du               3 x LM_NOALLOC_MAX_VOXELS floats
//   F fixed point       MAX_Q int32
//   F window sum (int32), variance (float): LM_NOALLOC_MAX_VOXELS each
//   loss partials       MAX_CTAS int64 (fixed point)
//   |g|^2 partials      MAX_CTAS floats
//   image range parts   MAX_CTAS float2
//   QScale, EvalOut, the one-pair descriptor table, g_raw's tensor map,
//   the pair's non-finite flags
constexpr size_t MAX_CTAS = 1024;
// J and F in fixed point take the LNCC kernel's halo-padded layout: room
// for three times the voxel limit (a volume whose padded layout needs more
// is refused)
constexpr size_t MAX_Q = 3 * (size_t)LM_NOALLOC_MAX_VOXELS;
constexpr size_t align256(size_t n) { return (n + 255) / 256 * 256; }
constexpr size_t OFF_GRAW = 0;
constexpr size_t OFF_JQ =
    OFF_GRAW + align256(3 * (size_t)LM_NOALLOC_MAX_VOXELS * sizeof(float));
constexpr size_t OFF_DJ = OFF_JQ + align256(MAX_Q * sizeof(int));
constexpr size_t OFF_FQ =
    OFF_DJ + align256(3 * (size_t)LM_NOALLOC_MAX_VOXELS * sizeof(float));
constexpr size_t OFF_FSUM = OFF_FQ + align256(MAX_Q * sizeof(int));
constexpr size_t OFF_FVAR =
    OFF_FSUM + align256((size_t)LM_NOALLOC_MAX_VOXELS * sizeof(int));
constexpr size_t OFF_LOSS =
    OFF_FVAR + align256((size_t)LM_NOALLOC_MAX_VOXELS * sizeof(float));
constexpr size_t OFF_G2 = OFF_LOSS + align256(MAX_CTAS * sizeof(long long));
constexpr size_t OFF_MM = OFF_G2 + align256(MAX_CTAS * sizeof(float));
constexpr size_t OFF_QS = OFF_MM + align256(MAX_CTAS * sizeof(float2));
constexpr size_t OFF_OUT = OFF_QS + align256(sizeof(lmk::QScale));
constexpr size_t OFF_PD = OFF_OUT + align256(sizeof(lmk::EvalOut));
constexpr size_t OFF_TMAP = OFF_PD + align256(sizeof(lmk::PairDesc));
constexpr size_t OFF_FLAGS = OFF_TMAP + 256;       // g_raw's tensor map
constexpr size_t SCRATCH_BYTES = OFF_FLAGS + 256;  // the pair's flags

__device__ __align__(256) unsigned char g_noalloc_scratch[SCRATCH_BYTES];

constexpr int MAX_DEVICES = 64;
std::mutex g_mu;
unsigned char* g_scratch_ptr[MAX_DEVICES] = {};
int g_num_sms[MAX_DEVICES] = {};

// Failures are described through lm_last_error(), like every entry point.
int fail(int code, const char* m) {
    lmk::set_last_error(m);
    return code;
}

// Once per device, with that device current: the device address of the
// static array (host code only knows a host-side stand-in for the symbol),
// the SM count, and the kernels' shared-memory opt-in.
int setup_device(int dev, unsigned char** ptr, int* sms) {
    std::lock_guard<std::mutex> lk(g_mu);
    if (dev < 0 || dev >= MAX_DEVICES)
        return fail(LM_EUNSUPPORTED,
                    "device ordinal beyond the no-alloc device table");
    if (!g_scratch_ptr[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) {
            cudaGetLastError();
            return fail(LM_ECUDA, "cudaGetSymbolAddress of the scratch failed");
        }
        int n = 0;
        if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) !=
                cudaSuccess ||
            n < 1) {
            cudaGetLastError();
            return fail(LM_ECUDA, "cannot query the SM count");
        }
        if (lmk::fused_setup() != cudaSuccess) {
            cudaGetLastError();
            return fail(LM_ECUDA, "kernel shared-memory set-up failed");
        }
        g_num_sms[dev] = n;
        g_scratch_ptr[dev] = (unsigned char*)p;
    }
    *ptr = g_scratch_ptr[dev];
    *sms = g_num_sms[dev];
    return LM_OK;
}

// Stores the one-pair descriptor table (passed by value) on the stream.
struct Map128 {
    alignas(64) unsigned char b[128];
};

// The pair table and the g_raw tensor map, written by value into the
// scratch; the release fence orders the map for the TMA unit's reads in
// the following kernels.
__global__ void k_noalloc_table(lmk::PairDesc* dst, lmk::PairDesc v,
                                Map128* map_dst, Map128 map) {
    if (threadIdx.x == 0) {
        *dst = v;
        *map_dst = map;
        asm volatile("fence.proxy.tensormap::generic.release.gpu;\n" ::: "memory");
    }
}

// Copies the reduced scalars to the caller's device outputs.
__global__ void k_noalloc_out(const lmk::EvalOut* __restrict__ o,
                              double* __restrict__ loss,
                              float* __restrict__ gmax) {
    if (threadIdx.x != 0) return;
    if (loss) *loss = o->status ? __longlong_as_double(0x7ff8000000000000LL)
                                : o->L;
    if (gmax) *gmax = o->gmax;
}

}  // namespace

extern "C" int lm_eval_noalloc(const lm_volume* fixed, const lm_volume* moving,
                               const lm_params* p, const float* u,
                               float* g_out, double* loss_out,
                               float* gmax_out, void* cuda_stream) {
    lmk::set_last_error("");
    if (!fixed || !moving || !u || !g_out)
        return fail(LM_EINVAL, "fixed, moving, u and g_out must be non-NULL");
    if (fixed->D != moving->D || fixed->H != moving->H ||
        fixed->W != moving->W || fixed->dtype != moving->dtype)
        return fail(LM_EINVAL, "fixed and moving differ in shape or dtype");
    if (fixed->D < 1 || fixed->H < 1 || fixed->W < 1 || !fixed->data ||
        !moving->data)
        return fail(LM_EINVAL, "bad image descriptor");
    if (fixed->dtype != LM_F32 && fixed->dtype != LM_BF16)
        return fail(LM_EINVAL, "unknown dtype");
    const long long V = (long long)fixed->D * fixed->H * fixed->W;
    if (V > (long long)LM_NOALLOC_MAX_VOXELS ||
        (long long)fixed->D * fixed->H * lmk::graw_pitch(fixed->W) >
            (long long)LM_NOALLOC_MAX_VOXELS)
        return fail(LM_EINVAL,
                    "volume exceeds LM_NOALLOC_MAX_VOXELS (2^19 voxels, rows "
                    "padded to a multiple of 4) of the static scratch");
    lm_params prm;
    if (p) {
        prm = *p;
    } else {
        lm_default_params(&prm);
    }
    // the same parameter rules as lm_init
    int rc = lmk::check_params(&prm);
    if (rc != LM_OK) return rc;
    if (prm.loss == LM_LOSS_MI)
        return fail(LM_EUNSUPPORTED,
                    "the MI loss needs its histogram buffers: use lm_init");
    // every pointer the kernels dereference must be device memory: a host
    // pointer here would only fail inside a kernel
    if (!lmk::is_device_ptr(fixed->data) || !lmk::is_device_ptr(moving->data))
        return fail(LM_EINVAL, "fixed or moving data is not a device pointer");
    if (!lmk::is_device_ptr(u) || !lmk::is_device_ptr(g_out))
        return fail(LM_EINVAL, "u or g_out is not a device pointer");
    if ((loss_out && !lmk::is_device_ptr(loss_out)) ||
        (gmax_out && !lmk::is_device_ptr(gmax_out)))
        return fail(LM_EINVAL, "loss_out or gmax_out is not a device pointer");

    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return fail(LM_ECUDA, "no current device");
    }
    unsigned char* base = nullptr;
    int sms = 0;
    rc = setup_device(dev, &base, &sms);
    if (rc != LM_OK) return rc;

    cudaStream_t s = (cudaStream_t)cuda_stream;
    lmk::PairDesc pd;
    memset(&pd, 0, sizeof(pd));
    pd.g.nx = fixed->W;
    pd.g.ny = fixed->H;
    pd.g.nz = fixed->D;
    pd.g.V = V;
    pd.F = fixed->data;
    pd.M = moving->data;
    pd.target = NAN;   // explicit evaluation only: no stopping rule
    pd.u_in = u;
    pd.g_out = g_out;
    pd.graw = (float*)(base + OFF_GRAW);
    if (lmk::set_q_layout(pd, prm.win, prm.loss) > (long long)MAX_Q)
        return fail(LM_EINVAL,
                    "volume exceeds the static scratch: its halo-padded "
                    "fixed-point layout needs more than 3 LM_NOALLOC_MAX_VOXELS "
                    "elements");
    pd.flags = (unsigned*)(base + OFF_FLAGS);
    pd.jq = (int*)(base + OFF_JQ);
    pd.dj = (float*)(base + OFF_DJ);
    pd.fq = (int*)(base + OFF_FQ);
    pd.fsum = (int*)(base + OFF_FSUM);
    pd.fvar = (float*)(base + OFF_FVAR);
    pd.qs = (lmk::QScale*)(base + OFF_QS);
    lmk::BatchPlan plan = lmk::plan_batch(&pd, 1, prm.win, sms);
    if ((size_t)plan.e1_ctas > MAX_CTAS || (size_t)plan.e2_ctas > MAX_CTAS ||
        (size_t)plan.mm_ctas > MAX_CTAS)
        return fail(LM_EUNSUPPORTED, "device has more SMs than the scratch covers");
    pd.gp_w = lmk::graw_pitch(pd.g.nx);
    pd.tm_graw = base + OFF_TMAP;
    Map128 map;
    {
        int rc2 = lmk::encode_graw_map(map.b, pd.graw, pd.g,
                                       lmk::make_taps(prm.sigma_grad).R);
        if (rc2 != LM_OK) return rc2;
    }
    lmk::PairDesc* dpd = (lmk::PairDesc*)(base + OFF_PD);
    lmk::EvalOut* out = (lmk::EvalOut*)(base + OFF_OUT);

    lmk::Batch b{};
    b.pd = dpd;
    b.npairs = 1;
    b.dtype = fixed->dtype;
    b.plan = plan;
    b.c.win = prm.win;
    b.c.eps_nr = prm.eps_nr;
    b.c.eps_dr = prm.eps_dr;
    b.c.inv_k3 = (float)(1.0 / ((double)prm.win * prm.win * prm.win));
    b.c.gtaps = lmk::make_taps(prm.sigma_grad);   // as lm_init's
    b.loss = prm.loss;
    b.method = prm.method;
    b.alpha = prm.alpha;
    b.d.mse = prm.loss == LM_LOSS_MSE;
    b.d.demons = prm.method == LM_METHOD_DEMONS;
    b.part.loss = (long long*)(base + OFF_LOSS);
    b.part.g2max = (float*)(base + OFF_G2);
    b.mm_part = (float2*)(base + OFF_MM);

    k_noalloc_table<<<1, 32, 0, s>>>(dpd, pd, (Map128*)(base + OFF_TMAP), map);
    lmk::batch_prepare(b, s);
    lmk::batch_eval(b, lmk::EVAL_EXPLICIT, 0, s);
    lmk::batch_finalize(b, lmk::FIN_EXPLICIT, 0, out, s);
    k_noalloc_out<<<1, 32, 0, s>>>(out, loss_out, gmax_out);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail(LM_ECUDA, cudaGetErrorString(e));
    return LM_OK;
}
