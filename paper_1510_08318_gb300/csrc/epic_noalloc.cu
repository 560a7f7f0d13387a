// epic_image_noalloc: the imaging step of an N_p = 512 plan in the two-pass form, for callers
// that cannot allocate device memory when they image -- a pipeline whose device memory is all
// reserved up front by another allocator (a framework's caching allocator, a fixed budget per
// stage), or a real-time data path that may not stop on an allocation between samples.  The
// two-pass form stages every sample's row-transformed grid (1 MB) in scratch memory; here that
// scratch is a file-scope device array of a fixed size, so the call allocates nothing: no
// cudaMalloc, no cudaFree, no allocating library routine.
//
// The array is a property of the library, not of a plan: every GPU that loads the library holds
// it (64 MB) until the process exits, and every call on a device shares it.  A call leaves its
// last chunk's rows in it; nothing in it needs to start at zero (the row pass writes every row
// of a sample before the column pass reads it).  Calls whose kernels overlap on the GPU (on two
// streams, or two host threads) race on the array: the caller orders them.
#include <mutex>

#include "../../include/epic.h"
#include "epic_internal.h"
#include "epic_plan.h"
#include "epic_trace.h"

namespace {

// samples of 256 x 512 complex64 rows the array holds
constexpr int kNoallocSamples = 64;
constexpr size_t kNoallocBytes = (size_t)kNoallocSamples * 256 * 512 * sizeof(float2);

static __device__ __align__(256) float2 g_noalloc_scratch[kNoallocBytes / sizeof(float2)];

// Device address of the array on each device, looked up once per device with that device
// current (in host code the array's name only stands for the symbol: a kernel handed it would
// read host memory or fault).
constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mu;
float2* g_noalloc_addr[kMaxDevices] = {};

epic_status noalloc_scratch(int device, float2** out) {
    if (device < 0 || device >= kMaxDevices) return epic_fail(EPIC_EUNSUPPORTED, "device %d", device);
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_addr[device]) {
        void* p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return epic_cuda_fail(e, "static scratch address");
        g_noalloc_addr[device] = static_cast<float2*>(p);
    }
    *out = g_noalloc_addr[device];
    return EPIC_OK;
}

}  // namespace

extern "C" epic_status epic_image_noalloc(const epic_plan* plan, const void* volt, int n_time, const float* gains,
                                          double* accum, double* power, int64_t t_prev, float* image,
                                          float* autocorr, int chunk_items, void* stream) {
    EpicRange range("epic_image_noalloc");
    epic_clear_error();
    if (!plan) return epic_fail(EPIC_EINVAL, "plan is NULL");
    if (plan->n_pad != 512)
        return epic_fail(EPIC_EUNSUPPORTED, "epic_image_noalloc images n_pad 512 plans only (plan: %d)", plan->n_pad);
    if (n_time < 1) return epic_fail(EPIC_EINVAL, "n_time = %d must be >= 1", n_time);
    if (!volt || !accum) return epic_fail(EPIC_EINVAL, "NULL device array");
    if (t_prev < 0) return epic_fail(EPIC_EINVAL, "t_prev must be >= 0");
    if (chunk_items < 1 || chunk_items > kNoallocSamples)
        return epic_fail(EPIC_EINVAL,
                         "chunk_items = %d: the static scratch holds 1 to %d samples of 1 MB (%zu bytes in all)",
                         chunk_items, kNoallocSamples, kNoallocBytes);
    if (autocorr && !power) return epic_fail(EPIC_EINVAL, "autocorr needs the power accumulator");
    if (autocorr && plan->lag_side == 0)
        return epic_fail(EPIC_EUNSUPPORTED, "footprints too wide for the auto-correlation tables");
    {
        const epic_status al = epic_check_alignment({{"volt", volt, epic_volt_bytes(plan->vdt)}, {"gains", gains, 8},
                                                     {"accum", accum, 8}, {"power", power, 8}, {"image", image, 4},
                                                     {"autocorr", autocorr, 4}});
        if (al != EPIC_OK) return al;
    }
    if ((long long)plan->n_chan * plan->n_pol * n_time > 2147483647LL)
        return epic_fail(EPIC_EUNSUPPORTED, "C * P * T must stay below 2^31 per call");
    EpicDeviceGuard guard(plan->device);
    if (!guard.ok) return epic_fail(EPIC_ECUDA, "cannot select CUDA device %d", plan->device);
    int smem_optin = 0;
    cudaDeviceGetAttribute(&smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, plan->device);
    if (epic::twopass_rows_smem_bytes(plan->n_ant) > (size_t)smem_optin)
        return epic_fail(EPIC_EUNSUPPORTED, "%d antennas do not fit the two-pass row kernel's shared memory", plan->n_ant);
    float2* scratch = nullptr;
    epic_status s = noalloc_scratch(plan->device, &scratch);
    if (s != EPIC_OK) return s;

    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int cp = plan->n_chan * plan->n_pol;
    const size_t npix = (size_t)cp * plan->n_pad * plan->n_pad;
    cudaError_t e;
    if (t_prev == 0) {
        if ((e = cudaMemsetAsync(accum, 0, npix * sizeof(double), st)) != cudaSuccess) return epic_cuda_fail(e, "memset accum");
        if (power && (e = cudaMemsetAsync(power, 0, (size_t)cp * plan->n_ant * sizeof(double), st)) != cudaSuccess)
            return epic_cuda_fail(e, "memset power");
    }
    epic::SegList L;
    L.seg[0] = epic_plan_fwd_args(plan, volt, n_time, reinterpret_cast<const float2*>(gains), accum, power);
    L.first[0] = 0;
    L.first[1] = (int)L.seg[0].n_items;
    L.weight[0] = 1;
    L.cost[0] = 0;
    L.cost[1] = L.seg[0].n_items;
    L.n_seg = 1;
    L.max_ant = plan->n_ant;
    L.max_workers = 0;
    if ((e = epic::launch_fwd512_twopass(plan->vdt, L, plan->n_sm, st, scratch, chunk_items)) != cudaSuccess)
        return epic_cuda_fail(e, "two-pass imaging kernels launch");
    const double inv_t = 1.0 / double(t_prev + n_time);
    if (image && (e = epic::launch_finalize_image(accum, image, (long long)npix, inv_t, st)) != cudaSuccess)
        return epic_cuda_fail(e, "image epilogue");
    if (autocorr && (e = epic::launch_autocorr(power, plan->lag_tab, cp, plan->n_ant, plan->lag_side, plan->n_pad,
                                               inv_t, autocorr, st)) != cudaSuccess)
        return epic_cuda_fail(e, "auto-correlation epilogue");
    return EPIC_OK;
}
