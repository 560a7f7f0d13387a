// The plan object and host helpers shared by the C ABI translation units.
#pragma once
#include <cstddef>
#include <cstdint>
#include <initializer_list>
#include <vector>
#include <cuda_runtime.h>

#include "../../include/epic.h"
#include "epic_internal.h"

struct epic_plan {
    int n_ant = 0, n_grid = 0, n_pad = 0, n_chan = 0, n_pol = 0, vdt = 0, device = 0, n_sm = 0;
    int lag_side = 0;
    int64_t nnz = 0, n_cells = 0;
    int* cell_ptr = nullptr;
    int2* cell_ent = nullptr;
    float* cell_wim = nullptr;   // nullptr when every weight is real
    int* wlane = nullptr;        // warp-interleaved copy of the cell-major mapping (N_p <= 128)
    int* wbase = nullptr;
    int2* went = nullptr;
    float* wwim = nullptr;
    int* fx_ptr = nullptr;       // antenna-major mapping for the FX route's visibility gridding (N_p <= 128):
    int2* fx_ent = nullptr;      // [A+1] row pointers, {weight re bits, (gy << 16) | gx}
    float* fx_wim = nullptr;     // weight imaginary parts, or nullptr
    std::vector<int> fx_ptr_h;   // the same antenna-major mapping on the host (for the lag table)
    std::vector<int2> fx_ent_h;
    std::vector<float> fx_wim_h;
    // The FX route's antenna-pair kernels B_ab(d) grouped by lag cell d (CSR over the N_p^2 wrapped
    // lags: {weight re bits, im bits, (a * A + b) * C * P, 0}) and the imaging scratch (the
    // visibilities pair-major, the lag planes), built by the first epic_fx_image call
    mutable int* fx_lag_ptr = nullptr;
    mutable int4* fx_lag_ent = nullptr;
    mutable float2* fx_vis_t = nullptr;
    mutable float2* fx_u = nullptr;
    mutable int64_t fx_lag_n = -1;   // entries; -1 until built
    int* ant_ptr = nullptr;
    int2* ant_ent = nullptr;
    float* ant_wim = nullptr;
    float2* twiddle = nullptr;
    float2* lag_tab = nullptr;
    int xform = EPIC_XFORM_FFT;
    uint16_t* dg_tab = nullptr;   // DFT operand tables of the tensor-core form
    int2* dg_lane = nullptr;      // gridding slot tables of the tensor-core form (N_p = 128)
    int* dg_base = nullptr;
    float* dg_wre = nullptr;
    float* dg_wim = nullptr;
    uint16_t* dg_ant = nullptr;
    uint32_t* dg_wpk = nullptr;   // packed FP16 weight | antenna entries (N_p = 256, real weights)
    float wsum_max = 0.f;         // max over cells of sum_a |M[g, a]|
    float2* tp_scratch = nullptr; // two-pass form (N_p = 512): row-transformed grids of one chunk
    int tp_chunk = 0;             // items per chunk of the two-pass form
    int* status = nullptr;        // device status word (epic::kStatus* bits), read by epic_sync
    int wait_tries = 1000;        // tries of each bounded tensor-core wait (about 1 ms each)
};

// Alignment a device array needs for the kernels' element (or vector) accesses.
struct EpicAlign {
    const char* name;
    const void* ptr;      // nullptr (an omitted optional array) passes
    size_t bytes;
};
// EPIC_EINVAL naming the first misaligned array, else EPIC_OK (checked before any launch).
epic_status epic_check_alignment(std::initializer_list<EpicAlign> arrays);
// Bytes of one voltage sample of a format (complex64 8, FP16 pair 4, 4+4-bit 1).
size_t epic_volt_bytes(int vdt);

// Thread-local error message of the C ABI.
void epic_clear_error();
epic_status epic_fail(epic_status st, const char* fmt, ...);
epic_status epic_cuda_fail(cudaError_t e, const char* what);

// Selects a device for the scope and restores the caller's current device afterwards.
struct EpicDeviceGuard {
    int prev = -1;
    bool ok = false;
    explicit EpicDeviceGuard(int dev) {
        if (cudaGetDevice(&prev) != cudaSuccess) return;
        ok = (prev == dev) || (cudaSetDevice(dev) == cudaSuccess);
    }
    ~EpicDeviceGuard() {
        if (ok && prev >= 0) cudaSetDevice(prev);
    }
};

// Forward-kernel arguments of one plan for one call (power may be nullptr).
epic::FwdArgs epic_plan_fwd_args(const epic_plan* p, const void* volt, int n_time, const float2* gains,
                                 double* accum, double* power);
// One persistent forward launch over a list of sub-arrays of padded size n_pad.
cudaError_t epic_launch_fwd_list(int n_pad, int vdt, const epic::SegList& L, int n_sm, cudaStream_t st,
                                 bool xpol = false);
// CTAs (or clusters) of the forward kernel of a size class resident on the whole GPU.
int epic_resident_workers(int n_pad, int vdt, const std::vector<epic_plan*>& plans, const std::vector<int>& members,
                          int n_sm);
