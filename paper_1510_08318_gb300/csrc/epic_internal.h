// Internal declarations shared by the host API and the kernel translation units.
#pragma once
#include <cstdint>
#include <vector>
#include <cuda_runtime.h>

namespace epic {

// Everything a launch needs, all device pointers.
struct FwdArgs {
    const void* volt;          // [T][C][P][A] raw voltages
    int n_time, n_cp, n_ant;   // T, C*P, A
    const float2* gains;       // [CP][A] or nullptr (unit gains)
    const int* cell_ptr;       // [NG*NG + 1] CSR by grid cell (NG = N_p / 2)
    const int2* cell_ent;      // {weight re bits, antenna}
    const float* cell_wim;     // weight imaginary parts, or nullptr when all weights are real
    // The same mapping in warp-interleaved order (forward kernels with N_p <= 128): one group
    // per (block of 32/S grid rows, n2) whose 32 lanes own the cells the row-pass threads of a
    // warp gather; step k of a group holds the k-th entry of every lane with more than k
    // entries, lanes ordered by decreasing entry count.
    const int* wlane;          // [groups][32] entry count | (rank of the lane in that order) << 16
    const int* wbase;          // [groups] first entry of the group
    const int2* went;          // entries, {weight re bits, antenna}
    const float* wwim;         // weight imaginary parts, or nullptr
    const float2* twiddle;     // [N_p] exp(+2 pi i j / N_p)
    double* accum;             // [CP][N_p][N_p] sum_t |F_t|^2
    double* power;             // [CP][A] sum_t |g V|^2 or nullptr
    long long n_items;         // CP * T
    int flush_every;           // samples per float32 partial before a float64 flush
    float wsum_max;            // max over cells of sum_a |M[g, a]| (scales the FP16 operands)
    int* status;               // device status word of the plan (kernels with bounded waits OR in
                               // kStatus* bits when a wait runs out), or nullptr
    int wait_tries;            // tries of each bounded wait of the pipeline (about 1 ms each)
};

// Bits of a plan's device status word, set by a kernel whose bounded wait ran out (the call's
// outputs are then undefined); read and cleared by epic_sync.
constexpr int kStatusImageTimeout = 1;       // tensor-core imaging kernel
constexpr int kStatusCorrelateTimeout = 2;   // X-engine
constexpr int kStatusClusterTimeout = 4;     // FFT imaging kernel's cluster exchange (N_p >= 256)

// Sub-array calls imaged by one persistent forward launch (same N_p and voltage format);
// a single epic_image call is a one-entry list.  Passed by value as a kernel parameter.
constexpr int kMaxSeg = 64;
struct SegList {
    FwdArgs seg[kMaxSeg];      // per sub-array (n_items of each = C * P * T)
    int first[kMaxSeg + 1];    // first global item of each sub-array; first[n_seg] = total
    long long weight[kMaxSeg]; // estimated cost of one item of each sub-array (any unit)
    long long cost[kMaxSeg + 1];  // cumulative cost before each sub-array; cost[n_seg] = total
    int n_seg;
    int max_ant;               // largest antenna count (shared-memory sizing)
    int max_workers;           // cap on CTAs (clusters) launched, 0 = every resident one
    int max_buffers = 0;       // FFT form's row-pass buffers: 1 = one, 0 = as many as fit (two at
                               // N_p = 256)
};

// Per-item cost estimate of a sub-array (relative units): transform work per padded pixel
// (measured on GB300, in units of one mapping entry's gridding cost) times N_p^2, plus the
// mapping's entries.
inline long long item_weight(int n_pad, long long nnz) {
    const double per_pixel = n_pad >= 512 ? 1.15 : n_pad >= 256 ? 0.85 : n_pad >= 128 ? 0.38 : 0.3;
    return (long long)(per_pixel * double(n_pad) * double(n_pad)) + nnz + 1;
}

struct BwdArgs {
    const void* volt;
    int n_time, n_cp, n_ant;
    const float2* gains;
    const int* cell_ptr;
    const int2* cell_ent;
    const float* cell_wim;
    const int* ant_ptr;        // [Q][A+1] CSR by antenna, per row block of the grid
    const int2* ant_ent;       // {weight re bits, cell (row-block local shared-memory offset)}
    const float* ant_wim;      // weight imaginary parts, or nullptr
    const float2* twiddle;
    const float* grad_image;   // [CP][N_p][N_p] dL/dI, image pixel order
    float2* grad_gains;        // [CP][A]
    long long n_items;
    float scale;               // 2 / T
};

// F-engine (fengine.cu): per-antenna temporal DFT of blocks of C samples.
struct FengArgs {
    const void* raw;           // [T * C][P][A] time samples
    void* volt;                // [T][C][P][A] spectra (complex64 or FP16 pairs)
    long long n_time;          // T, blocks (spectra) per antenna
    int n_pol, n_ant;
};
cudaError_t launch_fengine(int n_chan, int vin, int vout, const FengArgs& a, int n_sm, cudaStream_t st);

// X-engine of the FX route (xeng.cu): visibilities of every antenna pair.
struct XengArgs {
    const void* volt;          // [T][C][P][A] raw voltages (FP16 or 4+4-bit)
    int n_time, n_cp, n_ant;
    const float2* gains;       // [CP][A] or nullptr (unit gains)
    float2* vis;               // [CP][A][A]
    int* status;               // the plan's device status word, or nullptr
    int wait_tries;            // tries of each bounded wait of the pipeline
};
size_t xeng_smem_bytes();
// FX route's imaging of visibilities (xeng.cu), N_p <= 128
struct FxArgs {
    const float2* vis;         // [CP][A][A]
    int n_cp, n_ant;
    const int* lag_ptr;        // [N_p^2 + 1] CSR of the antenna-pair kernels by wrapped lag cell
    const int4* lag_ent;       // {B_ab(d) re bits, im bits, (a * A + b) * CP, 0} of each entry
    float2* vis_t;             // scratch [A * A][CP]: the visibilities pair-major
    float2* u;                 // scratch [CP][N_p][N_p]: the lag planes
    float* image;              // [CP][N_p][N_p]
};
cudaError_t launch_fx_image(int n_pad, const FxArgs& a, cudaStream_t st);
cudaError_t launch_xeng(int vdt, const XengArgs& a, int n_sm, cudaStream_t st);

// Standalone gridder (grid.cu): E_t(g) for every sample of a call, written to device memory.
struct GridArgs {
    const void* volt;          // [T][C][P][A] raw voltages
    int n_time, n_cp, n_ant;
    const float2* gains;       // [CP][A] or nullptr (unit gains)
    const int* cell_ptr;       // cell-major mapping CSR, rows csr_width cells wide
    const int2* cell_ent;
    const float* cell_wim;
    int nnz;                   // mapping entries (length of cell_ent and cell_wim)
    int csr_width;             // N_p / 2
    int n_grid;                // N_g (output rows and columns)
    float2* out;               // [T][CP][N_g][N_g]
};

// Kernel launchers, one translation unit per padded size.  Return cudaSuccess or the
// launch error.  Shared memory is sized by the launcher.  xpol: the cross-polarisation form of
// the forward kernel (4 virtual pols per channel, see moff_fwd.cuh).
cudaError_t launch_fwd_32(int vdt, const SegList& L, int n_sm, cudaStream_t st, bool xpol = false);
cudaError_t launch_fwd_64(int vdt, const SegList& L, int n_sm, cudaStream_t st, bool xpol = false);
cudaError_t launch_fwd_128(int vdt, const SegList& L, int n_sm, cudaStream_t st, bool xpol = false);
cudaError_t launch_fwd_256(int vdt, const SegList& L, int n_sm, cudaStream_t st, bool xpol = false);
cudaError_t launch_fwd_512(int vdt, const SegList& L, int n_sm, cudaStream_t st, bool xpol = false);
cudaError_t launch_bwd_32(int vdt, const BwdArgs& a, int n_sm, cudaStream_t st);
cudaError_t launch_bwd_64(int vdt, const BwdArgs& a, int n_sm, cudaStream_t st);
cudaError_t launch_bwd_128(int vdt, const BwdArgs& a, int n_sm, cudaStream_t st);
cudaError_t launch_bwd_256(int vdt, const BwdArgs& a, int n_sm, cudaStream_t st);
cudaError_t launch_bwd_512(int vdt, const BwdArgs& a, int n_sm, cudaStream_t st);

// CTAs (Q = 1) or clusters (Q > 1) of the forward kernel resident on the whole GPU.
int resident_fwd_workers(int n_pad, int vdt, int max_ant, int n_sm);
template <int NP, int VDT> int resident_fwd_workers_t(int max_ant, int n_sm);

// Shared-memory bytes the forward / backward kernels need for a given size and antenna count.
size_t fwd_smem_bytes(int n_pad, int n_ant);
size_t fwd_xpol_smem_bytes(int n_pad, int n_ant);
size_t bwd_smem_bytes(int n_pad, int n_ant);
int grid_rows_per_block(int n_pad);   // rows of the N_g grid each CTA of a cluster owns
int fwd_interleave_lanes(int n_pad);  // S of the warp-interleaved mapping, 0 if the size does not use it
int exchange_row_stride(int n_pad);   // row stride (float2) of the kernels' exchange buffer

// Tensor-core DFT form of the forward kernel, N_p = 128 (moff_dftgemm.cu).
// Its gridding walks the 2048 cell pairs (x, y), (x, y + 1), y even, of the 64 x 64 grid in 64
// slots of 32 pairs ranked by entry count (most first), lanes of a slot in rank order; step k
// of a slot holds the k-th entry of every lane whose pair has more than k entries (the entries
// of cell y in cell-major order, then those of cell y + 1).
struct DgGather {
    const int2* lane;      // [64][32] {entries of cell y | (entries of the pair) << 16, E^T table offset of (x, y)}
    const int* base;       // [64] first entry of each slot
    const float* wre;      // entry weights, real parts
    const float* wim;      // entry weights, imaginary parts, or nullptr when every weight is real
    const uint16_t* ant;   // entry antennas
    int n_ent;             // number of entries
    // entries as one word each, (FP16 weight bits << 16) | antenna, for real weights at N_p = 256
    // (read by the FP16-gridding form); nullptr otherwise
    const uint32_t* wpk = nullptr;
};
// the least a launch needs (tables read through L1); lp: the reduced-precision form (FP16
// operands and one product per real product)
size_t dftgemm_smem_bytes(int n_ant, bool xpol = false, bool lp = false);
void dftgemm_tables(std::vector<uint16_t>& out);
// false if a pair has more than 65535 entries or an antenna index does not fit 16 bits
bool dftgemm_gather_tables(const std::vector<int>& cptr, const std::vector<int2>& cent, const std::vector<float>& cwim,
                           std::vector<int2>& lane, std::vector<int>& base, std::vector<float>& wre,
                           std::vector<float>& wim, std::vector<uint16_t>& ant);
// The same slot tables for a grid of ng x ng cells (ng = 64 or 128; ng^2 / 64 slots) gridded by
// n_warps warps, warp w walking the ceil(slots / n_warps) positions from w * that (positions no
// slot took are empty).  false as above, or for another ng.
bool dftgemm_gather_tables_ng(int ng, int n_warps, const std::vector<int>& cptr, const std::vector<int2>& cent,
                              const std::vector<float>& cwim, std::vector<int2>& lane, std::vector<int>& base,
                              std::vector<float>& wre, std::vector<float>& wim, std::vector<uint16_t>& ant);
// xpol: the (channel, pol) items are the 4 C virtual pols of dual-pol data, as in the FFT form
cudaError_t launch_dftgemm(int vdt, const FwdArgs& a, const void* wtab, const DgGather& g, int n_sm, cudaStream_t st,
                           bool xpol = false, bool lp = false);

// Tensor-core DFT form for N_p = 256 (moff_dftgemm256.cu): two CTAs per image (one per half of
// the image rows), the W tables streamed from global memory in 16 KB chunks; gather tables from
// dftgemm_gather_tables_ng(128, ...).  Single-pol images only.
constexpr int kDg256GridWarps = 15;   // gridding warps of the N_p = 256 kernel (the 16th issues)
size_t dftgemm256_smem_bytes(int n_ant);
void dftgemm256_tables(std::vector<uint16_t>& out);
// fp16_grid: FP16 gridding operands (weights and calibrated voltages rounded to FP16, FP32 sums),
// the transform unchanged; real weights need g.wpk
cudaError_t launch_dftgemm256(int vdt, const FwdArgs& a, const void* wtab, const DgGather& g, int n_sm,
                              cudaStream_t st, bool fp16_grid = false);

// Two-pass form for N_p = 512 (moff_np512x2.cu): a row pass writes each item's row-transformed
// grid (256 x 512 complex64, 1 MB) to scratch, a column pass transforms, squares and accumulates;
// items in chunks of chunk_items, scratch of twopass_scratch_bytes(chunk_items), caller-owned.
size_t twopass_scratch_bytes(int chunk_items);
size_t twopass_rows_smem_bytes(int max_ant);
cudaError_t launch_fwd512_twopass(int vdt, const SegList& L, int n_sm, cudaStream_t st, float2* scratch,
                                  int chunk_items);

// Standalone gridder: samples per work unit (8, or 4 when 8 do not fit shared memory) and launch.
size_t grid_smem_bytes(int n_ant, int tb);
int grid_samples_per_unit(int n_ant, size_t smem_optin);
cudaError_t launch_grid(int vdt, int tb, const GridArgs& a, int n_sm, cudaStream_t st);

// Epilogue kernels (finalize.cu).
cudaError_t launch_finalize_image(const double* accum, float* image, long long n, double inv_t,
                                  cudaStream_t st);
cudaError_t launch_finalize_xpol(const double* accum4, float* image, float2* cross, int n_chan, long long npix,
                                 double inv_t, cudaStream_t st);
size_t autocorr_smem_bytes(int lag_side, int n_pad, int n_ant);
size_t weff_smem_bytes(int lag_side, int n_pad);
cudaError_t launch_weff(const float2* lag_tab, int n_ant, int lag_side, int n_pad, float* out, cudaStream_t st);
cudaError_t launch_isotropic(const float* image, const float* autocorr, const float* weff, float rel_floor,
                             int n_ant, long long n, int npix, float* iso, cudaStream_t st);
cudaError_t launch_autocorr(const double* power, const float2* lag_tab, int n_cp, int n_ant,
                            int lag_side, int n_pad, double inv_t, float* out, cudaStream_t st);

}  // namespace epic
