// F-engine (Sec. 3 "Temporal Fourier transform"): the time samples of every antenna are
// Fourier transformed, block by block, into electric-field spectra that feed the imaging:
//   V[t][c][p][a] = sum_{j < C} x[(t C + j)][p][a] exp(-2 pi i j c / C),   c = 0 .. C-1,
// an unnormalised forward DFT of each block of C consecutive samples (bins in FFT order:
// c > C/2 are the negative frequencies), no window.
//
// One CTA per (block t, pol, tile of 32 antennas) at a time, transformed along time with
// C = R1 R2 (Cooley-Tukey): thread (antenna, n1) loads samples n1 + R2 n2 of its antenna into
// registers (coalesced: antennas contiguous; the next unit's while this one is processed),
// does their R1-point DFT there, twiddles by exp(-2 pi i n1 k2 / C) and writes the results to
// shared memory; then each thread does R2-point DFTs of (antenna, k2) and writes bins
// k2 + R1 k1 with coalesced stores.  HBM-bound: it reads the raw samples once and writes the
// spectra once; shared memory sees one write and one read per value.
#include <cuda_fp16.h>
#include "moff_common.cuh"

namespace epic {
namespace fe {

constexpr int TA = 32;   // antennas per tile

template <int C> struct Split;
template <> struct Split<32>  { static constexpr int R2 = 4; };
template <> struct Split<64>  { static constexpr int R2 = 8; };
template <> struct Split<128> { static constexpr int R2 = 8; };
template <> struct Split<256> { static constexpr int R2 = 16; };
template <> struct Split<512> { static constexpr int R2 = 16; };

template <int C>
constexpr size_t smem_bytes() { return sizeof(float2) * ((size_t)C * TA + C); }

template <int OUT> struct Out;
template <> struct Out<0> {       // complex64
    using T = float2;
    static __device__ __forceinline__ T enc(float2 v) { return v; }
};
template <> struct Out<1> {       // FP16 pair
    using T = __half2;
    static __device__ __forceinline__ T enc(float2 v) { return __floats2half2_rn(v.x, v.y); }
};

template <int C, int VIN, int OUT>
__global__ void __launch_bounds__(TA * Split<C>::R2, (TA * Split<C>::R2 <= 256) ? 3 : 1) fengine_kernel(const FengArgs a) {
    constexpr int R2 = Split<C>::R2, R1 = C / R2, NT = TA * R2;
    static_assert(R1 >= R2 && R1 <= 64 && R1 % R2 == 0, "split");
    using VT = typename Volt<VIN>::T;
    using OT = typename Out<OUT>::T;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float2* X = reinterpret_cast<float2*>(smem_raw);     // [C][TA]
    float2* TW = X + C * TA;                             // [C] exp(-2 pi i j / C)
    const int tid = threadIdx.x, al = tid % TA, n1 = tid / TA;
    for (int j = tid; j < C; j += NT) {
        double s, c;
        sincospi(-2.0 * j / C, &s, &c);
        TW[j] = make_float2(float(c), float(s));
    }
    const int A = a.n_ant, P = a.n_pol;
    const int n_tiles = (A + TA - 1) / TA;
    const int n_units = a.n_time * P * n_tiles;   // < 2^31 (checked by the caller)
    const VT* raw = static_cast<const VT*>(a.raw);
    OT* out = static_cast<OT*>(a.volt);
    const long long row = (long long)P * A;       // elements from one sample (or bin) to the next
    // raw samples of a unit (rows n1 + R2 q of its block): the next unit's are loaded into
    // registers while the current one is transformed and stored.  Unit u = (t, p, tile) with
    // the tile fastest; 32-bit coordinates, one running pointer per thread.
    VT nxt[R1];
    auto load_unit = [&](int u) {
        const int tile = u % n_tiles, tp = u / n_tiles, p = tp % P, t = tp / P;
        const int ant = tile * TA + al;
        const VT* src = raw + ((long long)t * C + n1) * row + (long long)p * A + ant;
#pragma unroll
        for (int q = 0; q < R1; ++q) nxt[q] = ant < A ? __ldg(src + q * R2 * row) : VT{};
    };
    if (blockIdx.x < n_units) load_unit(blockIdx.x);
    for (int u = blockIdx.x; u < n_units; u += gridDim.x) {
        const int tile = u % n_tiles, tp = u / n_tiles, p = tp % P, t = tp / P;
        const int ant = tile * TA + al;
        // stage 1: R1-point DFT of samples n1 + R2 n2 (the rows this thread loaded, straight from
        // registers), then the twiddle exp(-2 pi i n1 k2 / C) on the way into shared memory
        {
            float2 x[R1];
#pragma unroll
            for (int q = 0; q < R1; ++q) x[q] = Volt<VIN>::dec(nxt[q]);
            if (u + gridDim.x < n_units) load_unit(u + gridDim.x);
            dft<R1, -1>(x);
            __syncthreads();                              // previous unit's stage-2 reads are done
#pragma unroll
            for (int k2 = 0; k2 < R1; ++k2) X[(n1 + R2 * k2) * TA + al] = cmul(x[k2], TW[n1 * k2]);   // n1 k2 < C
        }
        __syncthreads();
        // stage 2: for k2 = n1, n1 + R2, ...: R2-point DFT over n1' of the row n1' + R2 k2, bins
        // c = k2 + R1 k1
#pragma unroll
        for (int q = 0; q < R1 / R2; ++q) {
            const int k2 = n1 + R2 * q;
            float2 z[R2];
#pragma unroll
            for (int m = 0; m < R2; ++m) z[m] = X[(m + R2 * k2) * TA + al];
            dft<R2, -1>(z);
            if (ant < A) {
                OT* dst = out + ((long long)t * C + k2) * row + (long long)p * A + ant;
#pragma unroll
                for (int k1 = 0; k1 < R2; ++k1) dst[k1 * R1 * row] = Out<OUT>::enc(z[k1]);
            }
        }
    }
}

template <int C, int VIN, int OUT>
cudaError_t launch_t(const FengArgs& a, int n_sm, cudaStream_t st) {
    constexpr int NT = TA * Split<C>::R2;
    const size_t smem = smem_bytes<C>();
    cudaError_t e = ensure_smem<fengine_kernel<C, VIN, OUT>>(smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fengine_kernel<C, VIN, OUT>, NT, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    const long long n_units = (long long)a.n_time * a.n_pol * ((a.n_ant + TA - 1) / TA);
    if (n_units > 2147483647LL) return cudaErrorInvalidValue;
    const long long grid = n_units < (long long)per_sm * n_sm ? n_units : (long long)per_sm * n_sm;
    if (grid == 0) return cudaSuccess;
    fengine_kernel<C, VIN, OUT><<<(unsigned)grid, NT, smem, st>>>(a);
    return cudaGetLastError();
}

template <int C>
cudaError_t launch_c(int vin, int vout, const FengArgs& a, int n_sm, cudaStream_t st) {
    switch (vin * 2 + vout) {
        case 0: return launch_t<C, 0, 0>(a, n_sm, st);
        case 1: return launch_t<C, 0, 1>(a, n_sm, st);
        case 2: return launch_t<C, 1, 0>(a, n_sm, st);
        case 3: return launch_t<C, 1, 1>(a, n_sm, st);
        case 4: return launch_t<C, 2, 0>(a, n_sm, st);
        case 5: return launch_t<C, 2, 1>(a, n_sm, st);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace fe

// vin: EPIC_VOLT_* of the raw samples; vout: 0 = complex64, 1 = FP16 pairs
cudaError_t launch_fengine(int n_chan, int vin, int vout, const FengArgs& a, int n_sm, cudaStream_t st) {
    switch (n_chan) {
        case 32: return fe::launch_c<32>(vin, vout, a, n_sm, st);
        case 64: return fe::launch_c<64>(vin, vout, a, n_sm, st);
        case 128: return fe::launch_c<128>(vin, vout, a, n_sm, st);
        case 256: return fe::launch_c<256>(vin, vout, a, n_sm, st);
        case 512: return fe::launch_c<512>(vin, vout, a, n_sm, st);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace epic
