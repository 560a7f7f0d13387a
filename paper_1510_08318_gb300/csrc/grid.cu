// Standalone gridding (Sec. 3, gridding convolution: E_t(g) = sum_a M[g, a] g_a V_a(t)) of
// every (time, channel, pol) sample onto the N_g x N_g grid, written to device memory.
//
// A work unit is one (channel, pol) and a block of TB consecutive samples.  The CTA decodes
// the unit's voltages, applies the gains and stores them in shared memory as TB/2 planes of
// float4 (two samples of one antenna per 16 bytes, plane-major so that a warp reading
// scattered antennas of one plane spreads over the banks).  Each thread then owns grid cells:
// it reads a cell's mapping entries once from the cell-major CSR (atomics-free) and applies
// them to all TB samples, then streams the TB results out with coalesced evict-first stores.
// Output bytes (8 N_g^2 per sample) dominate the traffic; the gather (shared-memory reads of the
// planes and lanes whose cells have different entry counts) keeps it below the write bandwidth.
//
// SMAP: when the mapping CSR fits beside the planes with two CTAs per SM, each persistent CTA
// copies it into shared memory once, so that the per-entry loads do not wait on L1/L2.  Either
// way the next entry of a cell is loaded while the current one is applied.
#include "moff_common.cuh"

namespace epic {

constexpr int kGridThreads = 256;
constexpr int kGridDecodeBatch = 4;   // voltage pairs loaded per thread before any is used

template <int VDT, int TB, bool SMAP>
__global__ void __launch_bounds__(kGridThreads, 2) grid_kernel(const GridArgs a) {
    static_assert(TB % 2 == 0, "samples are paired per float4");
    using VT = typename Volt<VDT>::T;
    constexpr int NQ = TB / 2;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float4* VB = reinterpret_cast<float4*>(smem_raw);   // [NQ][A]
    const int tid = threadIdx.x;
    const int A = a.n_ant, T = a.n_time, NG = a.n_grid, W = a.csr_width;
    const int cells = NG * NG;
    const int n_blk = (T + TB - 1) / TB;
    const long long n_units = (long long)a.n_cp * n_blk;
    const VT* V = static_cast<const VT*>(a.volt);

    // mapping CSR: shared-memory copy (SMAP) or the plan's device arrays
    const int* cptr = a.cell_ptr;
    const int2* cent = a.cell_ent;
    const float* cwim = a.cell_wim;
    if constexpr (SMAP) {
        const int n_ptr = W * W + 1;
        int* sp = reinterpret_cast<int*>(smem_raw + (size_t)A * TB * sizeof(float2));
        int2* se = reinterpret_cast<int2*>(sp + ((n_ptr + 3) & ~3));
        float* sw = reinterpret_cast<float*>(se + a.nnz);
        for (int i = tid; i < n_ptr; i += kGridThreads) sp[i] = __ldg(a.cell_ptr + i);
        for (int i = tid; i < a.nnz; i += kGridThreads) se[i] = __ldg(a.cell_ent + i);
        if (a.cell_wim)
            for (int i = tid; i < a.nnz; i += kGridThreads) sw[i] = __ldg(a.cell_wim + i);
        cptr = sp;
        cent = se;
        cwim = a.cell_wim ? sw : nullptr;
    }
    auto ldi = [](const int* p) { if constexpr (SMAP) return *p; else return __ldg(p); };
    auto lde = [](const int2* p) { if constexpr (SMAP) return *p; else return __ldg(p); };
    auto ldw = [](const float* p) { if constexpr (SMAP) return *p; else return __ldg(p); };

    for (long long u = blockIdx.x; u < n_units; u += gridDim.x) {
        const int cp = int(u / n_blk);
        const int t0 = int(u - (long long)cp * n_blk) * TB;
        const int tb = min(TB, T - t0);
        // decode + gains -> shared planes; samples past the end of the call are zero.  The
        // loads of kGridDecodeBatch pairs are issued before any is decoded.
        for (int i0 = tid; i0 < NQ * A; i0 += kGridThreads * kGridDecodeBatch) {
            VT r0[kGridDecodeBatch], r1[kGridDecodeBatch];
#pragma unroll
            for (int k = 0; k < kGridDecodeBatch; ++k) {
                const int i = i0 + k * kGridThreads;
                const int q = i / A, aa = i - q * A;
                const int ta = t0 + 2 * q;
                if (i < NQ * A && ta < T) r0[k] = __ldg(V + ((long long)ta * a.n_cp + cp) * A + aa);
                if (i < NQ * A && ta + 1 < T) r1[k] = __ldg(V + ((long long)(ta + 1) * a.n_cp + cp) * A + aa);
            }
#pragma unroll
            for (int k = 0; k < kGridDecodeBatch; ++k) {
                const int i = i0 + k * kGridThreads;
                if (i < NQ * A) {
                    const int q = i / A, aa = i - q * A;
                    const int ta = t0 + 2 * q;
                    const float2 g = a.gains ? __ldg(a.gains + (size_t)cp * A + aa) : make_float2(1.f, 0.f);
                    const float2 v0 = ta < T ? cmul(g, Volt<VDT>::dec(r0[k])) : make_float2(0.f, 0.f);
                    const float2 v1 = ta + 1 < T ? cmul(g, Volt<VDT>::dec(r1[k])) : make_float2(0.f, 0.f);
                    VB[i] = make_float4(v0.x, v0.y, v1.x, v1.y);
                }
            }
        }
        __syncthreads();
        for (int c = tid; c < cells; c += kGridThreads) {
            const int gy = c / NG, gx = c - gy * NG;
            const int pc = gy * W + gx;
            const int e0 = ldi(cptr + pc), e1 = ldi(cptr + pc + 1);
            float2 acc[TB];
#pragma unroll
            for (int j = 0; j < TB; ++j) acc[j] = make_float2(0.f, 0.f);
            if (cwim) {
                int2 en = e0 < e1 ? lde(cent + e0) : make_int2(0, 0);
                float wi = e0 < e1 ? ldw(cwim + e0) : 0.f;
#pragma unroll 1
                for (int e = e0; e < e1; ++e) {
                    const float2 w = make_float2(__int_as_float(en.x), wi);
                    const int ant = en.y;
                    if (e + 1 < e1) {                        // next entry in flight
                        en = lde(cent + e + 1);
                        wi = ldw(cwim + e + 1);
                    }
#pragma unroll
                    for (int q = 0; q < NQ; ++q) {
                        const float4 v = VB[q * A + ant];
                        cfma(acc[2 * q], w, make_float2(v.x, v.y));
                        cfma(acc[2 * q + 1], w, make_float2(v.z, v.w));
                    }
                }
            } else {
                int2 en = e0 < e1 ? lde(cent + e0) : make_int2(0, 0);
#pragma unroll 1
                for (int e = e0; e < e1; ++e) {
                    const float w = __int_as_float(en.x);
                    const int ant = en.y;
                    if (e + 1 < e1) en = lde(cent + e + 1);   // next entry in flight
#pragma unroll
                    for (int q = 0; q < NQ; ++q) {
                        const float4 v = VB[q * A + ant];
                        acc[2 * q].x = fmaf(w, v.x, acc[2 * q].x);
                        acc[2 * q].y = fmaf(w, v.y, acc[2 * q].y);
                        acc[2 * q + 1].x = fmaf(w, v.z, acc[2 * q + 1].x);
                        acc[2 * q + 1].y = fmaf(w, v.w, acc[2 * q + 1].y);
                    }
                }
            }
            float2* dst = a.out + ((long long)t0 * a.n_cp + cp) * cells + c;
            const long long step = (long long)a.n_cp * cells;
#pragma unroll
            for (int j = 0; j < TB; ++j)
                if (j < tb) __stcs(dst + j * step, acc[j]);
        }
        __syncthreads();
    }
}

size_t grid_smem_bytes(int n_ant, int tb) { return (size_t)n_ant * tb * sizeof(float2); }

// The shared-memory copy of the mapping CSR: row pointers (padded to 16 bytes), entries, and
// the imaginary weights when any weight is complex.
static size_t grid_map_bytes(const GridArgs& a) {
    const size_t n_ptr = (size_t)a.csr_width * a.csr_width + 1;
    return ((n_ptr + 3) & ~size_t(3)) * sizeof(int) + (size_t)a.nnz * (sizeof(int2) + (a.cell_wim ? sizeof(float) : 0));
}

int grid_samples_per_unit(int n_ant, size_t smem_optin) {
    if (grid_smem_bytes(n_ant, 16) <= smem_optin / 2) return 16;   // two CTAs per SM
    return grid_smem_bytes(n_ant, 8) <= smem_optin ? 8 : 4;
}

namespace {
template <int VDT, int TB, bool SMAP>
cudaError_t launch_grid_t(const GridArgs& a, int n_sm, size_t smem, int per_sm, cudaStream_t st) {
    const long long n_units = (long long)a.n_cp * ((a.n_time + TB - 1) / TB);
    const long long g = std::min<long long>((long long)n_sm * per_sm, n_units);
    grid_kernel<VDT, TB, SMAP><<<(unsigned)g, kGridThreads, smem, st>>>(a);
    return cudaGetLastError();
}

// Residency of one kernel form at the given dynamic shared memory (0 when it does not fit).
template <int VDT, int TB, bool SMAP>
cudaError_t grid_residency(size_t smem, int* per_sm) {
    *per_sm = 0;
    int dev = 0, optin = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e != cudaSuccess) return e;
    if (smem > (size_t)optin) return cudaSuccess;
    e = ensure_smem<grid_kernel<VDT, TB, SMAP>>(smem);
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, grid_kernel<VDT, TB, SMAP>, kGridThreads, smem);
}

// The mapping goes to shared memory when that keeps two CTAs per SM; otherwise the CSR is read
// through L1 with the same residency as before.
template <int VDT, int TB>
cudaError_t launch_grid_pick(const GridArgs& a, int n_sm, cudaStream_t st) {
    const size_t base = grid_smem_bytes(a.n_ant, TB);
    const size_t with_map = base + grid_map_bytes(a);
    int per_sm = 0;
    cudaError_t e = grid_residency<VDT, TB, true>(with_map, &per_sm);
    if (e != cudaSuccess) return e;
    if (per_sm >= 2) return launch_grid_t<VDT, TB, true>(a, n_sm, with_map, per_sm, st);
    e = grid_residency<VDT, TB, false>(base, &per_sm);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    return launch_grid_t<VDT, TB, false>(a, n_sm, base, per_sm, st);
}
}  // namespace

cudaError_t launch_grid(int vdt, int tb, const GridArgs& a, int n_sm, cudaStream_t st) {
    if (a.n_cp == 0 || a.n_time == 0 || a.n_grid == 0) return cudaSuccess;
    if (tb == 16) {
        switch (vdt) {
            case 0: return launch_grid_pick<0, 16>(a, n_sm, st);
            case 1: return launch_grid_pick<1, 16>(a, n_sm, st);
            case 2: return launch_grid_pick<2, 16>(a, n_sm, st);
        }
    } else if (tb == 8) {
        switch (vdt) {
            case 0: return launch_grid_pick<0, 8>(a, n_sm, st);
            case 1: return launch_grid_pick<1, 8>(a, n_sm, st);
            case 2: return launch_grid_pick<2, 8>(a, n_sm, st);
        }
    } else if (tb == 4) {
        switch (vdt) {
            case 0: return launch_grid_pick<0, 4>(a, n_sm, st);
            case 1: return launch_grid_pick<1, 4>(a, n_sm, st);
            case 2: return launch_grid_pick<2, 4>(a, n_sm, st);
        }
    }
    return cudaErrorInvalidValue;
}

}  // namespace epic
