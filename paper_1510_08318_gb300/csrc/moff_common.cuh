// Geometry, voltage decoding and shared-memory layout common to the forward and
// adjoint MOFF kernels.
#pragma once
#include <cuda_fp16.h>
#include <cooperative_groups.h>
#include "dft.cuh"
#include "epic_internal.h"

namespace epic {
namespace cg = cooperative_groups;

// Per padded size N_p: S threads cooperate on each 1-D transform; a cluster of Q CTAs
// shares one image (each CTA owns N_p/Q output columns and N_g/Q grid rows).  N_p = 512 uses
// 16-CTA clusters (a non-portable cluster size).
template <int NP> struct Cfg;
// S, Q, minimum CTAs per SM, and the shared-memory row strides (in float2) chosen so that
// every warp-wide exchange access is free of bank conflicts.
// RR: gather the cells round-robin (measured faster for the cluster sizes) or cell by cell.
// NB: most row-pass output buffers of the forward kernel (2: alternate items between two, so
// that a cluster needs no barrier per item, used where the shared memory allows).
template <> struct Cfg<32>  { static constexpr int S = 4,  Q = 1, MINB = 8, RXS = 40,  RBS = 34, NB = 1; static constexpr bool RR = false; };
template <> struct Cfg<64>  { static constexpr int S = 8,  Q = 1, MINB = 2, RXS = 72,  RBS = 66, NB = 1; static constexpr bool RR = false; };
template <> struct Cfg<128> { static constexpr int S = 8,  Q = 1, MINB = 1, RXS = 136, RBS = 129, NB = 1; static constexpr bool RR = false; };
template <> struct Cfg<256> { static constexpr int S = 16, Q = 4, MINB = 1, RXS = 264, RBS = 65, NB = 2; static constexpr bool RR = true; };
template <> struct Cfg<512> { static constexpr int S = 16, Q = 16, MINB = 1, RXS = 520, RBS = 33, NB = 1; static constexpr bool RR = true; };

template <int NP> struct Geo {
    static constexpr int NG = NP / 2;          // unpadded grid side (2x padding, Sec. 3)
    static constexpr int S = Cfg<NP>::S;
    static constexpr int Q = Cfg<NP>::Q;
    static constexpr int MINB = Cfg<NP>::MINB;
    static constexpr int R1 = NP / S;          // first-stage sub-transform length
    static constexpr int NI = NG / S;          // its non-zero inputs (= R1 / 2)
    static constexpr int KP = R1 / S;          // second-stage sub-transforms per thread
    static constexpr int ROWS = NG / Q;        // grid rows per CTA in the row pass
    static constexpr int COLS = NP / Q;        // image columns per CTA in the column pass
    static constexpr int NT = ROWS * S;        // threads per CTA
    static constexpr int LPC = 32 / S;         // rows (or columns) per warp
    static constexpr int RXS = Cfg<NP>::RXS;   // row stride of the exchange buffer (float2)
    static constexpr int RBS = Cfg<NP>::RBS;   // row stride of the row-pass output (float2)
    static constexpr int NACC = 2 * R1;        // image pixels owned by each thread
    static constexpr int VPT = 2;              // voltages prefetched per thread
    static_assert(NI * 2 == R1 && KP * S == R1 && KP >= 1, "bad factorisation");
    static_assert(COLS % R1 == 0 || Q == 1, "row-pass outputs must map to one CTA per k1");
    static_assert(RXS >= NP && RBS >= COLS, "strides");
    // XOR swizzle of the exchange buffer: keeps the first-stage writes (one n1, all k2) and
    // the second-stage reads (one k2 block, all n1) free of bank conflicts.
    static __device__ __forceinline__ int swz(int k2) { return (k2 / KP) & (S - 1); }
    // Local column (of this CTA's COLS) handled by lane group cc of `warp` in column set s.
    // For N_p = 128 the two columns read by one half-warp are 8 apart, which with an odd
    // row stride (129) makes the column loads conflict-free.
    static __device__ __forceinline__ int col(int s, int warp, int cc) {
        if constexpr (NP == 128) {
            return s * ROWS + 16 * (warp >> 2) + 2 * (warp & 3) + (cc >> 1) + 8 * (cc & 1);
        } else {
            return s * ROWS + warp * LPC + cc;
        }
    }

    static constexpr int TWS = R1 + 2;         // twiddle row stride: [S][TWS], exp(+2 pi i n1 k2 / NP)
    static constexpr int TWN = S * TWS;        // twiddle table entries
    static_assert((ROWS * RXS + NG * RBS) % 2 == 0, "twiddle table must stay 16-byte aligned");

    // the forward kernel's exchange mbarriers (two 8-byte words, cluster forms only), in float2
    static constexpr int MBF = Q > 1 ? 2 : 0;

    // forward kernel: exchange rows, nb row-pass output buffers, twiddles, mbarriers, then
    // per antenna g V, gain and partial power
    static constexpr size_t smem_bytes(int n_ant, int nb = 1) {
        return sizeof(float2) * (size_t(ROWS) * RXS + size_t(nb) * NG * RBS + TWN + MBF)
             + size_t(n_ant) * (2 * sizeof(float2) + sizeof(float));
    }
    // the cross-polarisation form adds a table of phi_v g_Y per antenna (8-byte aligned)
    static constexpr size_t smem_bytes_xpol(int n_ant, int nb = 1) {
        return smem_bytes(n_ant, nb) + size_t(n_ant + 2) * sizeof(float2);
    }

    // Fill the twiddle table from the plan's exp(+2 pi i j / NP) table.
    static __device__ __forceinline__ void load_twiddles(float2* TW, const float2* tw, int tid, int nt) {
        for (int i = tid; i < TWN; i += nt) {
            const int n1 = i / TWS, k2 = i % TWS;
            TW[i] = k2 < R1 ? tw[(n1 * k2) & (NP - 1)] : make_float2(0.f, 0.f);
        }
    }

    // Second stage of the first sub-transform: Y[k2] * exp(+2 pi i n1 k2 / NP), written to the
    // exchange row `dst` in swizzled [k2][n1] order.  Twiddles are read two at a time (16 B).
    static __device__ __forceinline__ void twiddle_store(float2* dst, const float2 (&Y)[R1], const float2* TW, int n1) {
        const float4* tw4 = reinterpret_cast<const float4*>(TW + n1 * TWS);
#pragma unroll
        for (int k2 = 0; k2 < R1; k2 += 2) {
            const float4 t = tw4[k2 / 2];
            dst[k2 * S + (n1 ^ swz(k2))] = (k2 == 0) ? Y[0] : cmul(Y[k2], make_float2(t.x, t.y));
            dst[(k2 + 1) * S + (n1 ^ swz(k2 + 1))] = cmul(Y[k2 + 1], make_float2(t.z, t.w));
        }
    }

    // Transpose of twiddle_store: read row n1 of the exchange and undo the twiddle.
    static __device__ __forceinline__ void twiddle_load_conj(const float2* src, float2 (&Y)[R1], const float2* TW, int n1) {
        const float4* tw4 = reinterpret_cast<const float4*>(TW + n1 * TWS);
#pragma unroll
        for (int k2 = 0; k2 < R1; k2 += 2) {
            const float4 t = tw4[k2 / 2];
            const float2 v0 = src[k2 * S + (n1 ^ swz(k2))], v1 = src[(k2 + 1) * S + (n1 ^ swz(k2 + 1))];
            Y[k2] = (k2 == 0) ? v0 : cmulc(v0, make_float2(t.x, t.y));
            Y[k2 + 1] = cmulc(v1, make_float2(t.z, t.w));
        }
    }
};

// acc += |z|^2 as two fused multiply-adds
__device__ __forceinline__ void acc_norm(float& acc, float2 z) { acc = fmaf(z.y, z.y, fmaf(z.x, z.x, acc)); }

// ---- raw voltage formats ---------------------------------------------------------------
template <int VDT> struct Volt;
template <> struct Volt<0> {                   // complex64
    using T = float2;
    static __device__ __forceinline__ float2 dec(T v) { return v; }
};
template <> struct Volt<1> {                   // complex half
    using T = unsigned int;
    static __device__ __forceinline__ float2 dec(T v) {
        __half2 h = *reinterpret_cast<const __half2*>(&v);
        return __half22float2(h);
    }
};
template <> struct Volt<2> {                   // signed 4+4-bit
    using T = unsigned char;
    // a two's-complement nibble n is (n ^ 8) - 8; (n ^ 8) goes into the mantissa of 2^23 and one
    // exact FP32 subtraction of 2^23 + 8 leaves the value (no integer-to-float conversion)
    static __device__ __forceinline__ float2 dec(T v) {
        const unsigned b = v;
        return make_float2(__uint_as_float(0x4B000000u | ((b >> 4) ^ 8u)) - 8388616.0f,
                           __uint_as_float(0x4B000000u | ((b & 0xFu) ^ 8u)) - 8388616.0f);
    }
};

__device__ __forceinline__ void cfma(float2& acc, float2 w, float2 v) {
    acc.x = fmaf(w.x, v.x, fmaf(-w.y, v.y, acc.x));
    acc.y = fmaf(w.x, v.y, fmaf(w.y, v.x, acc.y));
}

// Shared-memory pointer p of cluster rank q (distributed shared memory).
template <typename T>
__device__ __forceinline__ T* cluster_ptr(T* p, int q) {
    return cg::this_cluster().map_shared_rank(p, q);
}

// Gridding gather for NI cells of one thread: x[n2] = sum over the CSR row of cell
// cell0 + n2 * cstep of w * VB[antenna] (atomics-free).  RR: entries are taken round-robin over
// the cells, so that up to NI independent loads are in flight; otherwise cell by cell.
template <int NI, bool RR>
__device__ __forceinline__ void gather_cells(float2 (&x)[NI], const int* __restrict__ cell_ptr, int cell0, int cstep,
                                             const int2* __restrict__ ent, const float* __restrict__ wim,
                                             const float2* VB) {
    if constexpr (!RR) {
#pragma unroll
        for (int n2 = 0; n2 < NI; ++n2) {
            const int cell = cell0 + n2 * cstep;
            const int e0 = __ldg(cell_ptr + cell), e1 = __ldg(cell_ptr + cell + 1);
            float2 s = make_float2(0.f, 0.f);
            if (wim) {
                for (int e = e0; e < e1; ++e) {
                    const int2 en = __ldg(ent + e);
                    cfma(s, make_float2(__int_as_float(en.x), __ldg(wim + e)), VB[en.y]);
                }
            } else {
                for (int e = e0; e < e1; ++e) {
                    const int2 en = __ldg(ent + e);
                    const float w = __int_as_float(en.x);
                    const float2 v = VB[en.y];
                    s.x = fmaf(w, v.x, s.x);
                    s.y = fmaf(w, v.y, s.y);
                }
            }
            x[n2] = s;
        }
        return;
    }
    int e[NI], c[NI], cmax = 0;
#pragma unroll
    for (int n2 = 0; n2 < NI; ++n2) {
        const int cell = cell0 + n2 * cstep;
        e[n2] = __ldg(cell_ptr + cell);
        c[n2] = __ldg(cell_ptr + cell + 1) - e[n2];
        cmax = max(cmax, c[n2]);
        x[n2] = make_float2(0.f, 0.f);
    }
    if (wim) {
        for (int j = 0; j < cmax; ++j) {
#pragma unroll
            for (int n2 = 0; n2 < NI; ++n2) {
                if (j < c[n2]) {
                    const int2 en = __ldg(ent + e[n2] + j);
                    cfma(x[n2], make_float2(__int_as_float(en.x), __ldg(wim + e[n2] + j)), VB[en.y]);
                }
            }
        }
    } else {
        for (int j = 0; j < cmax; ++j) {
#pragma unroll
            for (int n2 = 0; n2 < NI; ++n2) {
                if (j < c[n2]) {
                    const int2 en = __ldg(ent + e[n2] + j);
                    const float w = __int_as_float(en.x);
                    const float2 v = VB[en.y];
                    x[n2].x = fmaf(w, v.x, x[n2].x);
                    x[n2].y = fmaf(w, v.y, x[n2].y);
                }
            }
        }
    }
}

// Gridding gather over the warp-interleaved copy of the mapping: x[n2] = sum over the entries
// of this lane's cell in group g0 + n2.  The whole warp walks k = 0 .. (largest count of the
// group) - 1; at step k the lanes with more than k entries (ranks 0 .. n_k - 1) read entry
// (start of step k) + rank, so one step's loads are one contiguous run, and the start of step
// k + 1 is that of step k plus n_k (a ballot count).  Entries of one cell are summed in the
// cell-major order, as in gather_cells.  All 32 lanes must call it together.
template <int NI>
__device__ __forceinline__ void gather_interleaved(float2 (&x)[NI], const int* __restrict__ wlane,
                                                   const int* __restrict__ wbase, const int2* __restrict__ ent,
                                                   const float* __restrict__ wim, int g0, int lane,
                                                   const float2* VB) {
#pragma unroll
    for (int n2 = 0; n2 < NI; ++n2) {
        const int word = __ldg(wlane + (g0 + n2) * 32 + lane);
        const int cnt = word & 0xffff;
        int e = __ldg(wbase + g0 + n2) + (word >> 16);
        const int kmax = __reduce_max_sync(0xffffffffu, cnt);
        float2 s = make_float2(0.f, 0.f);
        if (wim) {
            for (int k = 0; k < kmax; ++k) {
                const bool on = k < cnt;
                const int n_k = __popc(__ballot_sync(0xffffffffu, on));
                if (on) {
                    const int2 en = __ldg(ent + e);
                    cfma(s, make_float2(__int_as_float(en.x), __ldg(wim + e)), VB[en.y]);
                }
                e += n_k;
            }
        } else {
            for (int k = 0; k < kmax; ++k) {
                const bool on = k < cnt;
                const int n_k = __popc(__ballot_sync(0xffffffffu, on));
                if (on) {
                    const int2 en = __ldg(ent + e);
                    const float w = __int_as_float(en.x);
                    const float2 v = VB[en.y];
                    s.x = fmaf(w, v.x, s.x);
                    s.y = fmaf(w, v.y, s.y);
                }
                e += n_k;
            }
        }
        x[n2] = s;
    }
}

template <int Q>
__device__ __forceinline__ void block_or_cluster_sync() {
    if constexpr (Q > 1) {
        cg::this_cluster().sync();
    } else {
        __syncthreads();
    }
}

// Raise a kernel's dynamic shared-memory limit only when a launch needs more than was set
// before on the current device, so that steady-state launches make no attribute calls.
// KEY is the kernel itself (one cache per kernel, not per kernel type).
template <auto KEY>
cudaError_t ensure_smem(size_t bytes) {
    static size_t done[16] = {0};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev >= 0 && dev < 16 && done[dev] >= bytes) return cudaSuccess;
    e = cudaFuncSetAttribute(KEY, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e == cudaSuccess && dev >= 0 && dev < 16) done[dev] = bytes;
    return e;
}

// Contiguous share [beg, end) of n items for worker w of nw.
__device__ __forceinline__ void work_range(long long n, int w, int nw, long long& beg, long long& end) {
    const long long per = n / nw, rem = n % nw;
    beg = (long long)w * per + (w < rem ? w : rem);
    end = beg + per + (w < rem ? 1 : 0);
}

}  // namespace epic
