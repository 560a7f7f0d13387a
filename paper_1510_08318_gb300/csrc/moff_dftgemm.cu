// MOFF imaging with the spatial transform as a dense DFT on the 5th-generation tensor cores
// (Eq. "dirty-image-MOFF"; the transform of Sec. 3 "Spatial Fourier Transform" written as two
// matrix products), N_p = 128 (N_g = 64):
//
//   X(ky, x)  = sum_y  W[ky][y] E(y, x)          stage 1, M = 128 (ky), K = 64 (y)
//   F(ky, kx) = sum_x  X(ky, x) W[kx][x]         stage 2, M = 128 (ky), K = 64 (x)
//   I(ky, kx) += |F|^2
//
// with W[k][n] = exp(+2 pi i n k / N_p).  Complex products are four real products; every real
// operand v is split as v = hi + lo (two FP16 numbers, hi = fp16(v), lo = fp16(v - hi)) and each
// real product is hi*hi + hi*lo + lo*hi accumulated in FP32 in tensor memory (about 22 bits of
// operand precision).  Stage 1 produces the real and imaginary parts of X in one MMA whose B
// operand stacks two E tables along N: A = Re W against B = [Re E ; Im E] and A = Im W against
// [-Im E ; Re E] (N = 128: Re X | Im X), 24 MMAs; as 48 MMAs of N = 64 it waited on shared
// memory.  Stage 2 reads A = Re X, Im X from tensor memory against B = Re W, Im W (N = 128),
// the minus sign of Re F = Re X Re W - Im X Im W taken by the instruction descriptor's negate-A
// bit, so no negated W table is stored: 48 MMAs.  Per image the gridded field is scaled by a
// power of two, chosen from a bound (largest |g V| of the sample times the largest
// sum_a |M[g, a]| of the plan), so that the FP16 operands stay in range; |F|^2 is scaled back
// exactly.
//
// One CTA per SM (16 worker warps and one issuer warp) owns all 512 TMEM columns.  Only the
// first thread of the issuer warp issues MMAs: issuing stalls while the tensor pipe's queue is
// full, and a worker that issued would hold up its share of the CUDA-core work and, through the
// CTA barriers, every other warp.  TMEM columns:
//   [0, 128)    stage-1 accumulator X (re 0..63, im 64..127), FP32
//   [128, 256)  stage-2 A operand: X re hi, re lo, im hi, im lo (FP16 pairs, 32 columns each)
//   [256, 512)  stage-2 accumulator F (re 256..383, im 384..511), FP32
// Shared memory holds the four W operand tables (re, im; hi, lo) and two buffers of the six E^T
// operand tables (-im, re, im of the hi parts, then of the lo parts, so that every stacked B
// operand is two adjacent tables), all K-major in 8 x 8 core matrices, no swizzle, and two
// buffers of decoded voltages.
//
// Pipeline (iteration i; stage 1 of image i is on the tensor pipe when it starts):
//   workers: grid image i+1 into E buffer (i+1) mod 2  |  |F|^2 epilogue of image i-1
//            (after stage 2 of i-1)  |  decode image i+2  |  split X(i) into the stage-2 A
//            operand (after stage 1 of i)  |  barrier
//   issuer:  after the barrier, stage 2 of image i, then stage 1 of image i+1
// so the gridding of the next image runs under both stages of the current one.
//
// The gridding gathers cell pairs (x, y), (x, y + 1) from slot tables in which the 32 pairs of
// a warp step have similar entry counts and store to 32 distinct shared-memory banks (on the
// 256-antenna ellipse a cell-major walk kept 40 % of the lanes busy, these slots 81 %, with the
// slowest warp at the heaviest slot).  Within a cell the builder orders the entries so that the
// antennas read at one warp step spread over the shared-memory banks of the 8-byte voltages
// (a fixed order: the sums are deterministic).  Entries are an FP32 weight and a 16-bit antenna
// index; the tables sit in shared memory when they fit beside the operand tables, else they are
// read through L1.
// Every wait on the tensor cores is bounded (the pipeline's waits by the plan's try count); on a
// timeout the CTA sets the image-timeout bit of the plan's status word, writes NaN into its
// accumulator block, waits with the full limit for the MMAs in flight and stops.
#include <cuda_fp16.h>
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <type_traits>
#include <vector>
#include "moff_common.cuh"
#include "tcgen05.cuh"

namespace epic {
namespace dg {
using namespace tc;

constexpr int NP = 128, NG = 64, NT = 512;
constexpr int VPT = 2;            // antennas per worker thread whose voltages are prefetched
constexpr int NTH = NT + 32;      // 16 worker warps + one warp whose first thread issues the MMAs
constexpr int ISSUER = NT;        // thread that issues every tcgen05.mma (never a worker)
constexpr int WTAB = NP * NG;     // halves per W table
constexpr int ETAB = NG * NG;     // halves per E^T table
enum { WR_HI, WI_HI, WR_LO, WI_LO, N_WTAB };
// E^T table order: a stacked B operand [T ; T'] is T followed by the next table in memory
enum { NEI_HI, ER_HI, EI_HI, NEI_LO, ER_LO, EI_LO, N_ETAB };
constexpr uint32_t kNegA = 1u << 13;   // instruction descriptor: negate the A operand

// (a, b) -> packed FP16 pairs hi = fp16(a, b), lo = fp16((a, b) - hi)
__device__ __forceinline__ void split2(float a, float b, uint32_t& hi, uint32_t& lo) {
    const __half2 h = __floats2half2_rn(a, b);
    const float2 f = __half22float2(h);
    const __half2 l = __floats2half2_rn(a - f.x, b - f.y);
    hi = *reinterpret_cast<const uint32_t*>(&h);
    lo = *reinterpret_cast<const uint32_t*>(&l);
}

constexpr int kWStep = 2 * WTAB / 16;    // descriptor start-field step per W table
constexpr int kEStep = 2 * ETAB / 16;    // ... per E^T table

// W and E^T tables held in shared memory: the split form keeps hi and lo parts, the reduced-
// precision form (LP) only the FP16 values (the hi tables: the first two W tables and the first
// three E^T tables of each buffer)
constexpr int n_wtab(bool lp) { return lp ? 2 : N_WTAB; }
constexpr int n_etab(bool lp) { return lp ? 3 : N_ETAB; }
constexpr size_t smem_fixed(bool lp = false) {
    return sizeof(__half) * ((size_t)n_wtab(lp) * WTAB + 2 * (size_t)n_etab(lp) * ETAB) + 64;
}
constexpr int NSLOT = NG * NG / 64;   // slots of 32 cell pairs

// Shared-memory bytes per antenna: two voltage buffers (float2, or half2 in the LP form), gains,
// power (and the Y gains of XP).
constexpr size_t ant_bytes(bool xp, bool lp = false) { return (xp ? 36 : 28) - (lp ? 8 : 0); }

// FP16 rounding of a float (the reduced-precision form's operands)
__device__ __forceinline__ float round_h(float x) { return __half2float(__float2half_rn(x)); }

// Bytes of the gather tables when they are copied into shared memory (after the per-antenna
// arrays, 16-byte aligned): slot words, slot bases, weights (and imaginary parts), antennas.
inline size_t table_smem_bytes(int n_ent, bool cw) {
    return 16 + sizeof(int2) * NSLOT * 32 + sizeof(int) * NSLOT + sizeof(float) * (size_t)n_ent * (cw ? 2 : 1) +
           sizeof(uint16_t) * (size_t)n_ent;
}

// Gather-table load: shared memory when the tables were copied there, else the read-only path.
template <bool SMT, typename T>
__device__ __forceinline__ T ldt(const T* p) {
    if constexpr (SMT) return *p;
    else return __ldg(p);
}

template <int VDT, bool SMT, bool XP, bool LP>
__global__ void __launch_bounds__(NTH, 1) moff_dftgemm_kernel(const FwdArgs a, const __half* __restrict__ wtab,
                                                              const DgGather g) {
    using VT = typename Volt<VDT>::T;
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    __half* sW = reinterpret_cast<__half*>(smem_raw);                      // [N_WTAB][WTAB]
    constexpr int NWT = n_wtab(LP), NET = n_etab(LP);
    __half* sE = sW + NWT * WTAB;                                         // [2][NET][ETAB]
    uint64_t* mbar = reinterpret_cast<uint64_t*>(sE + 2 * NET * ETAB);    // [2]
    uint32_t* tslot = reinterpret_cast<uint32_t*>(mbar + 2);
    unsigned int* vmax = reinterpret_cast<unsigned int*>(tslot + 2);      // [4] max |g V| (float bits) per image mod 4
    const int A = a.n_ant, T = a.n_time;
    float2* VB = reinterpret_cast<float2*>(smem_raw + smem_fixed(LP));    // [2][A] decoded voltages
    uint32_t* VBh = reinterpret_cast<uint32_t*>(VB);                     // LP: [2][A] half2
    float2* GN = LP ? reinterpret_cast<float2*>(VBh + 2 * A) : VB + 2 * A;
    float2* GY = GN + A;                                                  // XP only: phi_v g_Y
    float* PW = reinterpret_cast<float*>(GN + (XP ? 2 : 1) * A);
    // gather tables: copied into shared memory when they fit (SMT), else read through L1,
    // whose share of the SM's 256 KB shrinks as the shared-memory request grows
    int2* sLane = reinterpret_cast<int2*>(smem_raw + ((smem_fixed(LP) + (size_t)A * ant_bytes(XP, LP) + 15) & ~(size_t)15));
    int* sBase = reinterpret_cast<int*>(sLane + NSLOT * 32);
    float* sWre = reinterpret_cast<float*>(sBase + NSLOT);
    float* sWim = sWre + g.n_ent;
    uint16_t* sAnt = reinterpret_cast<uint16_t*>(sWre + (g.wim ? 2 : 1) * g.n_ent);
    const int2* tLane = SMT ? sLane : g.lane;
    const int* tBase = SMT ? sBase : g.base;
    const float* tWre = SMT ? sWre : g.wre;
    const float* tWim = g.wim == nullptr ? nullptr : SMT ? sWim : g.wim;
    const uint16_t* tAnt = SMT ? sAnt : g.ant;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const bool worker = tid < NT;     // the issuer warp does no gridding, decoding or epilogue work
    const VT* V = static_cast<const VT*>(a.volt);

    for (int i = tid; i < NWT * WTAB / 8; i += NTH)
        reinterpret_cast<uint4*>(sW)[i] = __ldg(reinterpret_cast<const uint4*>(wtab) + i);
    for (int aa = tid; aa < A; aa += NTH) PW[aa] = 0.f;
    if constexpr (SMT) {
        for (int q = tid; q < NSLOT * 32; q += NTH) sLane[q] = __ldg(g.lane + q);
        for (int q = tid; q < NSLOT; q += NTH) sBase[q] = __ldg(g.base + q);
        for (int q = tid; q < g.n_ent; q += NTH) {
            sWre[q] = __ldg(g.wre + q);
            sAnt[q] = __ldg(g.ant + q);
        }
        if (g.wim)
            for (int q = tid; q < g.n_ent; q += NTH) sWim[q] = __ldg(g.wim + q);
    }
    const uint32_t mb1 = smem_u32(&mbar[0]), mb2 = smem_u32(&mbar[1]);
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" :: "r"(mb1), "r"(1) : "memory");
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" :: "r"(mb2), "r"(1) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     :: "r"(smem_u32(tslot)), "r"(512) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid < 4) vmax[tid] = 0u;
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tmem = *tslot;
    const uint32_t tX = tmem, tXop = tmem + 128, tF = tmem + 256;
    const uint32_t lane_base = (uint32_t)(32 * (warp & 3)) << 16;
    // descriptors of the first W and E^T tables; the others differ only in the start-address
    // field (table size / 16 per table, 256 B / 16 per K step of 16 elements)
    const uint64_t dW0 = sdesc(smem_u32(sW), 1024), dE0 = sdesc(smem_u32(sE), 1024);
    const int qt = warp >> 2;                 // column quarter owned in the TMEM passes
    const int ky = 32 * (warp & 3) + lane;    // TMEM lane = output row

    long long beg_l, end_l;
    work_range(a.n_items, blockIdx.x, gridDim.x, beg_l, end_l);
    const int beg = (int)beg_l, n = (int)(end_l - beg_l);

    float acc[32];
#pragma unroll
    for (int j = 0; j < 32; ++j) acc[j] = 0.f;

    // voltage row of item (cp, t); for XP, cp = 4 c + v runs over the virtual pols of channel
    // c and the row is pol X of channel c (pol Y for v = 1), the Y row following it
    auto vrow = [&](int cp, int t) -> const VT* {
        if constexpr (XP) {
            const int c = cp >> 2, p = (cp & 3) == 1 ? 1 : 0;
            return V + ((long long)t * (a.n_cp >> 1) + 2 * c + p) * (long long)A;
        } else {
            return V + ((long long)t * a.n_cp + cp) * (long long)A;
        }
    };
    // raw voltages of antennas tid + NT * i (i < VPT) of an item, loaded one item ahead so the
    // decode does not wait on HBM; antennas beyond NT * VPT are loaded when decoded
    VT raw[VPT], rawy[XP ? VPT : 1];
    auto prefetch = [&](int item) {
        const int cp = item / T, t = item - cp * T;
        const VT* base = vrow(cp, t);
#pragma unroll
        for (int q = 0; q < VPT; ++q) {
            if (tid + NT * q < A) raw[q] = __ldg(base + tid + NT * q);
            if constexpr (XP) {
                if (tid + NT * q < A && (cp & 3) >= 2) rawy[q] = __ldg(base + A + tid + NT * q);
            }
        }
    };
    auto load_gains = [&](int cp) {
        if constexpr (XP) {
            // virtual pol v = cp & 3: X, Y, X + Y, X + iY; GY = phi_v g_Y (phi_2 = 1, phi_3 = i)
            const int c = cp >> 2, v = cp & 3, p = v == 1 ? 1 : 0;
            for (int aa = tid; aa < A; aa += NT) {
                GN[aa] = a.gains ? a.gains[(size_t)(2 * c + p) * A + aa] : make_float2(1.f, 0.f);
                const float2 gy = a.gains ? a.gains[(size_t)(2 * c + 1) * A + aa] : make_float2(1.f, 0.f);
                GY[aa] = v == 3 ? make_float2(-gy.y, gy.x) : gy;
            }
        } else {
            for (int aa = tid; aa < A; aa += NT)
                GN[aa] = a.gains ? a.gains[(size_t)cp * A + aa] : make_float2(1.f, 0.f);
        }
    };
    auto flush_power = [&](int cp) {
        for (int aa = tid; aa < A; aa += NT) {
            if (a.power != nullptr) atomicAdd(a.power + (size_t)cp * A + aa, (double)PW[aa]);
            PW[aa] = 0.f;
        }
    };
    // decode + gain of local image j into voltage buffer j mod 2 (workers; every thread owns the
    // same antennas in all arrays, so no barrier separates the gains, power and voltage updates);
    // the largest component magnitude goes to vmax[j mod 4] (positive float bits order like
    // unsigned integers); then the next image's voltages are prefetched
    auto decode = [&](int j) {
        const int item = beg + j, cp = item / T, t = item - cp * T;
        if (j == 0 || (item - 1) / T != cp) {
            if (j > 0) flush_power((item - 1) / T);
            load_gains(cp);
        }
        const VT* base = vrow(cp, t);
        float2* vb = VB + (j & 1) * A;
        const bool two = XP && (cp & 3) >= 2;     // virtual pol combining X and Y
        float m = 0.f;
#pragma unroll
        for (int q = 0; q < VPT; ++q) {
            const int aa = tid + NT * q;
            if (aa < A) {
                float2 vp = cmul(GN[aa], Volt<VDT>::dec(raw[q]));
                if constexpr (XP) {
                    if (two) {
                        const float2 w = cmul(GY[aa], Volt<VDT>::dec(rawy[q]));
                        vp.x += w.x;
                        vp.y += w.y;
                    }
                }
                if constexpr (LP) {
                    const __half2 hv = __floats2half2_rn(vp.x, vp.y);
                    VBh[(j & 1) * A + aa] = *reinterpret_cast<const uint32_t*>(&hv);
                } else {
                    vb[aa] = vp;
                }
                PW[aa] += cnorm(vp);
                m = fmaxf(m, fmaxf(fabsf(vp.x), fabsf(vp.y)));
            }
        }
        for (int aa = tid + NT * VPT; aa < A; aa += NT) {
            float2 vp = cmul(GN[aa], Volt<VDT>::dec(__ldg(base + aa)));
            if (two) {
                const float2 w = cmul(GY[aa], Volt<VDT>::dec(__ldg(base + A + aa)));
                vp.x += w.x;
                vp.y += w.y;
            }
            if constexpr (LP) {
                const __half2 hv = __floats2half2_rn(vp.x, vp.y);
                VBh[(j & 1) * A + aa] = *reinterpret_cast<const uint32_t*>(&hv);
            } else {
                vb[aa] = vp;
            }
            PW[aa] += cnorm(vp);
            m = fmaxf(m, fmaxf(fabsf(vp.x), fabsf(vp.y)));
        }
        if (j + 1 < n) prefetch(item + 1);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
        if (lane == 0 && m > 0.f) atomicMax(vmax + (j & 3), __float_as_uint(m));
    };
    // gridding of local image j into E buffer j mod 2 (workers); returns the image's scale 4^s
    auto grid = [&](int j) -> float {
        // |E| <= (largest sum_a |M[g, a]|) * sqrt(2) * (largest |g V| component)
        const float bound = a.wsum_max * 1.5f * __uint_as_float(vmax[j & 3]);
        int ex = 0;
        if (bound > 0.f) {
            frexpf(bound, &ex);
            ex = max(-100, min(100, ex - 9));    // scaled bound in [256, 512)
        }
        const float down = ldexpf(1.f, -ex);
        const float2* vb = VB + (j & 1) * A;
        const uint32_t* vbh = VBh + (j & 1) * A;
        // voltage of an entry's antenna: float2, or (LP) the FP16 pair widened exactly
        auto volt_of = [&](int an) -> float2 {
            if constexpr (LP) {
                const uint32_t u = vbh[an];
                return __half22float2(*reinterpret_cast<const __half2*>(&u));
            } else {
                return vb[an];
            }
        };
        // weights: FP32, or (LP) rounded to FP16 (so every product is an FP16 x FP16 product,
        // exact in FP32, and the sums accumulate in FP32)
        auto wt = [&](float w) -> float {
            if constexpr (LP) return round_h(w);
            else return w;
        };
        __half* sEj = sE + (j & 1) * NET * ETAB;
        // warp w gathers slots 4w .. 4w + 3, each 32 cell pairs of nearly equal entry count
#pragma unroll
        for (int jj = 0; jj < 4; ++jj) {
            const int slot = warp * 4 + jj;
            const int2 lw = ldt<SMT>(tLane + slot * 32 + lane);
            const int c0 = lw.x & 0xffff, cnt = (int)((unsigned)lw.x >> 16);
            const int kmax = __shfl_sync(0xffffffffu, cnt, 0);   // lane 0 has the longest list
            int e = ldt<SMT>(tBase + slot) + lane;
            float2 s0 = make_float2(0.f, 0.f), s1 = make_float2(0.f, 0.f);
            // U steps per iteration: the steps' table and voltage loads are issued before their
            // products, so U dependent load chains overlap (each lane still sums its entries in
            // table order; a lane with no entry at a step loads nothing).  Two steps made the
            // CUDA-core-bound one-product form 3 % faster (6.45 -> 6.23 ms on the LWA-like
            // workload) and the three-product form, whose tensor-core operand reads share the
            // shared-memory pipe, 2 % slower (6.49 -> 6.61 ms): one step there.
            constexpr int U = LP ? 2 : 1;
            auto walk = [&](auto cw_tag) {           // cw_tag: complex weights (tWim) or not
            constexpr bool CW = decltype(cw_tag)::value;
            for (int k = 0; k < kmax; k += U) {
                bool on[U];
                int ek[U], an[U];
                float2 w[U], v[U];
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    on[u] = k + u < cnt;
                    ek[u] = u == 0 ? e : ek[u - 1] + __popc(__ballot_sync(0xffffffffu, on[u - 1]));
                    w[u] = make_float2(0.f, 0.f);
                    an[u] = 0;
                    if (on[u]) {
                        w[u].x = wt(ldt<SMT>(tWre + ek[u]));
                        if constexpr (CW) w[u].y = wt(ldt<SMT>(tWim + ek[u]));
                        an[u] = ldt<SMT>(tAnt + ek[u]);
                    }
                }
#pragma unroll
                for (int u = 0; u < U; ++u) v[u] = on[u] ? volt_of(an[u]) : make_float2(0.f, 0.f);
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    if (!on[u]) continue;
                    if constexpr (CW) {
                        if (k + u < c0) cfma(s0, w[u], v[u]);
                        else cfma(s1, w[u], v[u]);
                    } else {
                        // both cells take the entry, one with weight 0 (adds an exact 0): no
                        // divergent branch inside the step
                        const float x0 = k + u < c0 ? w[u].x : 0.f, x1 = w[u].x - x0;
                        s0.x = fmaf(x0, v[u].x, s0.x);
                        s0.y = fmaf(x0, v[u].y, s0.y);
                        s1.x = fmaf(x1, v[u].x, s1.x);
                        s1.y = fmaf(x1, v[u].y, s1.y);
                    }
                }
                e = ek[U - 1] + __popc(__ballot_sync(0xffffffffu, on[U - 1]));
            }
            };
            if (tWim) walk(std::true_type{});
            else walk(std::false_type{});
            const int off = lw.y;   // E^T element (x, y), y even: one 32-bit word holds y and y + 1
            if constexpr (LP) {
                const __half2 hr = __floats2half2_rn(s0.x * down, s1.x * down);
                const __half2 hi2 = __floats2half2_rn(s0.y * down, s1.y * down);
                const uint32_t rh = *reinterpret_cast<const uint32_t*>(&hr);
                const uint32_t ih = *reinterpret_cast<const uint32_t*>(&hi2);
                *reinterpret_cast<uint32_t*>(sEj + ER_HI * ETAB + off) = rh;
                *reinterpret_cast<uint32_t*>(sEj + EI_HI * ETAB + off) = ih;
                *reinterpret_cast<uint32_t*>(sEj + NEI_HI * ETAB + off) = ih ^ 0x80008000u;
            } else {
                uint32_t rh, rl, ih, il;
                split2(s0.x * down, s1.x * down, rh, rl);
                split2(s0.y * down, s1.y * down, ih, il);
                *reinterpret_cast<uint32_t*>(sEj + ER_HI * ETAB + off) = rh;
                *reinterpret_cast<uint32_t*>(sEj + ER_LO * ETAB + off) = rl;
                *reinterpret_cast<uint32_t*>(sEj + EI_HI * ETAB + off) = ih;
                *reinterpret_cast<uint32_t*>(sEj + EI_LO * ETAB + off) = il;
                // split(-v) = -split(v) exactly: flip both halves' sign bits
                *reinterpret_cast<uint32_t*>(sEj + NEI_HI * ETAB + off) = ih ^ 0x80008000u;
                *reinterpret_cast<uint32_t*>(sEj + NEI_LO * ETAB + off) = il ^ 0x80008000u;
            }
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");   // E^T visible to the tensor cores
        return ldexpf(1.f, 2 * ex);
    };
    auto flush_acc = [&](int cp) {
        double* dst = a.accum + (size_t)cp * NP * NP;
        const int iy = (ky + NP / 2) & (NP - 1);
#pragma unroll
        for (int j = 0; j < 32; ++j) {
            const int ix = (32 * qt + j + NP / 2) & (NP - 1);
            atomicAdd(dst + iy * NP + ix, (double)acc[j]);
            acc[j] = 0.f;
        }
    };
    int since = 0;
    // |F|^2 epilogue of local image j (workers, after its stage 2 has completed)
    auto epilogue = [&](int j, float scale) {
#pragma unroll
        for (int c = 0; c < 32; c += 16) {
            float fr[16], fi[16];
            tld<16>(tF + lane_base + 32 * qt + c, fr);
            tld<16>(tF + 128 + lane_base + 32 * qt + c, fi);
            tld_wait();
#pragma unroll
            for (int u = 0; u < 16; ++u) acc[c + u] = fmaf(fmaf(fr[u], fr[u], fi[u] * fi[u]), scale, acc[c + u]);
        }
        ++since;
        const int item = beg + j, cp = item / T;
        if (j + 1 == n || (item + 1) / T != cp || since == a.flush_every) {
            flush_acc(cp);
            since = 0;
        }
    };
    // split X into the stage-2 A operand in TMEM (workers, after its stage 1 has completed);
    // quarter qt: part (re / im) = qt >> 1, x range 32 * (qt & 1) .. + 32
    auto split = [&]() {
        const int part = qt >> 1, hx = qt & 1;
        const uint32_t src = tX + lane_base + 64 * part + 32 * hx;
        const uint32_t dhi = tXop + lane_base + 64 * part + 16 * hx;
        const uint32_t dlo = dhi + 32;
#pragma unroll
        for (int c = 0; c < 32; c += 16) {
            float xv[16];
            tld<16>(src + c, xv);
            tld_wait();
            uint32_t ph[8], pl[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                if constexpr (LP) {
                    const __half2 h = __floats2half2_rn(xv[2 * u], xv[2 * u + 1]);
                    ph[u] = *reinterpret_cast<const uint32_t*>(&h);
                } else {
                    split2(xv[2 * u], xv[2 * u + 1], ph[u], pl[u]);
                }
            }
            tst8(dhi + c / 2, ph);
            if constexpr (!LP) tst8(dlo + c / 2, pl);
        }
        tst_wait();
    };
    // stage 1 of the image in E buffer b: X = W E (columns transformed)
    auto issue_stage1 = [&](int b) {
        constexpr uint32_t id1 = idesc(128);
        // A = W table, B = [table ; next table]: Re W [Re E ; Im E], Im W [-Im E ; Re E]
        constexpr int ta[6] = {WR_HI, WR_HI, WR_LO, WI_HI, WI_HI, WI_LO};
        constexpr int tb[6] = {ER_HI, ER_LO, ER_HI, NEI_HI, NEI_LO, NEI_HI};
        const uint64_t dE = dE0 + (uint64_t)(b * NET * kEStep);
#pragma unroll
        for (int q = 0; q < 6; ++q) {
            if (LP && q % 3 != 0) continue;     // LP: the hi*hi products only
#pragma unroll
            for (int j = 0; j < 4; ++j)
                mma_ss(tX, dW0 + (uint64_t)(ta[q] * kWStep + 16 * j), dE + (uint64_t)(tb[q] * kEStep + 16 * j), id1,
                       (q | j) != 0);
        }
        commit(mb1);
    };
    // stage 2: F = X W^T (rows transformed); A operand columns: X re hi/lo at +0/+32, X im
    // hi/lo at +64/+96.  Re F = Re X Re W - Im X Im W, Im F = Re X Im W + Im X Re W.
    auto issue_stage2 = [&]() {
        constexpr uint32_t id2 = idesc(128);
        constexpr int ar[6] = {0, 0, 32, 64, 64, 96};
        constexpr int bre[6] = {WR_HI, WR_LO, WR_HI, WI_HI, WI_LO, WI_HI};
        constexpr int bim[6] = {WI_HI, WI_LO, WI_HI, WR_HI, WR_LO, WR_HI};
#pragma unroll
        for (int q = 0; q < 6; ++q) {
            if (LP && q % 3 != 0) continue;     // LP: the hi*hi products only
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                mma_ts(tF, tXop + ar[q] + 8 * j, dW0 + (uint64_t)(bre[q] * kWStep + 16 * j), q < 3 ? id2 : id2 | kNegA,
                       (q | j) != 0);
                mma_ts(tF + 128, tXop + ar[q] + 8 * j, dW0 + (uint64_t)(bim[q] * kWStep + 16 * j), id2, (q | j) != 0);
            }
        }
        commit(mb2);
    };

    bool failed = false;
    int issued1 = 0, issued2 = 0;   // stage-1 / stage-2 batches committed
    float sc_prev = 1.f, sc_cur = 1.f, sc_next = 1.f;   // 4^s of images i-1, i, i+1
    if (n > 0) {
        // prologue: decode images 0 and 1, grid image 0, stage 1 of image 0
        if (worker) {
            prefetch(beg);
            decode(0);
        }
        __syncthreads();
        if (worker) {
            sc_cur = grid(0);
            if (n > 1) decode(1);
        }
        __syncthreads();
        if (tid == ISSUER) {
            fence_after();
            issue_stage1(0);
        }
        ++issued1;
        if (tid == 0) vmax[0] = 0u;
    }
    // a wait that runs out sets `failed` (the warp-collective TMEM passes after it still run, on
    // values that are then discarded), and the CTA stops at the next barrier
    for (int i = 0; i < n; ++i) {
        if (worker) {
            if (i + 1 < n) sc_next = grid(i + 1);
            if (i >= 1) {
                if (!mbar_wait(mb2, (i - 1) & 1, a.wait_tries)) failed = true;
                fence_after();
                epilogue(i - 1, sc_prev);
            }
            if (i + 2 < n) decode(i + 2);
            if (!mbar_wait(mb1, i & 1, a.wait_tries)) failed = true;
            fence_after();
            split();
        }
        fence_before();
        failed = __syncthreads_or(failed) != 0;   // uniform across the CTA
        if (failed) break;
        if (tid == ISSUER) {
            fence_after();
            issue_stage2();
            if (i + 1 < n) issue_stage1((i + 1) & 1);
        }
        ++issued2;
        if (i + 1 < n) ++issued1;
        if (tid == 0) vmax[(i + 1) & 3] = 0u;   // read by the gridding of image i + 1, done
        sc_prev = sc_cur;
        sc_cur = sc_next;
    }
    if (!failed && n > 0 && worker) {
        if (!mbar_wait(mb2, (n - 1) & 1, a.wait_tries)) failed = true;
        fence_after();
        epilogue(n - 1, sc_prev);
        flush_power((beg + n - 1) / T);
    }
    failed = __syncthreads_or(failed) != 0;
    if (failed) {
        // a tensor-core wait ran out: report it in the plan's status word, mark this CTA's first
        // (channel, pol) block with NaN, wait (bounded, with the full limit) for the batches
        // still in flight, so that no MMA writes the tensor memory after it is released, and stop
        if (n > 0 && tid == 0) {
            if (a.status) atomicOr(a.status, kStatusImageTimeout);
            a.accum[(size_t)(beg / T) * NP * NP] = __longlong_as_double(0x7ff8000000000000LL);
        }
        if (issued1 > 0) mbar_wait(mb1, (issued1 - 1) & 1);
        if (issued2 > 0) mbar_wait(mb2, (issued2 - 1) & 1);
    }
    fence_before();
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(tmem), "r"(512) : "memory");
}

}  // namespace dg

size_t dftgemm_smem_bytes(int n_ant, bool xpol, bool lp) {
    return dg::smem_fixed(lp) + (size_t)n_ant * dg::ant_bytes(xpol, lp);
}

// W operand tables for N_p = 128: four [128][64] K-major FP16 tables (re, im hi parts, then
// the same lo parts) of W[k][n] = exp(+2 pi i n k / 128), computed in float64.
void dftgemm_tables(std::vector<uint16_t>& out) {
    using namespace dg;
    out.assign((size_t)N_WTAB * WTAB, 0);
    for (int k = 0; k < NP; ++k)
        for (int n = 0; n < NG; ++n) {
            const double ang = 2.0 * 3.14159265358979323846 * double((n * k) % NP) / double(NP);
            const double vals[2] = {std::cos(ang), std::sin(ang)};
            const int thi[2] = {WR_HI, WI_HI}, tlo[2] = {WR_LO, WI_LO};
            for (int c = 0; c < 2; ++c) {
                const __half hi = __double2half(vals[c]);
                const __half lo = __double2half(vals[c] - (double)__half2float(hi));
                out[(size_t)thi[c] * WTAB + koff(k, n, NG)] = __half_as_ushort(hi);
                out[(size_t)tlo[c] * WTAB + koff(k, n, NG)] = __half_as_ushort(lo);
            }
        }
}

// Slot tables of the tensor-core forms' gridding on an ng x ng grid (64 for N_p = 128, 128 for
// N_p = 256).  The word of pair (x, y), y even, lands in shared-memory bank
// 4 (x mod 8) + (y / 2 mod 4) of every E^T table, so the ng^2 / 2 pairs fall into 32 bank
// classes.  Within each class pairs are ranked by entry count (most first,
// ties by position) and slot r takes the r-th pair of every class: its 32 lanes store to 32
// distinct banks, and classes interleave finely enough over the aperture that the r-th pairs
// of all classes have similar counts.  A slot takes max(count) warp steps; slots go to the
// n_warps gridding warps heaviest first, each to the warp with the fewest steps so far among
// those holding fewer than ceil(slots / n_warps) (ties to the lowest warp), so the slowest
// warp's gridding is about the heaviest slot or the mean, whichever is larger.  Warp w walks
// positions w * ceil(slots / n_warps) ..; positions no slot took hold no entries.
bool dftgemm_gather_tables_ng(int ng, int n_warps, const std::vector<int>& cptr, const std::vector<int2>& cent,
                              const std::vector<float>& cwim, std::vector<int2>& lane, std::vector<int>& base,
                              std::vector<float>& wre, std::vector<float>& wim, std::vector<uint16_t>& ant) {
    using tc::koff;
    const int NW = n_warps;
    const int NPAIR = ng * ng / 2, nslot = NPAIR / 32;
    if ((ng != 64 && ng != 128) || NW < 1 || NW > 32) return false;
    const int per_warp = (nslot + NW - 1) / NW;   // positions per warp; those left over stay empty
    for (const int2& c : cent)
        if (c.y < 0 || c.y > 0xffff) return false;
    struct Pair { int cell, c0, cnt, off; };
    std::vector<Pair> pr(NPAIR);
    for (int yp = 0; yp < ng / 2; ++yp)
        for (int x = 0; x < ng; ++x) {
            const int c = 2 * yp * ng + x;
            const int n0 = cptr[c + 1] - cptr[c], n1 = cptr[c + ng + 1] - cptr[c + ng];
            if (n0 + n1 > 0xffff) return false;
            pr[yp * ng + x] = {c, n0, n0 + n1, koff(x, 2 * yp, ng)};
        }
    auto heavier = [&](int u, int v) { return pr[u].cnt > pr[v].cnt; };
    std::vector<std::vector<int>> cls(32);
    for (int q = 0; q < NPAIR; ++q) cls[4 * ((q % ng) & 7) + ((q / ng) & 3)].push_back(q);
    for (auto& c : cls) std::stable_sort(c.begin(), c.end(), heavier);
    std::vector<std::vector<int>> slots(nslot);
    for (int r = 0; r < nslot; ++r) {
        for (int c = 0; c < 32; ++c) slots[r].push_back(cls[c][r]);
        std::stable_sort(slots[r].begin(), slots[r].end(), heavier);   // lanes in rank order
    }
    std::stable_sort(slots.begin(), slots.end(), [&](const std::vector<int>& u, const std::vector<int>& v) {
        return pr[u[0]].cnt > pr[v[0]].cnt;
    });
    std::vector<int> order;
    for (const auto& sl : slots) order.insert(order.end(), sl.begin(), sl.end());
    lane.assign((size_t)NW * per_warp * 32, int2{0, 0});
    base.assign((size_t)NW * per_warp, -1);   // -1: a position no slot takes (skipped by the kernels)
    wre.clear();
    wim.clear();
    ant.clear();
    std::vector<int> held(NW, 0), steps(NW, 0);
    for (int r = 0; r < nslot; ++r) {
        int w = -1;
        for (int v = 0; v < NW; ++v)
            if (held[v] < per_warp && (w < 0 || steps[v] < steps[w])) w = v;
        const int pos = per_warp * w + held[w]++;
        steps[w] += pr[order[32 * r]].cnt;
        const Pair* P[32];
        for (int i = 0; i < 32; ++i) P[i] = &pr[order[32 * r + i]];
        base[pos] = (int)wre.size();
        for (int i = 0; i < 32; ++i)
            lane[(size_t)pos * 32 + i] = int2{(int)((unsigned)P[i]->c0 | ((unsigned)P[i]->cnt << 16)), P[i]->off};
        // Each lane takes its first cell's entries, then its second's; within a cell the order is
        // free (any fixed order is deterministic), so step by step each lane takes, of its cell's
        // remaining entries, one whose antenna shares a shared-memory bank pair (8-byte voltages:
        // antenna mod 16) with as few antennas already read at this step by its half-warp as
        // possible; lanes with the fewest candidates choose first.
        std::vector<int> rem[32][2];
        for (int i = 0; i < 32; ++i) {
            for (int e = cptr[P[i]->cell]; e < cptr[P[i]->cell + 1]; ++e) rem[i][0].push_back(e);
            for (int e = cptr[P[i]->cell + ng]; e < cptr[P[i]->cell + ng + 1]; ++e) rem[i][1].push_back(e);
        }
        for (int k = 0; k < P[0]->cnt; ++k) {
            int n_act = 0;
            while (n_act < 32 && P[n_act]->cnt > k) ++n_act;
            auto cand = [&](int i) -> std::vector<int>& { return rem[i][k < P[i]->c0 ? 0 : 1]; };
            int ord[32], pick[32], load[2][16] = {};
            std::vector<int> seen[2];            // antennas read at this step, per half-warp
            for (int i = 0; i < n_act; ++i) ord[i] = i;
            std::stable_sort(ord, ord + n_act, [&](int u, int v) { return cand(u).size() < cand(v).size(); });
            for (int t = 0; t < n_act; ++t) {
                const int i = ord[t], h = i / 16;
                std::vector<int>& c = cand(i);
                size_t best = 0;
                int best_cost = 1 << 30;
                for (size_t j = 0; j < c.size(); ++j) {
                    const int an = cent[c[j]].y;
                    const bool dup = std::find(seen[h].begin(), seen[h].end(), an) != seen[h].end();
                    const int cost = dup ? -1 : load[h][an & 15];
                    if (cost < best_cost) {
                        best_cost = cost;
                        best = j;
                    }
                }
                pick[i] = c[best];
                c.erase(c.begin() + (long)best);
                const int an = cent[pick[i]].y;
                if (best_cost >= 0) {
                    ++load[h][an & 15];
                    seen[h].push_back(an);
                }
            }
            for (int i = 0; i < n_act; ++i) {
                const int e = pick[i];
                float wv;
                std::memcpy(&wv, &cent[e].x, sizeof(float));
                wre.push_back(wv);
                wim.push_back(cwim[e]);
                ant.push_back((uint16_t)cent[e].y);
            }
        }
    }
    return true;
}

bool dftgemm_gather_tables(const std::vector<int>& cptr, const std::vector<int2>& cent, const std::vector<float>& cwim,
                           std::vector<int2>& lane, std::vector<int>& base, std::vector<float>& wre,
                           std::vector<float>& wim, std::vector<uint16_t>& ant) {
    static_assert(dg::NSLOT * 32 == dg::NG * dg::NG / 2 && dg::NSLOT == 4 * (dg::NT / 32),
                  "four slots of 32 pairs per worker warp");
    return dftgemm_gather_tables_ng(dg::NG, dg::NT / 32, cptr, cent, cwim, lane, base, wre, wim, ant);
}

cudaError_t launch_dftgemm(int vdt, const FwdArgs& a, const void* wtab, const DgGather& g, int n_sm, cudaStream_t st,
                           bool xpol, bool lp) {
    const __half* w = static_cast<const __half*>(wtab);
    int dev = 0, optin = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev)) != cudaSuccess) return e;
    // the gather tables go into shared memory when the whole request still fits one block
    if (lp && xpol) return cudaErrorInvalidValue;
    const size_t base = (dftgemm_smem_bytes(a.n_ant, xpol, lp) + 15) & ~(size_t)15;
    const size_t with_tables = base + dg::table_smem_bytes(g.n_ent, g.wim != nullptr);
    const bool smt = with_tables <= (size_t)optin;
    const size_t smem = smt ? with_tables : dftgemm_smem_bytes(a.n_ant, xpol, lp);
    long long grid = n_sm;
    if (grid > a.n_items) grid = a.n_items;
    switch (vdt * 8 + (smt ? 4 : 0) + (xpol ? 2 : 0) + (lp ? 1 : 0)) {
#define EPIC_DG_CASE(V, S, X, L)                                                                             \
    case V * 8 + S * 4 + X * 2 + L:                                                                          \
        e = ensure_smem<dg::moff_dftgemm_kernel<V, S, X, L>>(smem);                                          \
        if (e != cudaSuccess) return e;                                                                      \
        if (grid > 0) dg::moff_dftgemm_kernel<V, S, X, L><<<(unsigned)grid, dg::NTH, smem, st>>>(a, w, g);    \
        return cudaGetLastError();
        EPIC_DG_CASE(0, 0, 0, 0)
        EPIC_DG_CASE(0, 0, 1, 0)
        EPIC_DG_CASE(0, 0, 0, 1)
        EPIC_DG_CASE(0, 1, 0, 0)
        EPIC_DG_CASE(0, 1, 1, 0)
        EPIC_DG_CASE(0, 1, 0, 1)
        EPIC_DG_CASE(1, 0, 0, 0)
        EPIC_DG_CASE(1, 0, 1, 0)
        EPIC_DG_CASE(1, 0, 0, 1)
        EPIC_DG_CASE(1, 1, 0, 0)
        EPIC_DG_CASE(1, 1, 1, 0)
        EPIC_DG_CASE(1, 1, 0, 1)
        EPIC_DG_CASE(2, 0, 0, 0)
        EPIC_DG_CASE(2, 0, 1, 0)
        EPIC_DG_CASE(2, 0, 0, 1)
        EPIC_DG_CASE(2, 1, 0, 0)
        EPIC_DG_CASE(2, 1, 1, 0)
        EPIC_DG_CASE(2, 1, 0, 1)
#undef EPIC_DG_CASE
        default:
            return cudaErrorInvalidValue;
    }
}

}  // namespace epic
