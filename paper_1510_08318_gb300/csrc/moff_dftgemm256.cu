// MOFF imaging with the spatial transform as a dense DFT on the 5th-generation tensor cores for
// N_p = 256 (N_g = 128) (Eq. "dirty-image-MOFF"; the transform of Sec. 3 "Spatial Fourier
// Transform" written as two matrix products):
//
//   X(ky, x)  = sum_y  W[ky][y] E(y, x)          stage 1, M = 128 (ky of this CTA's half), K = 128 (y)
//   F(ky, kx) = sum_x  X(ky, x) W[kx][x]         stage 2, M = 128 (ky), K = 128 (x), N = 128 kx per pass
//   I(ky, kx) += |F|^2
//
// with W[k][n] = exp(+2 pi i n k / 256) for k < 256, n < 128 (the zero-padded half of every input
// pruned).  Operands are FP16 hi + lo pairs and each real product is hi*hi + hi*lo + lo*hi with
// FP32 accumulation in tensor memory, as in the N_p = 128 form.
//
// Sizing.  Both stages' accumulators for all 256 image rows do not fit one SM's 512 TMEM columns,
// and the operands (W: 256 KB of hi/lo tables, E: 128 KB) not its shared memory.  So an image is
// split by rows: two CTAs (on two SMs) each compute the 128 rows ky of one half for the same
// image, and each grids the whole image (E is the B operand of both halves' stage 1; gridding is
// a minor cost beside 288 MMAs per half image).  The W tables stream from global memory (L2)
// through a ring of 16 KB chunks filled by the bulk copy engine: a chunk is one K step (16) of
// the four tables (re hi, re lo, im hi, im lo) for 128 rows, the A operand of stage 1 and the B
// operand of stage 2 alike (W is symmetric in its use: rows are ky in stage 1 and kx in stage 2).
// Per image a CTA consumes 24 chunks: stage 1 (its half's rows, 8 K steps), then stage 2 in two
// passes of 128 kx (8 K steps each).  A pair of CTAs working on one image would be a
// cta_group::2 MMA; it saves nothing here, because both halves need the whole of E and their own
// W rows either way, so the two CTAs stay independent and never wait on each other.
//
// TMEM columns (all 512, one CTA per SM):
//   [0, 256)    stage-1 accumulator X (re 0..127, im 128..255), FP32; split in place into the
//               stage-2 A operand: per 16 columns (16 x values) 8 columns of hi pairs then 8 of
//               lo pairs
//   [256, 512)  stage-2 accumulator of one pass (re F 256..383, im F 384..511), FP32
//
// Pipeline of image j.  16 warps (so that a scheduler partition holds at most four and a thread
// may have 128 registers: the 64 FP32 partial sums below live in registers); warps 0 .. 14 grid
// and decode, the first thread of warp 15 issues every MMA and bulk copy, and all 16 warps take
// the tensor-memory passes (split, |F|^2), warp 15 after its issuing:
//   all:      split X(j) (after stage 1 of j) | barrier
//   issuer:   stage-2 pass 0 of j
//   warps 0-14: grid image j+1 into E (E is free once stage 1 of j is done), decode image j+2
//   all:      |F|^2 of pass 0 (after it) | barrier
//   issuer:   stage-2 pass 1 of j, wait for it, stage 1 of j+1
//   all:      |F|^2 of pass 1 (after it), under stage 1 of j+1
// so the tensor pipe idles only during the split and the first pass's epilogue.  Each CTA keeps
// its 128 x 256 pixels' FP32 partial sums in registers (64 per thread) and adds them to the FP64
// accumulator with atomics when the (channel, pol) changes, every flush_every samples and at the
// end.
//
// Gridding gathers cell pairs (x, y), (x, y + 1) from the slot tables of the 128 x 128 grid (256
// slots of 32 pairs over 15 warps of 18 positions each; each cell's entries in the builder's
// fixed order; a position no slot took has base -1 and is skipped), read through L1 (the
// operand buffers leave no room for them in shared memory).  The per-image scale is a
// power of two that keeps |E| below 256, so |X| stays below 2^15 and its FP16 split in range.
// Every wait is bounded (the pipeline's by the plan's try count); on a timeout the CTA sets the
// image-timeout bit of the plan's status word, writes NaN into its accumulator block, waits with
// the full limit for the copies and products in flight and stops.
//
// FP16 gridding (LPG, EPIC_XFORM_DFTGEMM_FP16_GRID): the gridding operands are FP16 -- each
// weight and each calibrated voltage is rounded to FP16, so every product is exact in FP32 --
// and the cells' sums stay FP32; the transform keeps its hi + lo operands.  The voltages are
// held as FP16 pairs (4 bytes per antenna instead of 8) and, for real weights, each gather entry
// is one 32-bit word (FP16 weight in the high half, antenna in the low half) instead of an FP32
// weight and a 16-bit antenna in two arrays: one 4-byte read per step instead of two reads of
// 6 bytes.  Complex weights are read from the FP32 tables and rounded as they are read.
#include <cuda_fp16.h>
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <type_traits>
#include <vector>
#include "moff_common.cuh"
#include "tcgen05.cuh"

namespace epic {
namespace dg2 {
using namespace tc;

constexpr int NP = 256, NG = 128;
constexpr int NTH = 512;          // 16 warps: every warp takes part in the tensor-memory passes
constexpr int NGW = kDg256GridWarps;   // warps 0 .. 14 grid and decode
constexpr int NGT = 32 * NGW;     // gridding / decoding threads
constexpr int ISSUER = NGT;       // first thread of warp 15 issues every MMA and bulk copy
constexpr int VPT = 2;            // antennas per decoding thread whose voltages are prefetched
constexpr int KS = 16;                       // K per chunk (one MMA K step)
constexpr int NKS = NG / KS;                 // 8 K steps per stage pass
constexpr int CTAB = 128 * KS;               // halves per table in a chunk (4 KB)
constexpr int CHUNK = 4 * CTAB;              // halves per chunk (16 KB)
constexpr uint32_t CHUNK_BYTES = CHUNK * 2;
enum { C_RHI, C_RLO, C_IHI, C_ILO };         // tables of a chunk
constexpr int RING = 3;                      // chunks in flight
constexpr int PER_IMAGE = 3 * NKS;           // chunks per image: stage 1, stage 2 pass 0, pass 1
constexpr int ETAB = NG * NG;                // halves per E^T table (32 KB)
enum { E_RHI, E_RLO, E_IHI, E_ILO, N_ETAB };
constexpr int NSLOT = NG * NG / 64;          // slots of 32 cell pairs
constexpr int SPW = (NSLOT + NGW - 1) / NGW; // slot positions per gridding warp
constexpr uint32_t kNegA = 1u << 13;

__device__ __forceinline__ void split2(float a, float b, uint32_t& hi, uint32_t& lo) {
    const __half2 h = __floats2half2_rn(a, b);
    const float2 f = __half22float2(h);
    const __half2 l = __floats2half2_rn(a - f.x, b - f.y);
    hi = *reinterpret_cast<const uint32_t*>(&h);
    lo = *reinterpret_cast<const uint32_t*>(&l);
}

constexpr size_t smem_fixed() {
    return sizeof(__half) * ((size_t)N_ETAB * ETAB + (size_t)RING * CHUNK) + 128;
}
constexpr size_t ant_bytes() { return 28; }   // two voltage buffers, gains, power

__device__ __forceinline__ float round_h(float x) { return __half2float(__float2half_rn(x)); }
__device__ __forceinline__ float2 half2_bits_to_float2(uint32_t u) {
    return __half22float2(*reinterpret_cast<const __half2*>(&u));
}

template <int VDT, bool LPG>
__global__ void __launch_bounds__(NTH, 1) moff_dftgemm256_kernel(const FwdArgs a, const __half* __restrict__ wtab,
                                                                 const DgGather g) {
    using VT = typename Volt<VDT>::T;
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    __half* sE = reinterpret_cast<__half*>(smem_raw);                     // [N_ETAB][ETAB]
    __half* sW = sE + N_ETAB * ETAB;                                      // [RING][CHUNK]
    uint64_t* mbar = reinterpret_cast<uint64_t*>(sW + RING * CHUNK);      // full[RING], empty[RING], s1, s2, drain
    uint32_t* tslot = reinterpret_cast<uint32_t*>(mbar + 2 * RING + 3);
    unsigned int* vmax = reinterpret_cast<unsigned int*>(tslot + 2);      // [4]
    const int A = a.n_ant, T = a.n_time;
    float2* VB = reinterpret_cast<float2*>(smem_raw + smem_fixed());      // [2][A]
    uint32_t* VBh = reinterpret_cast<uint32_t*>(VB);                      // LPG: [2][A] FP16 pairs
    float2* GN = VB + 2 * A;
    float* PW = reinterpret_cast<float*>(GN + A);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const bool gw = warp < NGW;             // gridding / decoding warp
    const int h = blockIdx.x & 1;           // row half of every image this CTA computes
    const VT* V = static_cast<const VT*>(a.volt);

    for (int aa = tid; aa < A; aa += NTH) PW[aa] = 0.f;
    auto full = [&](int s) { return smem_u32(&mbar[s]); };
    auto empty = [&](int s) { return smem_u32(&mbar[RING + s]); };
    const uint32_t mb1 = smem_u32(&mbar[2 * RING]), mb2 = smem_u32(&mbar[2 * RING + 1]),
                   mbd = smem_u32(&mbar[2 * RING + 2]);
    if (tid == 0) {
        for (int s = 0; s < 2 * RING + 3; ++s) mbar_init(smem_u32(&mbar[s]), 1);
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
    const uint32_t tX = tmem, tF = tmem + 256;
    const uint32_t lane_base = (uint32_t)(32 * (warp & 3)) << 16;
    const int qg = warp >> 2;                 // column group of this warp in the TMEM passes
    const int kyl = 32 * (warp & 3) + lane;   // TMEM lane = row within the half
    const uint64_t dE0 = sdesc(smem_u32(sE), 2048);
    constexpr int kEStep = 2 * ETAB / 16;     // descriptor start step per E^T table
    constexpr int kCStep = 2 * CTAB / 16;     // ... per table of a chunk

    long long beg_l, end_l;
    work_range(a.n_items, blockIdx.x >> 1, gridDim.x >> 1, beg_l, end_l);
    const int beg = (int)beg_l, n = (int)(end_l - beg_l);
    const int total = PER_IMAGE * n;          // chunks this CTA consumes

    float acc[64];
#pragma unroll
    for (int j = 0; j < 64; ++j) acc[j] = 0.f;

    auto vrow = [&](int cp, int t) -> const VT* { return V + ((long long)t * a.n_cp + cp) * (long long)A; };
    VT raw[VPT];
    auto prefetch = [&](int item) {
        const int cp = item / T, t = item - cp * T;
        const VT* base = vrow(cp, t);
#pragma unroll
        for (int q = 0; q < VPT; ++q)
            if (tid + NGT * q < A) raw[q] = __ldg(base + tid + NGT * q);
    };
    auto load_gains = [&](int cp) {
        for (int aa = tid; aa < A; aa += NGT) GN[aa] = a.gains ? a.gains[(size_t)cp * A + aa] : make_float2(1.f, 0.f);
    };
    // the pair's two CTAs decode the same samples: only the first half adds the antenna power
    auto flush_power = [&](int cp) {
        for (int aa = tid; aa < A; aa += NGT) {
            if (a.power != nullptr && h == 0) atomicAdd(a.power + (size_t)cp * A + aa, (double)PW[aa]);
            PW[aa] = 0.f;
        }
    };
    // calibrated voltage of antenna aa into buffer vb: FP32 pair, or (LPG) rounded to an FP16
    // pair in the same buffer slot's half-size array
    auto store_volt = [&](float2* vb, int aa, float2 vp) {
        if constexpr (LPG) {
            const __half2 hv = __floats2half2_rn(vp.x, vp.y);
            VBh[(vb - VB) + aa] = *reinterpret_cast<const uint32_t*>(&hv);
        } else {
            vb[aa] = vp;
        }
    };
    auto decode = [&](int j) {
        const int item = beg + j, cp = item / T, t = item - cp * T;
        if (j == 0 || (item - 1) / T != cp) {
            if (j > 0) flush_power((item - 1) / T);
            load_gains(cp);
        }
        const VT* base = vrow(cp, t);
        float2* vb = VB + (j & 1) * A;
        float m = 0.f;
#pragma unroll
        for (int q = 0; q < VPT; ++q) {
            const int aa = tid + NGT * q;
            if (aa < A) {
                const float2 vp = cmul(GN[aa], Volt<VDT>::dec(raw[q]));
                store_volt(vb, aa, vp);
                PW[aa] += cnorm(vp);
                m = fmaxf(m, fmaxf(fabsf(vp.x), fabsf(vp.y)));
            }
        }
        for (int aa = tid + NGT * VPT; aa < A; aa += NGT) {
            const float2 vp = cmul(GN[aa], Volt<VDT>::dec(__ldg(base + aa)));
            store_volt(vb, aa, vp);
            PW[aa] += cnorm(vp);
            m = fmaxf(m, fmaxf(fabsf(vp.x), fabsf(vp.y)));
        }
        if (j + 1 < n) prefetch(item + 1);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
        if (lane == 0 && m > 0.f) atomicMax(vmax + (j & 3), __float_as_uint(m));
    };
    // power-of-two exponent s of local image j's operand scale 2^-s, from the bound on |E|
    // (every warp derives it: warp 15 takes part in the epilogue but not in the gridding)
    auto image_exp = [&](int j) -> int {
        const float bound = a.wsum_max * 1.5f * __uint_as_float(vmax[j & 3]);
        int ex = 0;
        if (bound > 0.f) {
            frexpf(bound, &ex);
            ex = max(-100, min(100, ex - 8));    // scaled bound in [128, 256)
        }
        return ex;
    };
    // gridding of local image j into the E^T tables (gridding warps), scaled by 2^-s
    auto grid = [&](int j) {
        const float down = ldexpf(1.f, -image_exp(j));
        const float2* vb = VB + (j & 1) * A;
        const uint32_t* vbh = VBh + (j & 1) * A;
        // weight as the gridding uses it: FP32, or (LPG) rounded to FP16
        auto wt = [&](float w) -> float {
            if constexpr (LPG) return round_h(w);
            else return w;
        };
        // calibrated voltage of an antenna: FP32 pair, or (LPG) the FP16 pair widened exactly
        auto volt_of = [&](int an) -> float2 {
            if constexpr (LPG) return half2_bits_to_float2(vbh[an]);
            else return vb[an];
        };
        // A warp walks its slots one after another, and each step's entry and voltage reads
        // depend on the table reads before them; so the next slot's header is loaded while this
        // slot is walked, and U = 2 steps are taken per iteration, their table reads issued
        // before their voltage reads and products (each lane still sums its entries in table
        // order: the sums are those of one step per iteration, bit for bit).
        constexpr int U = 2;
        int slot = warp * SPW;
        int2 lw_next = __ldg(g.lane + slot * 32 + lane);
        int base_next = __ldg(g.base + slot);
#pragma unroll 1
        for (int jj = 0; jj < SPW; ++jj, ++slot) {
            const int2 lw = lw_next;
            const int sbase = base_next;
            if (jj + 1 < SPW) {
                lw_next = __ldg(g.lane + (slot + 1) * 32 + lane);
                base_next = __ldg(g.base + slot + 1);
            }
            if (sbase < 0) continue;   // a position no slot took (uniform across the warp)
            const int c0 = lw.x & 0xffff, cnt = (int)((unsigned)lw.x >> 16);
            const int kmax = __shfl_sync(0xffffffffu, cnt, 0);   // lane 0 has the longest list
            int e = sbase + lane;
            float2 s0 = make_float2(0.f, 0.f), s1 = make_float2(0.f, 0.f);
            // cw_tag: complex weights; pk_tag: packed FP16 weight | antenna entries (LPG, real)
            auto walk = [&](auto cw_tag, auto pk_tag) {
                constexpr bool CW = decltype(cw_tag)::value, PK = decltype(pk_tag)::value;
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
                            if constexpr (PK) {
                                const uint32_t pk = __ldg(g.wpk + ek[u]);
                                w[u].x = __half2float(__ushort_as_half((unsigned short)(pk >> 16)));
                                an[u] = (int)(pk & 0xffffu);
                            } else {
                                w[u].x = wt(__ldg(g.wre + ek[u]));
                                if constexpr (CW) w[u].y = wt(__ldg(g.wim + ek[u]));
                                an[u] = __ldg(g.ant + ek[u]);
                            }
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
                            // both cells take the entry, one with weight 0 (adds an exact 0)
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
            if (g.wim) walk(std::true_type{}, std::false_type{});
            else if constexpr (LPG) walk(std::false_type{}, std::true_type{});
            else walk(std::false_type{}, std::false_type{});
            uint32_t rh, rl, ih, il;
            split2(s0.x * down, s1.x * down, rh, rl);
            split2(s0.y * down, s1.y * down, ih, il);
            const int off = lw.y;
            *reinterpret_cast<uint32_t*>(sE + E_RHI * ETAB + off) = rh;
            *reinterpret_cast<uint32_t*>(sE + E_RLO * ETAB + off) = rl;
            *reinterpret_cast<uint32_t*>(sE + E_IHI * ETAB + off) = ih;
            *reinterpret_cast<uint32_t*>(sE + E_ILO * ETAB + off) = il;
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    };
    auto flush_acc = [&](int cp) {
        double* dst = a.accum + (size_t)cp * NP * NP;
        const int iy = (128 * h + kyl + NP / 2) & (NP - 1);
#pragma unroll
        for (int p = 0; p < 2; ++p)
#pragma unroll
            for (int j = 0; j < 32; ++j) {
                const int ix = (128 * p + 32 * qg + j + NP / 2) & (NP - 1);
                atomicAdd(dst + iy * NP + ix, (double)acc[32 * p + j]);
                acc[32 * p + j] = 0.f;
            }
    };
    // |F|^2 of stage-2 pass p (every warp: lane quarter warp & 3, columns 32 qg .. + 32)
    auto epilogue = [&](int p, float scale) {
#pragma unroll
        for (int c = 0; c < 32; c += 8) {
            float fr[8], fi[8];
            tld<8>(tF + lane_base + 32 * qg + c, fr);
            tld<8>(tF + 128 + lane_base + 32 * qg + c, fi);
            tld_wait();
#pragma unroll
            for (int u = 0; u < 8; ++u)
                acc[32 * p + c + u] = fmaf(fmaf(fr[u], fr[u], fi[u] * fi[u]), scale, acc[32 * p + c + u]);
        }
    };
    // X -> the stage-2 A operand in place: warp's columns 64 qg .. + 64 (re for qg < 2, im else)
    auto split = [&]() {
#pragma unroll 1
        for (int c = 0; c < 64; c += 16) {
            const uint32_t col = tX + lane_base + 64 * qg + c;
            float xv[16];
            tld<16>(col, xv);
            tld_wait();
            uint32_t ph[8], pl[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) split2(xv[2 * u], xv[2 * u + 1], ph[u], pl[u]);
            tst8(col, ph);
            tst8(col + 8, pl);
        }
        tst_wait();
    };

    // ---- issuer: bulk copies of W chunks and the MMAs ----
    int loaded = 0, consumed = 0;             // chunks copied / whose copy was waited for
    auto load = [&](int c) {                  // chunk c into ring slot c % RING
        const int r = c % PER_IMAGE, rb = r < NKS ? h : (r < 2 * NKS ? 0 : 1), ks = r % NKS;
        const int s = c % RING;
        mbar_expect_tx(full(s), CHUNK_BYTES);
        bulk_g2s(smem_u32(sW + s * CHUNK), wtab + (size_t)(rb * NKS + ks) * CHUNK, CHUNK_BYTES, full(s));
        ++loaded;
    };
    // MMAs of chunk c; false if a wait ran out
    auto issue_chunk = [&](int c) -> bool {
        const int r = c % PER_IMAGE, ks = r % NKS, s = c % RING;
        if (!mbar_wait(full(s), (c / RING) & 1, a.wait_tries)) return false;
        ++consumed;
        fence_after();
        const uint64_t dC = sdesc(smem_u32(sW + s * CHUNK), 256);
        constexpr uint32_t id = idesc(128);
        const uint32_t acc0 = ks != 0;
        if (r < NKS) {
            // stage 1: Re X += Re W Re E - Im W Im E, Im X += Re W Im E + Im W Re E
            const uint64_t dE = dE0 + (uint64_t)(16 * ks);
            constexpr int ta[6] = {C_RHI, C_RHI, C_RLO, C_IHI, C_IHI, C_ILO};
            constexpr int bre[6] = {E_RHI, E_RLO, E_RHI, E_IHI, E_ILO, E_IHI};
            constexpr int bim[6] = {E_IHI, E_ILO, E_IHI, E_RHI, E_RLO, E_RHI};
#pragma unroll
            for (int q = 0; q < 6; ++q) {
                const uint64_t dA = dC + (uint64_t)(ta[q] * kCStep);
                mma_ss(tX, dA, dE + (uint64_t)(bre[q] * kEStep), q < 3 ? id : id | kNegA, acc0 | (q != 0));
                mma_ss(tX + 128, dA, dE + (uint64_t)(bim[q] * kEStep), id, acc0 | (q != 0));
            }
        } else {
            // stage 2: Re F += Re X Re W - Im X Im W, Im F += Re X Im W + Im X Re W
            const uint32_t xre = tX + 16 * ks, xim = tX + 128 + 16 * ks;
            const uint32_t ar[6] = {xre, xre, xre + 8, xim, xim, xim + 8};
            constexpr int bre[6] = {C_RHI, C_RLO, C_RHI, C_IHI, C_ILO, C_IHI};
            constexpr int bim[6] = {C_IHI, C_ILO, C_IHI, C_RHI, C_RLO, C_RHI};
#pragma unroll
            for (int q = 0; q < 6; ++q) {
                mma_ts(tF, ar[q], dC + (uint64_t)(bre[q] * kCStep), q < 3 ? id : id | kNegA, acc0 | (q != 0));
                mma_ts(tF + 128, ar[q], dC + (uint64_t)(bim[q] * kCStep), id, acc0 | (q != 0));
            }
        }
        commit(empty(s));
        // refill the slot of chunk c - 1 once its MMAs are done (chunk c's are queued behind them)
        if (c >= 1 && c - 1 + RING < total) {
            if (!mbar_wait(empty((c - 1) % RING), ((c - 1) / RING) & 1, a.wait_tries)) return false;
            load(c - 1 + RING);
        }
        return true;
    };
    // the 8 chunks of one stage pass of local image j: stage 0 = stage 1, 1 / 2 = stage-2 passes
    auto issue_pass = [&](int j, int stage) -> bool {
        for (int k = 0; k < NKS; ++k)
            if (!issue_chunk(PER_IMAGE * j + NKS * stage + k)) return false;
        commit(stage == 0 ? mb1 : mb2);
        return true;
    };

    bool failed = false;
    int since = 0;
    float sc_cur = 1.f, sc_next = 1.f;
    if (n > 0) {
        if (tid == ISSUER)
            for (int c = 0; c < RING && c < total; ++c) load(c);
        if (gw) {
            prefetch(beg);
            decode(0);
        }
        __syncthreads();
        sc_cur = ldexpf(1.f, 2 * image_exp(0));   // |F|^2 scale 4^s
        if (gw) {
            grid(0);
            if (n > 1) decode(1);
        }
        fence_before();
        __syncthreads();
        if (tid == ISSUER) {
            fence_after();
            failed = !issue_pass(0, 0);
        }
        if (tid == 0) vmax[0] = 0u;
    }
    // Warp 15's first thread issues while the rest of its warp waits at __syncwarp; then the whole
    // warp takes its share of the (warp-collective) tensor-memory passes like every other warp.
    // A wait that runs out sets `failed` for the warp, then for the CTA at the next barrier.
    for (int j = 0; j < n; ++j) {
        // stage 1 of j done -> split X(j) into the stage-2 A operand
        failed = __any_sync(0xffffffffu, failed || !mbar_wait(mb1, j & 1, a.wait_tries)) != 0;
        fence_after();
        if (!failed) split();
        fence_before();
        failed = __syncthreads_or(failed) != 0;
        if (failed) break;
        if (tid == ISSUER) {
            fence_after();
            failed = !issue_pass(j, 1);
        }
        __syncwarp();
        // grid image j + 1 (E is free: stage 1 of j is done), decode j + 2, epilogue of pass 0
        if (j + 1 < n) sc_next = ldexpf(1.f, 2 * image_exp(j + 1));
        if (gw) {
            if (j + 1 < n) grid(j + 1);
            if (j + 2 < n) decode(j + 2);
        }
        failed = __any_sync(0xffffffffu, failed || !mbar_wait(mb2, 0, a.wait_tries)) != 0;
        fence_after();
        if (!failed) epilogue(0, sc_cur);
        fence_before();
        failed = __syncthreads_or(failed) != 0;
        if (failed) break;
        if (tid == 0) vmax[(j + 1) & 3] = 0u;   // read by the gridding of image j + 1, done
        if (tid == ISSUER) {
            fence_after();
            failed = !issue_pass(j, 2);
            // stage 1 of j + 1 overwrites the columns pass 1 reads: wait for pass 1 first
            if (!failed && j + 1 < n) {
                failed = !mbar_wait(mb2, 1, a.wait_tries);
                fence_after();
                if (!failed) failed = !issue_pass(j + 1, 0);
            }
        }
        __syncwarp();
        failed = __any_sync(0xffffffffu, failed || !mbar_wait(mb2, 1, a.wait_tries)) != 0;
        fence_after();
        if (!failed) {
            epilogue(1, sc_cur);
            ++since;
            const int item = beg + j, cp = item / T;
            if (j + 1 == n || (item + 1) / T != cp || since == a.flush_every) {
                flush_acc(cp);
                since = 0;
            }
        }
        sc_cur = sc_next;
    }
    if (!failed && n > 0 && gw) flush_power((beg + n - 1) / T);
    failed = __syncthreads_or(failed) != 0;
    if (failed) {
        // report, mark this CTA's first block, then drain: every bulk copy still in flight (they
        // write this CTA's shared memory) and every MMA issued (a commit after the last one)
        if (n > 0 && tid == 0) {
            if (a.status) atomicOr(a.status, kStatusImageTimeout);
            a.accum[(size_t)(beg / T) * NP * NP + (size_t)((128 * h + NP / 2) & (NP - 1)) * NP] =
                __longlong_as_double(0x7ff8000000000000LL);
        }
        if (tid == ISSUER) {
            for (int c = consumed; c < loaded; ++c) mbar_wait(full(c % RING), (c / RING) & 1);
            commit(mbd);
        }
        mbar_wait(mbd, 0);
    }
    fence_before();
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(tmem), "r"(512) : "memory");
}

}  // namespace dg2

size_t dftgemm256_smem_bytes(int n_ant) { return dg2::smem_fixed() + (size_t)n_ant * dg2::ant_bytes(); }

// W operand chunks for N_p = 256: for row block rb (rows k = 128 rb ..) and K step ks (columns
// n = 16 ks ..), four [128][16] K-major FP16 tables (re hi, re lo, im hi, im lo) of
// W[k][n] = exp(+2 pi i n k / 256), computed in float64; 16 chunks of 16 KB, chunk rb * 8 + ks.
void dftgemm256_tables(std::vector<uint16_t>& out) {
    using namespace dg2;
    out.assign((size_t)2 * NKS * CHUNK, 0);
    for (int rb = 0; rb < 2; ++rb)
        for (int ks = 0; ks < NKS; ++ks) {
            uint16_t* ch = out.data() + (size_t)(rb * NKS + ks) * CHUNK;
            for (int r = 0; r < 128; ++r)
                for (int kk = 0; kk < KS; ++kk) {
                    const int k = 128 * rb + r, nn = KS * ks + kk;
                    const double ang = 2.0 * 3.14159265358979323846 * double((nn * k) % NP) / double(NP);
                    const double vals[2] = {std::cos(ang), std::sin(ang)};
                    const int thi[2] = {C_RHI, C_IHI}, tlo[2] = {C_RLO, C_ILO};
                    for (int c = 0; c < 2; ++c) {
                        const __half hi = __double2half(vals[c]);
                        const __half lo = __double2half(vals[c] - (double)__half2float(hi));
                        ch[(size_t)thi[c] * CTAB + koff(r, kk, KS)] = __half_as_ushort(hi);
                        ch[(size_t)tlo[c] * CTAB + koff(r, kk, KS)] = __half_as_ushort(lo);
                    }
                }
        }
}

cudaError_t launch_dftgemm256(int vdt, const FwdArgs& a, const void* wtab, const DgGather& g, int n_sm,
                              cudaStream_t st, bool fp16_grid) {
    // the FP16-gridding form reads real weights from the packed entries
    if (fp16_grid && !g.wim && !g.wpk) return cudaErrorInvalidValue;
    const __half* w = static_cast<const __half*>(wtab);
    const size_t smem = dftgemm256_smem_bytes(a.n_ant);
    long long pairs = n_sm / 2;
    if (pairs > a.n_items) pairs = a.n_items;
    const unsigned grid = (unsigned)(2 * pairs);
    cudaError_t e;
    switch (vdt) {
#define EPIC_DG2_LAUNCH(V, LPG)                                                                      \
    e = ensure_smem<dg2::moff_dftgemm256_kernel<V, LPG>>(smem);                                      \
    if (e != cudaSuccess) return e;                                                                  \
    if (grid > 0) dg2::moff_dftgemm256_kernel<V, LPG><<<grid, dg2::NTH, smem, st>>>(a, w, g);        \
    return cudaGetLastError();
#define EPIC_DG2_CASE(V)                                                                             \
    case V:                                                                                          \
        if (fp16_grid) {                                                                             \
            EPIC_DG2_LAUNCH(V, true)                                                                 \
        } else {                                                                                     \
            EPIC_DG2_LAUNCH(V, false)                                                                \
        }
        EPIC_DG2_CASE(0)
        EPIC_DG2_CASE(1)
        EPIC_DG2_CASE(2)
#undef EPIC_DG2_CASE
#undef EPIC_DG2_LAUNCH
        default:
            return cudaErrorInvalidValue;
    }
}

}  // namespace epic
