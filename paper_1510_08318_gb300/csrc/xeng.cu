// X-engine of the FX route (Sec. 3 "FX" flow; Eq. "cc-vis"): the visibilities
//   V_ab = g_a conj(g_b) (1/T) sum_t V_a(t) conj(V_b(t))
// of every antenna pair of every (channel, pol), as a Hermitian product E E^H on the
// 5th-generation tensor cores.
//
// Per (channel, pol) the voltages form E [A x T] complex; with R = Re E and I = Im E
//   Re V = R_a R_b^T + I_a I_b^T,   Im V = I_a R_b^T - R_a I_b^T   (summed over t),
// four real products with K = T.  4+4-bit and FP16 voltages are exact in FP16, and each product
// (at most 64 in magnitude for 4+4-bit) is accumulated in FP32 exactly while the sums stay below
// 2^24, so the raw sums are exact.
//
// Work unit: a 128 x 128 block (antenna rows a in block ab, columns b in block bb, bb >= ab:
// the upper block triangle, the lower one follows by Hermitian symmetry) of one (channel,
// pol); one persistent CTA per SM takes a contiguous range of units, K walked in chunks of 32
// samples.  A chunk's operands are K-major FP16 planes: the B tile [R_b; I_b; -R_b] (384 rows)
// and the A tile [R_a; I_a] (a diagonal unit takes its A planes from the B tile), so that two
// MMAs with N = 256 per 16 samples give D = R_a [R_b; I_b]^T + I_a [I_b; -R_b]^T:
// Re V in columns 0..127 and -Im V in 128..255.  The CTA's warps have three roles, handing work
// over through mbarriers only (no CTA-wide barrier inside the loop):
//   - two sets of 8 decode warps take alternate chunks and convert their voltages (loaded into
//     registers two of the set's chunks ahead) into one stage of a 5-stage ring; each warp fences
//     its stores for the tensor cores and arrives on the stage's full barrier, and refills a
//     stage after the MMAs that read it have completed (the stage's empty barrier, signalled by
//     tcgen05.commit);
//   - one thread of the MMA warp issues the 4 MMAs (M = 128, N = 256, K = 16) of a chunk into one
//     of two TMEM accumulator buffers (all 512 columns), commits each chunk to its stage's empty
//     barrier and a unit's last chunk to the buffer's full barrier;
//   - 4 epilogue warps (one per TMEM lane quarter) read a finished buffer (tcgen05.ld), scale
//     by g_a conj(g_b) / T, write the block (16-byte stores along rows) and, off the diagonal,
//     its mirrored conjugate, then release the buffer, while the next unit fills the other one.
// Every wait is bounded by the plan's try count and taken by a whole warp; on a timeout the role
// stops, the CTA sets the correlator-timeout bit of the plan's status word and writes NaN into
// its first output element; the MMA warp waits (full limit) for the MMAs it issued before the
// tensor memory is released.
//
// WIDE (4+4-bit voltages, A a multiple of 4, 4-byte aligned input): a thread loads 4 antennas
// of each of its 8 samples with 4-byte loads (a warp reads whole 128-byte rows), transposes the
// 4 x 4 byte blocks with byte permutes and converts each 4 samples of an antenna with two
// permute + packed-subtraction pairs per plane.  Other voltages are read one by one.
#include <cuda_fp16.h>
#include <cstdint>
#include "moff_common.cuh"
#include "tcgen05.cuh"

namespace epic {
namespace xe {
using namespace tc;

constexpr int NDS = 3;                      // decode warp sets, taking alternate chunks
constexpr int NDW = 8 * NDS;                // decode warps (a set's tile mappings take 256 threads)
constexpr int NEW = 4;                      // epilogue warps, one per TMEM lane quarter
constexpr int MMA_WARP = NDW;               // the warp whose first thread issues the MMAs
constexpr int NT = 32 * (NDW + 1 + NEW);    // one CTA per SM
constexpr int TC = 32;                      // samples per K chunk (K = 32: one real plane per operand row)
// K-major FP16 planes without swizzle: 8 x 8 core matrices of 128 bytes, a row group of 8 rows
// holding the chunk's 4 core matrices along K
constexpr int kRowGroupBytes = 4 * 128;
constexpr int kPlaneBytes = 16 * kRowGroupBytes;       // 128 rows x 32 samples (8 KB)
constexpr int kBTileBytes = 3 * kPlaneBytes;           // [Re_b; Im_b; -Re_b]: 384 rows
constexpr int kATileBytes = 2 * kPlaneBytes;           // [Re_a; Im_a]
constexpr int kStageBytes = kBTileBytes + kATileBytes; // 40 KB
constexpr int NSTAGE = 5;
// mbarriers: stage full [NSTAGE], stage empty [NSTAGE], accumulator full [2], accumulator
// empty [2], drain
constexpr int N_MBAR = 2 * NSTAGE + 5;

constexpr size_t smem_bytes() { return (size_t)NSTAGE * kStageBytes + 8 * N_MBAR + 16; }

// One voltage as an FP16 (re, im) pair (half2 bits).  FP16 input is already the pair.  A
// 4+4-bit byte holds two 4-bit two's-complement values (re in the high nibble); XOR with 8 biases
// each to n + 8 in [0, 15], which placed in the mantissa of 1024 (bits 0x6400 | (n + 8)) is
// exactly 1032 + n, so one packed subtraction of 1032 yields both components exactly.
template <int VDT>
__device__ __forceinline__ uint32_t voltage_pair(typename Volt<VDT>::T raw) {
    if constexpr (VDT == 1) {
        return raw;
    } else {
        const uint32_t t = (uint32_t)raw ^ 0x88u;
        const uint32_t u = ((t >> 4) & 0xFu) | ((t & 0xFu) << 16) | 0x64006400u;
        const __half2 h = __hsub2(*reinterpret_cast<const __half2*>(&u), __halves2half2(__ushort_as_half(0x6408),
                                                                                          __ushort_as_half(0x6408)));
        return *reinterpret_cast<const uint32_t*>(&h);
    }
}

// unit -> (cp, row block, column block), column block >= row block (32-bit: the launcher
// checks that the units fit)
__device__ __forceinline__ void unit_coords(int u, int nab, int& cp, int& ab, int& bb) {
    const int upc = nab * (nab + 1) / 2;
    cp = u / upc;
    int r = u - cp * upc;
    ab = 0;
    while (r >= nab - ab) {
        r -= nab - ab;
        ++ab;
    }
    bb = ab + r;
}

template <int VDT, bool WIDE>
__global__ void __launch_bounds__(NT, 1) xeng_kernel(const XengArgs a) {
    static_assert(!WIDE || VDT == 2, "the wide loads are for 4+4-bit voltages");
    using VT = typename Volt<VDT>::T;
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char* sT = smem_raw;                                               // [NSTAGE] stages
    uint64_t* mbar = reinterpret_cast<uint64_t*>(sT + (size_t)NSTAGE * kStageBytes);   // [N_MBAR]
    uint32_t* tslot = reinterpret_cast<uint32_t*>(mbar + N_MBAR);
    int* s_fail = reinterpret_cast<int*>(tslot + 1);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int A = a.n_ant, T = a.n_time, CP = a.n_cp;
    const int nab = (A + 127) / 128;
    const int n_units = CP * (nab * (nab + 1) / 2);
    const int n_chunks = (T + TC - 1) / TC;
    const VT* V = static_cast<const VT*>(a.volt);
    auto mb_full = [&](int s) { return smem_u32(&mbar[s]); };
    auto mb_empty = [&](int s) { return smem_u32(&mbar[NSTAGE + s]); };
    auto mb_accf = [&](int b) { return smem_u32(&mbar[2 * NSTAGE + b]); };
    auto mb_acce = [&](int b) { return smem_u32(&mbar[2 * NSTAGE + 2 + b]); };
    const uint32_t mb_drain = smem_u32(&mbar[2 * NSTAGE + 4]);
    // a bounded wait taken by a whole warp: the warp goes on only if every lane saw the phase
    auto warp_wait = [&](uint32_t mb, int parity) -> bool {
        return __all_sync(0xffffffffu, mbar_wait(mb, (uint32_t)parity, a.wait_tries)) != 0;
    };

    if (tid == 0) {
        for (int s = 0; s < NSTAGE; ++s) {
            mbar_init(mb_full(s), 8);
            mbar_init(mb_empty(s), 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(mb_accf(b), 1);
            mbar_init(mb_acce(b), NEW);
        }
        mbar_init(mb_drain, 1);
        *s_fail = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == MMA_WARP) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     :: "r"(smem_u32(tslot)), "r"(512) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tmem = *tslot;             // accumulator buffer b: columns 256 b (Re), 256 b + 128 (Im)

    long long beg_l, end_l;
    work_range(n_units, blockIdx.x, gridDim.x, beg_l, end_l);
    const int beg = (int)beg_l, end = (int)end_l;

    if (warp < NDW) {
        // ---------------- decode warps: raw voltages -> FP16 operand planes of stage g % NSTAGE ----
        // Set dset decodes the CTA's chunks g = dset, dset + NDS, ...  Within a set, warps 0-3 fill
        // the B tile ([Re; Im; -Re] of the column block) and warps 4-7 the A tile ([Re; Im] of the
        // row block; nothing on a diagonal unit), warp dw taking samples 8 (dw % 4) .. + 7 of the
        // chunk and lane l antennas 4 l .. 4 l + 3 of the block.  The thread's slot i holds antenna
        // 4 l + (i + rot) % 4, rot = (l / 2) % 4, so that the 8 lanes of a quarter-warp write the
        // 16-byte rows of 8 distinct rows mod 8 (all 32 banks) with each 16-byte store.
        const int dw = warp & 7, dset = warp >> 3;
        const bool bside = dw < 4;
        const int so = dw & 3, rot = (lane >> 1) & 3;
        int soff[4];                                   // byte offset in a plane of slot i's row
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int r = 4 * lane + ((i + rot) & 3);
            soff[i] = (r >> 3) * kRowGroupBytes + so * 128 + (r & 7) * 16;
        }
        // (unit, chunk) cursors step NDS chunks at a time; true when the unit changed
        auto advance = [&](int& uu, int& kk, int by) -> bool {
            kk += by;
            bool changed = false;
            while (kk >= n_chunks && uu < end) {
                kk -= n_chunks;
                ++uu;
                changed = true;
            }
            return changed;
        };
        const long long RS = (long long)CP * A;       // sample stride of the voltages
        // slot i's row of the Re, Im (and, B tile, -Re) planes: 8 samples each
        auto put_planes = [&](unsigned char* tile, int i, const uint4& re, const uint4& im, bool neg) {
            *reinterpret_cast<uint4*>(tile + soff[i]) = re;
            *reinterpret_cast<uint4*>(tile + kPlaneBytes + soff[i]) = im;
            if (neg)
                *reinterpret_cast<uint4*>(tile + 2 * kPlaneBytes + soff[i]) =
                    make_uint4(re.x ^ 0x80008000u, re.y ^ 0x80008000u, re.z ^ 0x80008000u, re.w ^ 0x80008000u);
        };
        // the same from the slot's 8 samples as (re, im) FP16 pairs x[s]
        auto put_pairs = [&](unsigned char* tile, int i, const uint32_t (&x)[8], bool neg) {
            const uint4 re = make_uint4(__byte_perm(x[0], x[1], 0x5410), __byte_perm(x[2], x[3], 0x5410),
                                        __byte_perm(x[4], x[5], 0x5410), __byte_perm(x[6], x[7], 0x5410));
            const uint4 im = make_uint4(__byte_perm(x[0], x[1], 0x7632), __byte_perm(x[2], x[3], 0x7632),
                                        __byte_perm(x[4], x[5], 0x7632), __byte_perm(x[6], x[7], 0x7632));
            put_planes(tile, i, re, im, neg);
        };
        // raw words of this thread's 8 samples (fast path: byte i = antenna 4 l + i), two chunks
        uint32_t rw0[8], rw1[8];
        int lu = beg, lkc = 0, lcp = 0, lab = 0, lbb = 0;                       // load cursor
        advance(lu, lkc, dset);
        if (lu < end) unit_coords(lu, nab, lcp, lab, lbb);
        const unsigned char* VB = static_cast<const unsigned char*>(a.volt);
        auto fast_load = [&](uint32_t (&w)[8]) {
#pragma unroll
            for (int s = 0; s < 8; ++s) w[s] = 0;
            if (lu < end && (bside || lab != lbb)) {
                const int col = (bside ? lbb : lab) * 128 + 4 * lane;
                if (col < A) {
                    const unsigned char* base = VB + (long long)lcp * A + col;
                    const int t0 = lkc * TC + 8 * so;
#pragma unroll
                    for (int s = 0; s < 8; ++s)
                        if (t0 + s < T) w[s] = __ldg(reinterpret_cast<const uint32_t*>(base + (long long)(t0 + s) * RS));
                }
            }
            if (advance(lu, lkc, NDS) && lu < end) unit_coords(lu, nab, lcp, lab, lbb);
        };
        // 4+4-bit words (4 samples of one slot) -> FP16 pairs: the biased nibble h = n ^ 8 in
        // [0, 15] placed under the exponent byte 0x64 is exactly 1024 + h, and 1024 + h - 1032 = n
        auto nib_pairs = [](uint32_t N, uint32_t& p01, uint32_t& p23) {
            const __half2 bias = __halves2half2(__ushort_as_half(0x6408), __ushort_as_half(0x6408));
            uint32_t u0 = __byte_perm(N, 0x64646464u, 0x4140), u1 = __byte_perm(N, 0x64646464u, 0x4342);
            const __half2 h0 = __hsub2(*reinterpret_cast<const __half2*>(&u0), bias);
            const __half2 h1 = __hsub2(*reinterpret_cast<const __half2*>(&u1), bias);
            p01 = *reinterpret_cast<const uint32_t*>(&h0);
            p23 = *reinterpret_cast<const uint32_t*>(&h1);
        };
        auto fast_decode = [&](const uint32_t (&w)[8], unsigned char* tile) {
            // rotate each sample's word so that byte i is slot i's antenna, then transpose the two
            // 4 x 4 byte blocks: q[i][h] = samples 4 h .. 4 h + 3 of slot i
            uint32_t x[8], q[4][2];
#pragma unroll
            for (int s = 0; s < 8; ++s) x[s] = __funnelshift_r(w[s], w[s], 8 * rot);
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const uint32_t lo01 = __byte_perm(x[4 * h], x[4 * h + 1], 0x5140);
                const uint32_t hi01 = __byte_perm(x[4 * h], x[4 * h + 1], 0x7362);
                const uint32_t lo23 = __byte_perm(x[4 * h + 2], x[4 * h + 3], 0x5140);
                const uint32_t hi23 = __byte_perm(x[4 * h + 2], x[4 * h + 3], 0x7362);
                q[0][h] = __byte_perm(lo01, lo23, 0x5410);
                q[1][h] = __byte_perm(lo01, lo23, 0x7632);
                q[2][h] = __byte_perm(hi01, hi23, 0x5410);
                q[3][h] = __byte_perm(hi01, hi23, 0x7632);
            }
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                uint4 re, im;
                // re = high nibbles, im = low nibbles, each biased by 8
                const uint32_t H0 = ((q[i][0] >> 4) & 0x0F0F0F0Fu) ^ 0x08080808u, L0 = (q[i][0] & 0x0F0F0F0Fu) ^ 0x08080808u;
                const uint32_t H1 = ((q[i][1] >> 4) & 0x0F0F0F0Fu) ^ 0x08080808u, L1 = (q[i][1] & 0x0F0F0F0Fu) ^ 0x08080808u;
                nib_pairs(H0, re.x, re.y);
                nib_pairs(H1, re.z, re.w);
                nib_pairs(L0, im.x, im.y);
                nib_pairs(L1, im.z, im.w);
                put_planes(tile, i, re, im, bside);
            }
        };
        // any voltage type, any A: slot by slot, voltage by voltage
        auto slow_decode = [&](int cp, int blk, int kc, unsigned char* tile) {
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const int ant = blk * 128 + 4 * lane + ((i + rot) & 3);
                uint32_t x[8];
#pragma unroll
                for (int s = 0; s < 8; ++s) {
                    const int t = kc * TC + 8 * so + s;
                    const VT raw = (ant < A && t < T) ? __ldg(V + (long long)t * RS + (long long)cp * A + ant) : VT(0);
                    x[s] = voltage_pair<VDT>(raw);
                }
                put_pairs(tile, i, x, bside);
            }
        };
        if constexpr (WIDE) {
            fast_load(rw0);
            fast_load(rw1);
        }
        bool failed = false;
        int cu = beg, ckc = 0, ccp = 0, cab = 0, cbb = 0;                       // decode cursor
        advance(cu, ckc, dset);
        if (cu < end) unit_coords(cu, nab, ccp, cab, cbb);
        for (int i = 0; cu < end; ++i) {
            const int g = (cu - beg) * n_chunks + ckc;
            const int s = g % NSTAGE;
            // the stage is free once the MMAs of its previous chunk have completed
            if (g >= NSTAGE && !warp_wait(mb_empty(s), (g / NSTAGE - 1) & 1)) {
                failed = true;
                break;
            }
            const bool diag = cab == cbb;
            unsigned char* st = sT + (size_t)s * kStageBytes;
            if (bside || !diag) {
                unsigned char* tile = bside ? st : st + kBTileBytes;
                if constexpr (WIDE) {
                    if ((i & 1) == 0)
                        fast_decode(rw0, tile);
                    else
                        fast_decode(rw1, tile);
                } else {
                    slow_decode(ccp, bside ? cbb : cab, ckc, tile);
                }
            }
            // this warp's stores, visible to the tensor cores, then its arrival
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            __syncwarp();
            if (lane == 0) mbar_arrive(mb_full(s));
            // the set's chunk after next into the register set just decoded
            if constexpr (WIDE) {
                if ((i & 1) == 0)
                    fast_load(rw0);
                else
                    fast_load(rw1);
            }
            if (advance(cu, ckc, NDS) && cu < end) unit_coords(cu, nab, ccp, cab, cbb);
        }
        if (failed) *s_fail = 1;
    } else if (warp == MMA_WARP) {
        // ---------------- MMA warp: per K step of 16 samples two MMAs (M = 128, N = 256) ----
        //   D += Re_a [Re_b; Im_b]^T,  D += Im_a [Im_b; -Re_b]^T
        // so that D[:, 0:128] = Re_a Re_b + Im_a Im_b = Re V and D[:, 128:256] = Re_a Im_b - Im_a Re_b
        // = -Im V (summed over the samples); on a diagonal unit the A planes are the B tile's.
        bool failed = false;
        int g = 0;                                // chunks whose MMAs this warp issued
        int n = 0;                                // units started
        const uint64_t d0 = sdesc(smem_u32(sT), kRowGroupBytes);
        constexpr uint32_t id = idesc(256);
        for (int u = beg; u < end && !failed; ++u, ++n) {
            int cp, ab, bb;
            unit_coords(u, nab, cp, ab, bb);
            const bool diag = ab == bb;
            const int b = n & 1;
            // accumulator buffer b is free once the epilogue has read the unit before last
            if (n >= 2 && !warp_wait(mb_acce(b), ((n >> 1) - 1) & 1)) {
                failed = true;
                break;
            }
            fence_after();
            const uint32_t tacc = tmem + 256 * b;
            for (int kc = 0; kc < n_chunks; ++kc) {
                const int s = g % NSTAGE;
                if (!warp_wait(mb_full(s), (g / NSTAGE) & 1)) {
                    failed = true;
                    break;
                }
                fence_after();
                if (lane == 0) {
                    // descriptor start fields count 16 bytes
                    const uint64_t dB1 = d0 + (uint64_t)(s * kStageBytes / 16);
                    const uint64_t dB2 = dB1 + kPlaneBytes / 16;
                    const uint64_t dA1 = diag ? dB1 : dB1 + kBTileBytes / 16;
                    const uint64_t dA2 = dA1 + kPlaneBytes / 16;
#pragma unroll
                    for (int j = 0; j < TC / 16; ++j) {
                        mma_ss(tacc, dA1 + 16 * j, dB1 + 16 * j, id, (kc | j) != 0);
                        mma_ss(tacc, dA2 + 16 * j, dB2 + 16 * j, id, 1);
                    }
                    commit(mb_empty(s));
                    if (kc == n_chunks - 1) commit(mb_accf(b));
                }
                __syncwarp();
                ++g;
            }
        }
        // every MMA this warp issued has completed before the tensor memory is released
        if (g > 0) {
            if (lane == 0) commit(mb_drain);
            __syncwarp();
            mbar_wait(mb_drain, 0);
        }
        if (failed) *s_fail = 1;
    } else {
        // ---------------- epilogue warps: D -> V_ab = g_a conj(g_b) D / T (and the mirrored block) ----
        bool failed = false;
        const int q = warp & 3;                   // TMEM lane quarter this warp may read
        const float inv_t = 1.f / float(T);
        // 16-byte row stores when every row starts on a 16-byte boundary
        const bool vec = (A % 2 == 0) && ((reinterpret_cast<uintptr_t>(a.vis) & 15) == 0);
        int n = 0;
        for (int u = beg; u < end; ++u, ++n) {
            const int b = n & 1;
            if (!warp_wait(mb_accf(b), (n >> 1) & 1)) {
                failed = true;
                break;
            }
            fence_after();
            int cp, ab, bb;
            unit_coords(u, nab, cp, ab, bb);
            const bool diag = ab == bb;
            const int a0 = ab * 128, b0 = bb * 128;
            const int aa = a0 + 32 * q + lane;
            const uint32_t tacc = tmem + 256 * b + ((uint32_t)(32 * q) << 16);
            const float2 ga = (aa < A && a.gains) ? a.gains[(size_t)cp * A + aa] : make_float2(1.f, 0.f);
            float2* out = a.vis + (size_t)cp * A * A;
#pragma unroll 1
            for (int c = 0; c < 128; c += 8) {
                float dr[8], di[8];
                tld<8>(tacc + c, dr);
                tld<8>(tacc + 128 + c, di);
                tld_wait();
                if (aa < A) {
                    float2 v[8];
#pragma unroll
                    for (int j = 0; j < 8; ++j) {
                        const int bcol = b0 + c + j;
                        const float2 gb = (a.gains && bcol < A) ? __ldg(a.gains + (size_t)cp * A + bcol)
                                                                : make_float2(1.f, 0.f);
                        const float2 w = cmul(ga, make_float2(gb.x, -gb.y));
                        v[j] = cmul(w, make_float2(dr[j] * inv_t, -di[j] * inv_t));   // D holds -Im V
                    }
                    float2* row = out + (size_t)aa * A + b0 + c;
                    if (vec && b0 + c + 8 <= A) {
                        float4* r4 = reinterpret_cast<float4*>(row);
#pragma unroll
                        for (int j = 0; j < 4; ++j) r4[j] = make_float4(v[2 * j].x, v[2 * j].y, v[2 * j + 1].x, v[2 * j + 1].y);
                    } else {
#pragma unroll
                        for (int j = 0; j < 8; ++j)
                            if (b0 + c + j < A) row[j] = v[j];
                    }
                    if (!diag) {
#pragma unroll
                        for (int j = 0; j < 8; ++j)
                            if (b0 + c + j < A) out[(size_t)(b0 + c + j) * A + aa] = make_float2(v[j].x, -v[j].y);
                    }
                }
            }
            // this warp's reads of buffer b are complete: the MMA warp may overwrite it
            fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(mb_acce(b));
        }
        if (failed) *s_fail = 1;
    }

    fence_before();
    __syncthreads();
    if (tid == 0 && *s_fail && beg < end) {
        if (a.status) atomicOr(a.status, kStatusCorrelateTimeout);
        int cp, ab, bb;
        unit_coords(beg, nab, cp, ab, bb);
        a.vis[(size_t)cp * A * A + (size_t)(ab * 128) * A + bb * 128] =
            make_float2(__int_as_float(0x7fc00000), __int_as_float(0x7fc00000));
    }
    if (warp == MMA_WARP) {
        fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(tmem), "r"(512) : "memory");
    }
}

// ---- the FX route's imaging of an integration's visibilities (Eq. "dirty-image-FX") ----
//   U(d) = sum_{a, b} V_ab B_ab(d),  B_ab(d) = sum_g M[g, a] conj(M[g - d, b]),
//   I(k) = Re sum_d U(d) exp(+2 pi i d.k / N_p)  (image pixel order, k = 0 at the centre).
// Three launches.  (1) The visibilities are transposed to pair-major order with the (channel,
// pol) index innermost, so that the values of one pair for consecutive (channel, pol) are
// contiguous.  (2) The lag planes are gathered from the plan's table of the antenna-pair kernels
// grouped by lag cell (B_ab(d) summed over the mapping entries of a and b once, on the host): a
// warp takes one lag cell for a group of G (channel, pol) planes, its lanes G planes x 32 / G
// entries, so that each entry's visibilities are one coalesced load for the G planes (no
// atomics; a shuffle sum over the entries).  The lag planes (wrapped mod N_p; with
// N_p >= 2 N_g - 1 none alias) go to a scratch array.  (3) One CTA per (channel, pol) takes its
// lag plane into shared memory and transforms it: N_p = S1 x S2 Cooley-Tukey per line (S2-point
// register DFTs, a twiddle, S1-point register DFTs across the line's threads), rows then
// columns, the real part written as the image.

// (1) vis [CP][P2] -> vis_t [P2][CP] through 32 x 32 shared-memory tiles
__global__ void __launch_bounds__(256) fx_transpose_kernel(const float2* __restrict__ vis, int n_cp, long long n_pair,
                                                           float2* __restrict__ vis_t) {
    __shared__ float2 tile[32][33];
    const long long p0 = (long long)blockIdx.x * 32;
    const int c0 = blockIdx.y * 32, tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
#pragma unroll
    for (int j = 0; j < 32; j += 8) {
        const int c = c0 + ty + j;
        const long long p = p0 + tx;
        if (c < n_cp && p < n_pair) tile[ty + j][tx] = __ldg(vis + (size_t)c * n_pair + p);
    }
    __syncthreads();
#pragma unroll
    for (int j = 0; j < 32; j += 8) {
        const long long p = p0 + ty + j;
        const int c = c0 + tx;
        if (c < n_cp && p < n_pair) vis_t[(size_t)p * n_cp + c] = tile[tx][ty + j];
    }
}

// (2) U[cp][d] = sum over the entries of lag cell d of vis_t[off / CP][cp] * B (each entry
// holds the element offset off = pair * CP of its pair's row).  A CTA takes an 8 x 8 tile of lag
// cells (neighbouring cells share most of their pairs, which then stay in L1) for one group of
// G planes; the CTAs of one tile (all groups) are adjacent in launch order so that they share
// the tile's table entries in L2.  A warp takes whole lag cells.  It reads the entries of a cell
// 32 at a time with one coalesced load into its own shared-memory slots (slots past the cell's
// end hold zero weights at offset 0; the next 32 entries are loaded while these are used).
// V4 (an even number of planes, G = 64): lane c takes planes 2c, 2c + 1 of the group with one
// 16-byte load per entry, every lane every entry, 8 entries in flight.  Otherwise lane =
// e * G + c (plane c, G <= 32) takes entries e, e + E, ... of the 32 (E = 32 / G) with 8-byte
// loads, up to 16 in flight, and the sum over a cell's entries ends with a shuffle over e.
constexpr int FXG_NT = 256;

template <int G, bool V4>
__global__ void __launch_bounds__(FXG_NT, V4 ? 2 : 3) fx_gather_kernel(const FxArgs a, int np) {
    static_assert(V4 ? G == 64 : G <= 32, "group width");
    constexpr int E = V4 ? 1 : 32 / G;                                   // entry slots per step
    constexpr int U = V4 ? 8 : ((16 * E <= 32) ? 16 : 32 / E);           // entries per lane in flight
    static_assert(U * E <= 32 && 32 % (U * E) == 0, "steps");
    __shared__ int4 sent[FXG_NT / 32][32];
    const int CP = a.n_cp, n_groups = (CP + G - 1) / G;
    const int tiles_x = np / 8;
    const int tile = blockIdx.x / n_groups, gi = blockIdx.x - tile * n_groups;
    const int ty0 = 8 * (tile / tiles_x), tx0 = 8 * (tile % tiles_x);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int e = V4 ? 0 : lane / G;
    const int cp = V4 ? gi * G + 2 * lane : gi * G + lane % G;          // first plane of the lane
    const bool valid = cp < CP;
    const float2* Vt = a.vis_t + (valid ? cp : 0);
    int4* sw = sent[warp];
    for (int j = warp; j < 64; j += FXG_NT / 32) {
        const int d = (ty0 + (j >> 3)) * np + tx0 + (j & 7);
        const int p0 = __ldg(a.lag_ptr + d), p1 = __ldg(a.lag_ptr + d + 1);
        float2 acc = make_float2(0.f, 0.f), acc1 = make_float2(0.f, 0.f);
        int4 nxt = p0 + lane < p1 ? __ldg(a.lag_ent + p0 + lane) : make_int4(0, 0, 0, 0);
        for (int q0 = p0; q0 < p1; q0 += 32) {
            const int nb = min(32, p1 - q0);
            __syncwarp();
            sw[lane] = nxt;
            __syncwarp();
            nxt = q0 + 32 + lane < p1 ? __ldg(a.lag_ent + q0 + 32 + lane) : make_int4(0, 0, 0, 0);
            for (int k = 0; k < nb; k += U * E) {
                if constexpr (V4) {
                    float4 v[U];
                    float2 w[U];
#pragma unroll
                    for (int u = 0; u < U; ++u) {
                        const int4 en = sw[k + u];
                        w[u] = make_float2(__int_as_float(en.x), __int_as_float(en.y));
                        v[u] = __ldg(reinterpret_cast<const float4*>(Vt + en.z));
                    }
#pragma unroll
                    for (int u = 0; u < U; ++u) {
                        acc.x = fmaf(v[u].x, w[u].x, fmaf(-v[u].y, w[u].y, acc.x));
                        acc.y = fmaf(v[u].x, w[u].y, fmaf(v[u].y, w[u].x, acc.y));
                        acc1.x = fmaf(v[u].z, w[u].x, fmaf(-v[u].w, w[u].y, acc1.x));
                        acc1.y = fmaf(v[u].z, w[u].y, fmaf(v[u].w, w[u].x, acc1.y));
                    }
                } else {
                    float2 v[U], w[U];
#pragma unroll
                    for (int u = 0; u < U; ++u) {
                        const int4 en = sw[k + u * E + e];
                        w[u] = make_float2(__int_as_float(en.x), __int_as_float(en.y));
                        v[u] = __ldg(Vt + en.z);
                    }
#pragma unroll
                    for (int u = 0; u < U; ++u) {
                        acc.x = fmaf(v[u].x, w[u].x, fmaf(-v[u].y, w[u].y, acc.x));
                        acc.y = fmaf(v[u].x, w[u].y, fmaf(v[u].y, w[u].x, acc.y));
                    }
                }
            }
        }
        const size_t npix = (size_t)np * np;
        if constexpr (V4) {
            if (valid) {
                a.u[(size_t)cp * npix + d] = acc;
                a.u[(size_t)(cp + 1) * npix + d] = acc1;
            }
        } else {
#pragma unroll
            for (int o = 16; o >= G; o >>= 1) {
                acc.x += __shfl_xor_sync(0xffffffffu, acc.x, o);
                acc.y += __shfl_xor_sync(0xffffffffu, acc.y, o);
            }
            if (e == 0 && valid) a.u[(size_t)cp * npix + d] = acc;
        }
    }
}

// (3) the transform of one lag plane.  Line of length NP = S1 x S2, n = S1 m + r, k = k1 + S2 k2:
//   X[k1 + S2 k2] = sum_r exp(2 pi i r k2 / S1) [exp(2 pi i r k1 / NP) Y_r[k1]],
//   Y_r[k1] = sum_m x[S1 m + r] exp(2 pi i m k1 / S2).
// Thread (line, r) computes Y_r in registers and stores Y_r[k1] at line position
// r S2 + (k1 xor r) (the xor spreads the S1 threads of a line over distinct banks); thread
// (line, r') then takes k1 = r' + S1 i and does the S1-point DFTs.  Rows are padded to NP + S1
// elements so that the lines a warp touches fall into complementary halves of the banks.  The
// centring (k measured from N_p / 2) is the sign (-1)^(dx + dy) applied to U on loading.
template <int NP>
struct FxDft {
    static constexpr int S1 = NP == 32 ? 4 : 8, S2 = NP / S1, NT = 4 * NP, P = NP + S1;
    static constexpr size_t smem = sizeof(float2) * ((size_t)NP * P + NP);
};

template <int NP>
__global__ void __launch_bounds__(FxDft<NP>::NT) fx_dft_kernel(const float2* __restrict__ u, float* __restrict__ image) {
    using D = FxDft<NP>;
    constexpr int S1 = D::S1, S2 = D::S2, NT = D::NT, P = D::P, MSK = NP - 1;
    static_assert(S1 * S2 == NP && S2 >= S1 && NT % NP == 0, "factorisation");
    extern __shared__ __align__(16) unsigned char fx_smem[];
    float2* L = reinterpret_cast<float2*>(fx_smem);       // [NP][P]
    float2* TW = L + NP * P;                               // [NP] exp(+2 pi i j / NP)
    const int tid = threadIdx.x, cp = blockIdx.x;
    for (int j = tid; j < NP; j += NT) {
        double s, c;
        sincospi(2.0 * j / NP, &s, &c);
        TW[j] = make_float2(float(c), float(s));
    }
    const float2* U = u + (size_t)cp * NP * NP;
    for (int i = tid; i < NP * NP; i += NT) {
        const int dy = i / NP, dx = i % NP;
        float2 v = __ldg(U + i);
        if ((dx + dy) & 1) v = make_float2(-v.x, -v.y);
        L[dy * P + dx] = v;
    }
    __syncthreads();
    // rows: line dy, element dx at L[dy * P + dx]
    {
        constexpr int LPI = NT / S1;                        // lines per iteration
        const int r = tid % S1;
#pragma unroll 1
        for (int l0 = 0; l0 < NP; l0 += LPI) {
            float2* row = L + (l0 + tid / S1) * P;
            float2 x[S2];
#pragma unroll
            for (int m = 0; m < S2; ++m) x[m] = row[S1 * m + r];
            dft<S2, 1>(x);
#pragma unroll
            for (int k1 = 1; k1 < S2; ++k1) x[k1] = cmul(x[k1], TW[(r * k1) & MSK]);
            __syncthreads();
#pragma unroll
            for (int k1 = 0; k1 < S2; ++k1) row[r * S2 + (k1 ^ r)] = x[k1];
        }
        __syncthreads();
#pragma unroll 1
        for (int l0 = 0; l0 < NP; l0 += LPI) {
            float2* row = L + (l0 + tid / S1) * P;
            float2 y[S2 / S1][S1];
#pragma unroll
            for (int i = 0; i < S2 / S1; ++i) {
                const int k1 = r + S1 * i;
#pragma unroll
                for (int q = 0; q < S1; ++q) y[i][q] = row[q * S2 + (k1 ^ q)];
                dft<S1, 1>(y[i]);
            }
            __syncthreads();
#pragma unroll
            for (int i = 0; i < S2 / S1; ++i)
#pragma unroll
                for (int k2 = 0; k2 < S1; ++k2) row[r + S1 * i + S2 * k2] = y[i][k2];
        }
    }
    __syncthreads();
    // columns: line ix, element dy at L[dy * P + ix]; thread -> (ix = tid % NP, r), a warp 32
    // consecutive columns
    {
        constexpr int RPI = NT / NP, RIT = S1 / RPI;        // r values per iteration, iterations
        static_assert(RPI * RIT == S1, "column split");
        const int ix = tid % NP;
        // every r of a column is read before any is overwritten (the iterations share columns)
        float2 x[RIT][S2];
#pragma unroll
        for (int it = 0; it < RIT; ++it) {
            const int r = RPI * it + tid / NP;
#pragma unroll
            for (int m = 0; m < S2; ++m) x[it][m] = L[(S1 * m + r) * P + ix];
            dft<S2, 1>(x[it]);
#pragma unroll
            for (int k1 = 1; k1 < S2; ++k1) x[it][k1] = cmul(x[it][k1], TW[(r * k1) & MSK]);
        }
        __syncthreads();
#pragma unroll
        for (int it = 0; it < RIT; ++it) {
            const int r = RPI * it + tid / NP;
#pragma unroll
            for (int k1 = 0; k1 < S2; ++k1) L[(r * S2 + (k1 ^ r)) * P + ix] = x[it][k1];
        }
        __syncthreads();
        float* img = image + (size_t)cp * NP * NP;
#pragma unroll 1
        for (int r0 = 0; r0 < S1; r0 += RPI) {
            const int r = r0 + tid / NP;
#pragma unroll
            for (int i = 0; i < S2 / S1; ++i) {
                const int k1 = r + S1 * i;
                float2 y[S1];
#pragma unroll
                for (int q = 0; q < S1; ++q) y[q] = L[(q * S2 + (k1 ^ q)) * P + ix];
                dft<S1, 1>(y);
#pragma unroll
                for (int k2 = 0; k2 < S1; ++k2) img[(size_t)(k1 + S2 * k2) * NP + ix] = y[k2].x;
            }
        }
    }
}

template <int NP>
cudaError_t launch_fx_image_t(const FxArgs& a, cudaStream_t st) {
    const long long n_pair = (long long)a.n_ant * a.n_ant;
    fx_transpose_kernel<<<dim3((unsigned)((n_pair + 31) / 32), (unsigned)((a.n_cp + 31) / 32)), 256, 0, st>>>(
        a.vis, a.n_cp, n_pair, a.vis_t);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const long long tiles = (NP / 8) * (NP / 8);
    if (a.n_cp >= 64 && a.n_cp % 2 == 0) {
        fx_gather_kernel<64, true><<<(unsigned)(tiles * ((a.n_cp + 63) / 64)), FXG_NT, 0, st>>>(a, NP);
    } else {
        int g = 1;
        while (g < 32 && g < a.n_cp) g *= 2;
        const unsigned blocks = (unsigned)(tiles * ((a.n_cp + g - 1) / g));
        switch (g) {
            case 1: fx_gather_kernel<1, false><<<blocks, FXG_NT, 0, st>>>(a, NP); break;
            case 2: fx_gather_kernel<2, false><<<blocks, FXG_NT, 0, st>>>(a, NP); break;
            case 4: fx_gather_kernel<4, false><<<blocks, FXG_NT, 0, st>>>(a, NP); break;
            case 8: fx_gather_kernel<8, false><<<blocks, FXG_NT, 0, st>>>(a, NP); break;
            case 16: fx_gather_kernel<16, false><<<blocks, FXG_NT, 0, st>>>(a, NP); break;
            default: fx_gather_kernel<32, false><<<blocks, FXG_NT, 0, st>>>(a, NP); break;
        }
    }
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    using D = FxDft<NP>;
    if ((e = ensure_smem<fx_dft_kernel<NP>>(D::smem)) != cudaSuccess) return e;
    fx_dft_kernel<NP><<<a.n_cp, D::NT, D::smem, st>>>(a.u, a.image);
    return cudaGetLastError();
}

}  // namespace xe

size_t xeng_smem_bytes() { return xe::smem_bytes(); }

cudaError_t launch_fx_image(int n_pad, const FxArgs& a, cudaStream_t st) {
    if (a.n_cp == 0) return cudaSuccess;
    switch (n_pad) {
        case 32: return xe::launch_fx_image_t<32>(a, st);
        case 64: return xe::launch_fx_image_t<64>(a, st);
        case 128: return xe::launch_fx_image_t<128>(a, st);
        default: return cudaErrorInvalidValue;
    }
}

namespace {
template <int VDT, bool WIDE>
cudaError_t launch_xeng_t(const XengArgs& a, long long grid, cudaStream_t st) {
    const size_t smem = xe::smem_bytes();
    const cudaError_t e = ensure_smem<xe::xeng_kernel<VDT, WIDE>>(smem);
    if (e != cudaSuccess) return e;
    xe::xeng_kernel<VDT, WIDE><<<(unsigned)grid, xe::NT, smem, st>>>(a);
    return cudaGetLastError();
}
}  // namespace

cudaError_t launch_xeng(int vdt, const XengArgs& a, int n_sm, cudaStream_t st) {
    const int nab = (a.n_ant + 127) / 128;
    const long long n_units = (long long)a.n_cp * (nab * (nab + 1) / 2);
    if (n_units == 0) return cudaSuccess;
    if (n_units > 2147483647LL) return cudaErrorInvalidValue;   // the kernel indexes units in 32 bits
    const long long grid = n_units < n_sm ? n_units : n_sm;
    switch (vdt) {
        case 1:
            return launch_xeng_t<1, false>(a, grid, st);
        case 2:
            // 4-byte loads of 4 antennas need every group of 4 to start on a 4-byte boundary
            if (a.n_ant % 4 == 0 && reinterpret_cast<uintptr_t>(a.volt) % 4 == 0)
                return launch_xeng_t<2, true>(a, grid, st);
            return launch_xeng_t<2, false>(a, grid, st);
        default:
            return cudaErrorInvalidValue;
    }
}

}  // namespace epic
