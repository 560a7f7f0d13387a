// Two-pass form of the MOFF imaging step for N_p = 512 (N_g = 256): the zero-padded 2-D spatial
// transform (Sec. 3 "Spatial Fourier Transform") done as a row pass and a column pass with the
// row-transformed grid staged through device memory, instead of one 16-CTA cluster per image.
//
// The cluster form keeps a 512 x 512 image's row-pass output in the distributed shared memory of
// 16 CTAs; only one such cluster fits a GPC, so 112 of 152 SMs work, each with 8 warps.  Here:
//
//   row pass     (twopass_rows_kernel) per image: decode + gain, then the 256 non-zero grid rows
//                in 16 rounds of 16 rows: gather row y's cells (atomics-free, cell-major CSR),
//                pruned 512-point transform along x (Cooley-Tukey 32 x 16, the same register
//                sub-transforms and exchange as the cluster form), row written to the scratch
//                image Y[item][y][kx] with coalesced 16-byte stores;
//   column pass  (twopass_cols_kernel) per (column block of 16 kx, range of items): each item's
//                256 x 16 block of Y staged into shared memory with coalesced loads, the pruned
//                512-point transform along y of each column, |.|^2 accumulated in FP32
//                registers (32 pixels per thread), added to the FP64 accumulator with atomics
//                when the (sub-array, channel, pol) changes, every flush_every samples and at
//                the end.
//
// Items (sub-array, channel*pol, time) are processed in chunks that fit the scratch buffer
// (1 MB of FP32 complex per 512 x 512 item); both kernels run two 256-thread CTAs per SM on
// every SM.  The scratch is owned by the caller of the launcher (a plan or a batch).
#include "moff_common.cuh"

namespace epic {
namespace tp {

constexpr int NP = 512, NG = 256;
using G = Geo<512>;                      // S = 16, R1 = 32, NI = 16, KP = 2, twiddle layout
constexpr int S = G::S, R1 = G::R1, NI = G::NI, KP = G::KP;
constexpr int NT = 256;                  // threads per CTA: 16 transforms of 16 threads
constexpr int LANES = NT / S;            // transforms in flight per CTA (rows or columns)
constexpr int RXS = G::RXS;              // exchange row stride (float2)
constexpr int STS = LANES + 1;           // staging row stride of the column pass (float2)
constexpr size_t ITEM_F2 = (size_t)NG * NP;   // scratch float2 per item (1 MB)
constexpr int VPT = 2;
static_assert(S == 16 && R1 == 32 && KP == 2, "the 512-point factorisation of the cluster form");

constexpr size_t rows_smem_bytes(int max_ant) {
    return sizeof(float2) * ((size_t)LANES * RXS + G::TWN) + (size_t)max_ant * (2 * sizeof(float2) + sizeof(float));
}
constexpr size_t cols_smem_bytes() { return sizeof(float2) * ((size_t)NG * STS + (size_t)LANES * RXS + G::TWN); }

// sub-array (segment) of global item g, starting the search at s
__device__ __forceinline__ int seg_of(const SegList& L, int g, int s) {
    while (s + 1 < L.n_seg && L.first[s + 1] <= g) ++s;
    return s;
}

template <int VDT>
__global__ void __launch_bounds__(NT, 2) twopass_rows_kernel(const __grid_constant__ SegList L, int item0, int item1,
                                                             float2* __restrict__ scratch) {
    using VT = typename Volt<VDT>::T;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float2* RX = reinterpret_cast<float2*>(smem_raw);          // [LANES][RXS]
    float2* TW = RX + LANES * RXS;                             // [S][TWS]
    float2* VB = TW + G::TWN;                                  // [A] g_a V_a
    float2* GN = VB + L.max_ant;                               // [A] gains
    float* PW = reinterpret_cast<float*>(GN + L.max_ant);      // [A] partial sums |g V|^2

    const int tid = threadIdx.x, lane = tid & 31;
    const int n1 = lane % S, r = tid / S;
    G::load_twiddles(TW, L.seg[0].twiddle, tid, NT);
    for (int aa = tid; aa < L.max_ant; aa += NT) PW[aa] = 0.f;

    // this CTA's contiguous share of the chunk's items
    const int n = item1 - item0;
    const int beg = item0 + (int)((long long)n * blockIdx.x / gridDim.x);
    const int end = item0 + (int)((long long)n * (blockIdx.x + 1) / gridDim.x);
    int sg = seg_of(L, beg, 0), cur_sg = -1, cur_cp = -1;
    VT raw[VPT];
    auto prefetch = [&](int g) {
        const int s = seg_of(L, g, sg);
        const FwdArgs& p = L.seg[s];
        const int li = g - L.first[s], cp = li / p.n_time, t = li - cp * p.n_time;
        const VT* base = static_cast<const VT*>(p.volt) + ((long long)t * p.n_cp + cp) * (long long)p.n_ant;
#pragma unroll
        for (int i = 0; i < VPT; ++i)
            if (tid + NT * i < p.n_ant) raw[i] = __ldg(base + tid + NT * i);
    };
    auto flush_power = [&]() {
        if (cur_sg < 0) return;
        const FwdArgs& p = L.seg[cur_sg];
        for (int aa = tid; aa < p.n_ant; aa += NT) {
            if (p.power != nullptr) atomicAdd(p.power + (size_t)cur_cp * p.n_ant + aa, (double)PW[aa]);
            PW[aa] = 0.f;
        }
    };
    if (beg < end) prefetch(beg);
    for (int g = beg; g < end; ++g) {
        sg = seg_of(L, g, sg);
        const FwdArgs& a = L.seg[sg];
        const int li = g - L.first[sg], cp = li / a.n_time, t = li - cp * a.n_time, A = a.n_ant;
        if (sg != cur_sg || cp != cur_cp) {
            flush_power();
            for (int aa = tid; aa < A; aa += NT)
                GN[aa] = a.gains ? a.gains[(size_t)cp * A + aa] : make_float2(1.f, 0.f);
            cur_sg = sg;
            cur_cp = cp;
        }
        // decode + gain (owner threads), prefetch the next item
        const VT* base = static_cast<const VT*>(a.volt) + ((long long)t * a.n_cp + cp) * (long long)A;
#pragma unroll
        for (int i = 0; i < VPT; ++i) {
            const int aa = tid + NT * i;
            if (aa < A) {
                const float2 vp = cmul(GN[aa], Volt<VDT>::dec(raw[i]));
                VB[aa] = vp;
                PW[aa] += cnorm(vp);
            }
        }
        for (int aa = tid + NT * VPT; aa < A; aa += NT) {
            const float2 vp = cmul(GN[aa], Volt<VDT>::dec(__ldg(base + aa)));
            VB[aa] = vp;
            PW[aa] += cnorm(vp);
        }
        if (g + 1 < end) prefetch(g + 1);
        __syncthreads();
        float2* out = scratch + (size_t)(g - item0) * ITEM_F2;
        float2* rx = RX + r * RXS;
#pragma unroll 1
        for (int y = r; y < NG; y += LANES) {
            float2 x[NI];
            gather_cells<NI, true>(x, a.cell_ptr, y * NG + n1, S, a.cell_ent, a.cell_wim, VB);
            float2 Y[R1];
            dft_halfzero_in<R1, +1>(x, Y);
            G::twiddle_store(rx, Y, TW, n1);
            __syncwarp();
            float2 z[KP][S];
#pragma unroll
            for (int q = 0; q < KP; ++q) {
                const int k2 = n1 * KP + q;
#pragma unroll
                for (int m = 0; m < S; ++m) z[q][m] = rx[k2 * S + (m ^ n1)];
                dft<S, +1>(z[q]);
            }
            // kx = n1 KP + q + R1 k1: the two q of one k1 are adjacent, one 16-byte store
            float4* row = reinterpret_cast<float4*>(out + (size_t)y * NP);
#pragma unroll
            for (int k1 = 0; k1 < S; ++k1)
                __stcg(row + (n1 + (R1 / KP) * k1), make_float4(z[0][k1].x, z[0][k1].y, z[1][k1].x, z[1][k1].y));
            __syncwarp();
        }
        __syncthreads();
    }
    flush_power();
}

__global__ void __launch_bounds__(NT, 2) twopass_cols_kernel(const __grid_constant__ SegList L, int item0, int item1,
                                                             const float2* __restrict__ scratch) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float2* ST = reinterpret_cast<float2*>(smem_raw);          // [NG][STS] staged block of Y
    float2* RX = ST + NG * STS;                                // [LANES][RXS]
    float2* TW = RX + LANES * RXS;                             // [S][TWS]
    const int tid = threadIdx.x, lane = tid & 31;
    const int n1 = lane % S, c = tid / S;
    G::load_twiddles(TW, L.seg[0].twiddle, tid, NT);

    constexpr int NB = NP / LANES;                             // column blocks (32)
    const int blk = blockIdx.x % NB, grp = blockIdx.x / NB, n_grp = gridDim.x / NB;
    const int kx = LANES * blk + c;
    const int n = item1 - item0;
    const int beg = item0 + (int)((long long)n * grp / n_grp);
    const int end = item0 + (int)((long long)n * (grp + 1) / n_grp);

    float acc[KP * S];
#pragma unroll
    for (int i = 0; i < KP * S; ++i) acc[i] = 0.f;
    int sg = seg_of(L, beg < end ? beg : item0, 0), cur_sg = -1, cur_cp = -1, since = 0;
    auto flush = [&]() {
        if (cur_sg < 0) return;
        double* dst = L.seg[cur_sg].accum + (size_t)cur_cp * NP * NP;
        const int ix = (kx + NP / 2) & (NP - 1);
#pragma unroll
        for (int q = 0; q < KP; ++q)
#pragma unroll
            for (int k1 = 0; k1 < S; ++k1) {
                const int ky = n1 * KP + q + R1 * k1;
                const int iy = (ky + NP / 2) & (NP - 1);
                atomicAdd(dst + iy * NP + ix, (double)acc[q * S + k1]);
                acc[q * S + k1] = 0.f;
            }
    };
    float2* cx = RX + c * RXS;
    for (int g = beg; g < end; ++g) {
        sg = seg_of(L, g, sg);
        const FwdArgs& a = L.seg[sg];
        const int cp = (g - L.first[sg]) / a.n_time;
        if (sg != cur_sg || cp != cur_cp || since == a.flush_every) {
            flush();
            cur_sg = sg;
            cur_cp = cp;
            since = 0;
        }
        ++since;
        // stage rows 0 .. NG-1, columns LANES blk .. + LANES of the item's row-transformed grid
        const float4* src = reinterpret_cast<const float4*>(scratch + (size_t)(g - item0) * ITEM_F2 + LANES * blk);
        constexpr int PER_ROW = LANES / 2;                     // float4 per staged row (8)
#pragma unroll 4
        for (int i = tid; i < NG * PER_ROW; i += NT) {
            const int row = i / PER_ROW, q4 = i % PER_ROW;
            const float4 v = __ldcg(src + (size_t)row * (NP / 2) + q4);
            ST[row * STS + 2 * q4] = make_float2(v.x, v.y);
            ST[row * STS + 2 * q4 + 1] = make_float2(v.z, v.w);
        }
        __syncthreads();
        float2 x[NI];
#pragma unroll
        for (int n2 = 0; n2 < NI; ++n2) x[n2] = ST[(n1 + S * n2) * STS + c];
        float2 Y[R1];
        dft_halfzero_in<R1, +1>(x, Y);
        G::twiddle_store(cx, Y, TW, n1);
        __syncwarp();
#pragma unroll
        for (int q = 0; q < KP; ++q) {
            const int k2 = n1 * KP + q;
            float2 z[S];
#pragma unroll
            for (int m = 0; m < S; ++m) z[m] = cx[k2 * S + (m ^ n1)];
            dft<S, +1>(z);
#pragma unroll
            for (int k1 = 0; k1 < S; ++k1) acc_norm(acc[q * S + k1], z[k1]);
        }
        __syncthreads();        // the staging buffer and the exchange rows are reused by the next item
    }
    flush();
}

}  // namespace tp

size_t twopass_scratch_bytes(int chunk_items) { return (size_t)chunk_items * tp::ITEM_F2 * sizeof(float2); }
size_t twopass_rows_smem_bytes(int max_ant) { return tp::rows_smem_bytes(max_ant); }

cudaError_t launch_fwd512_twopass(int vdt, const SegList& L, int n_sm, cudaStream_t st, float2* scratch,
                                  int chunk_items) {
    const int total = L.first[L.n_seg];
    if (total == 0) return cudaSuccess;
    if (!scratch || chunk_items < 1) return cudaErrorInvalidValue;
    const size_t rsm = tp::rows_smem_bytes(L.max_ant), csm = tp::cols_smem_bytes();
    cudaError_t e;
    switch (vdt) {
        case 0: e = ensure_smem<tp::twopass_rows_kernel<0>>(rsm); break;
        case 1: e = ensure_smem<tp::twopass_rows_kernel<1>>(rsm); break;
        case 2: e = ensure_smem<tp::twopass_rows_kernel<2>>(rsm); break;
        default: return cudaErrorInvalidValue;
    }
    if (e != cudaSuccess) return e;
    if ((e = ensure_smem<tp::twopass_cols_kernel>(csm)) != cudaSuccess) return e;
    // two CTAs per SM for both passes; the column pass as whole groups of the 32 column blocks
    int workers = 2 * n_sm;
    if (L.max_workers > 0 && workers > 2 * L.max_workers) workers = 2 * L.max_workers;
    const int groups = workers / 32 > 0 ? workers / 32 : 1;
    for (int i0 = 0; i0 < total; i0 += chunk_items) {
        const int i1 = i0 + chunk_items < total ? i0 + chunk_items : total;
        const int rows_grid = workers < i1 - i0 ? workers : i1 - i0;
        switch (vdt) {
            case 0: tp::twopass_rows_kernel<0><<<rows_grid, tp::NT, rsm, st>>>(L, i0, i1, scratch); break;
            case 1: tp::twopass_rows_kernel<1><<<rows_grid, tp::NT, rsm, st>>>(L, i0, i1, scratch); break;
            default: tp::twopass_rows_kernel<2><<<rows_grid, tp::NT, rsm, st>>>(L, i0, i1, scratch); break;
        }
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        const int g = groups < i1 - i0 ? groups : i1 - i0;
        tp::twopass_cols_kernel<<<32 * g, tp::NT, csm, st>>>(L, i0, i1, scratch);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace epic
