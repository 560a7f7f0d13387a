// Adjoint MOFF kernel: gradient of a real image-domain loss with respect to the complex
// per-antenna gains, by the chain rule through Eq. "dirty-image-MOFF" with the gains
// applied before gridding (Sec. 3 "Calibration").
//
// With F_t(k) = sum_g E_t(g) exp(+2 pi i g.k/N_p), E_t = M (g . V_t), I = (1/T) sum_t |F_t|^2
// and G(k) = dL/dI(k):
//     grad_a = (2/T) sum_t conj(V_a(t)) sum_g conj(M[g, a]) Q_t(g),
//     Q_t(g) = sum_k G(k) F_t(k) exp(-2 pi i g.k / N_p),   g in the unpadded N_g x N_g grid.
// Per item the kernel recomputes F_t exactly as the forward kernel does (nothing is stored
// between the two passes), multiplies by G in registers, runs the transposed pruned
// transform (second stage, twiddle, first stage keeping only the N_g non-zero outputs) along
// y and then along x, and degrids Q_t per antenna from shared memory with an antenna-major
// CSR of M (atomics-free); per-antenna sums stay in shared memory and are added to the
// output with float32 atomics when the (channel, pol) changes.
#pragma once
#include "moff_common.cuh"

namespace epic {

template <int NP>
struct BwdLayout {
    using G = Geo<NP>;
    static constexpr int IBS = NP + 1;   // row stride of the column-pass output, [ROWS][IBS]
    static_assert(G::ROWS * IBS <= G::NG * G::RBS, "inverse buffer must fit in the row-pass buffer");
    static constexpr size_t smem_bytes(int n_ant) {
        return sizeof(float2) * (size_t(G::ROWS) * G::RXS + size_t(G::NG) * G::RBS + G::TWN)
             + size_t(n_ant) * 4 * sizeof(float2);
    }
};

template <int NP, int VDT>
__global__ void __launch_bounds__(Geo<NP>::NT, Geo<NP>::MINB)
moff_bwd_kernel(const BwdArgs a) {
    using G = Geo<NP>;
    constexpr int S = G::S, R1 = G::R1, NI = G::NI, KP = G::KP, NT = G::NT, NG = G::NG;
    constexpr int Q = G::Q, IBS = BwdLayout<NP>::IBS;
    using VT = typename Volt<VDT>::T;

    extern __shared__ __align__(16) unsigned char smem_raw[];
    float2* RX = reinterpret_cast<float2*>(smem_raw);        // [ROWS][RXS] exchange, then Q_t rows
    float2* RB = RX + G::ROWS * G::RXS;                      // [NG][RBS] row output; then [ROWS][IBS]
    float2* TW = RB + NG * G::RBS;                           // [S][TWS] exp(+2 pi i n1 k2 / NP)
    float2* VB = TW + G::TWN;                                    // [A] g_a V_a
    float2* VR = VB + a.n_ant;                               // [A] V_a
    float2* GN = VR + a.n_ant;                               // [A] gains
    float2* GA = GN + a.n_ant;                               // [A] partial gradient sums

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int n1 = lane % S;
    const int r = tid / S;
    const int cc = lane / S;
    int rank = 0, wid = blockIdx.x, nw = gridDim.x;
    if constexpr (Q > 1) {
        rank = blockIdx.x % Q;
        wid = blockIdx.x / Q;
        nw = gridDim.x / Q;
    }
    const int y = rank * G::ROWS + r;

    G::load_twiddles(TW, a.twiddle, tid, NT);
    for (int aa = tid; aa < a.n_ant; aa += NT) GA[aa] = make_float2(0.f, 0.f);

    long long beg_l, end_l;
    work_range(a.n_items, wid, nw, beg_l, end_l);
    const int beg = (int)beg_l, end = (int)end_l;   // the host guarantees n_items < 2^31
    const int A = a.n_ant, T = a.n_time;
    const VT* V = static_cast<const VT*>(a.volt);
    const int* aptr = a.ant_ptr + (size_t)rank * (A + 1);

    float gk[2][R1];   // dL/dI at this thread's pixels of the current (channel, pol)

    auto flush = [&](int cp) {
        for (int aa = tid; aa < A; aa += NT) {
            float2* dst = a.grad_gains + (size_t)cp * A + aa;
            atomicAdd(&dst->x, a.scale * GA[aa].x);
            atomicAdd(&dst->y, a.scale * GA[aa].y);
            GA[aa] = make_float2(0.f, 0.f);
        }
    };

    // raw voltages of an item, loaded one item ahead (owner threads aa = tid + NT i)
    constexpr int VPT = G::VPT;
    VT raw[VPT];
    auto prefetch = [&](int item) {
        const int cpn = item / T, tn = item - cpn * T;
        const VT* base = V + ((long long)tn * a.n_cp + cpn) * (long long)A;
#pragma unroll
        for (int i = 0; i < VPT; ++i) {
            const int aa = tid + NT * i;
            if (aa < A) raw[i] = __ldg(base + aa);
        }
    };
    if (beg < end) prefetch(beg);

    int cur = -1;
    for (int item = beg; item < end; ++item) {
        const int cp = item / T;
        const int t = item - cp * T;
        if (cp != cur) {
            if (cur >= 0) flush(cur);
            for (int aa = tid; aa < A; aa += NT)
                GN[aa] = a.gains ? a.gains[(size_t)cp * A + aa] : make_float2(1.f, 0.f);
            const float* gi = a.grad_image + (size_t)cp * NP * NP;
#pragma unroll
            for (int s = 0; s < 2; ++s) {
                const int kx = rank * G::COLS + G::col(s, warp, cc);
                const int ix = (kx + NP / 2) & (NP - 1);
#pragma unroll
                for (int q = 0; q < KP; ++q)
#pragma unroll
                    for (int k1 = 0; k1 < S; ++k1) {
                        const int ky = n1 * KP + q + R1 * k1;
                        gk[s][q * S + k1] = __ldg(gi + ((ky + NP / 2) & (NP - 1)) * NP + ix);
                    }
            }
            cur = cp;
        }

        // ---- decode (this item's voltages were loaded during the previous one), prefetch ----
        {
            const VT* base = V + ((long long)t * a.n_cp + cp) * (long long)A;
#pragma unroll
            for (int i = 0; i < VPT; ++i) {
                const int aa = tid + NT * i;
                if (aa < A) {
                    const float2 v = Volt<VDT>::dec(raw[i]);
                    VR[aa] = v;
                    VB[aa] = cmul(GN[aa], v);
                }
            }
            for (int aa = tid + NT * VPT; aa < A; aa += NT) {
                const float2 v = Volt<VDT>::dec(__ldg(base + aa));
                VR[aa] = v;
                VB[aa] = cmul(GN[aa], v);
            }
            if (item + 1 < end) prefetch(item + 1);
        }
        block_or_cluster_sync<Q>();

        // ---- forward row pass (as in the forward kernel) ----
        {
            float2 x[NI];
            gather_cells<NI, Cfg<NP>::RR>(x, a.cell_ptr, y * NG + n1, S, a.cell_ent, a.cell_wim, VB);
            float2 Y[R1];
            dft_halfzero_in<R1, +1>(x, Y);
            float2* rx = RX + r * G::RXS;
            G::twiddle_store(rx, Y, TW, n1);
            __syncwarp();
#pragma unroll
            for (int q = 0; q < KP; ++q) {
                const int k2 = n1 * KP + q;
                float2 z[S];
#pragma unroll
                for (int m = 0; m < S; ++m) z[m] = rx[k2 * S + (m ^ n1)];
                dft<S, +1>(z);
#pragma unroll
                for (int k1 = 0; k1 < S; ++k1) {
                    const int kx = k2 + R1 * k1;
                    if constexpr (Q > 1) {
                        cluster_ptr(RB, (R1 * k1) / G::COLS)[y * G::RBS + (kx % G::COLS)] = z[k1];
                    } else {
                        RB[y * G::RBS + kx] = z[k1];
                    }
                }
            }
        }
        block_or_cluster_sync<Q>();

        // ---- column loads (both columns), then the row-pass buffer is free ----
        float2 xc[2][NI];
#pragma unroll
        for (int s = 0; s < 2; ++s) {
            const int c = G::col(s, warp, cc);
#pragma unroll
            for (int n2 = 0; n2 < NI; ++n2) xc[s][n2] = RB[(n1 + S * n2) * G::RBS + c];
        }
        block_or_cluster_sync<Q>();

        // ---- column pass: F_t, times G, transposed transform back to the N_g rows ----
#pragma unroll
        for (int s = 0; s < 2; ++s) {
            const int kxg = rank * G::COLS + G::col(s, warp, cc);   // global column
            float2 Y[R1];
            dft_halfzero_in<R1, +1>(xc[s], Y);
            float2* cx = RX + (warp * G::LPC + cc) * G::RXS;
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
                for (int k1 = 0; k1 < S; ++k1) {
                    const float gv = gk[s][q * S + k1];
                    z[k1] = make_float2(gv * z[k1].x, gv * z[k1].y);
                }
                dft<S, -1>(z);
#pragma unroll
                for (int m = 0; m < S; ++m) cx[k2 * S + (m ^ n1)] = z[m];
            }
            __syncwarp();
            G::twiddle_load_conj(cx, Y, TW, n1);
            float2 xo[NI];
            dft_halfzero_out<R1, -1>(Y, xo);
#pragma unroll
            for (int n2 = 0; n2 < NI; ++n2) {
                const int yy = n1 + S * n2;
                if constexpr (Q > 1) {
                    cluster_ptr(RB, yy / G::ROWS)[(yy % G::ROWS) * IBS + kxg] = xo[n2];
                } else {
                    RB[yy * IBS + kxg] = xo[n2];
                }
            }
            __syncwarp();
        }
        block_or_cluster_sync<Q>();

        // ---- transposed row pass: Q_t(y, x) for the N_g cells of row y ----
        {
            float2* rx = RX + r * G::RXS;
            const float2* ib = RB + r * IBS;
#pragma unroll
            for (int q = 0; q < KP; ++q) {
                const int k2 = n1 * KP + q;
                float2 z[S];
#pragma unroll
                for (int k1 = 0; k1 < S; ++k1) z[k1] = ib[k2 + R1 * k1];
                dft<S, -1>(z);
#pragma unroll
                for (int m = 0; m < S; ++m) rx[k2 * S + (m ^ n1)] = z[m];
            }
            __syncwarp();
            float2 Y[R1];
            G::twiddle_load_conj(rx, Y, TW, n1);
            float2 xo[NI];
            dft_halfzero_out<R1, -1>(Y, xo);
            __syncwarp();
#pragma unroll
            for (int n2 = 0; n2 < NI; ++n2) rx[n1 + S * n2] = xo[n2];
        }
        __syncthreads();

        // ---- degrid: per antenna, sum_g conj(M[g, a]) Q_t(g) over this CTA's rows ----
        for (int aa = tid; aa < A; aa += NT) {
            float2 s = make_float2(0.f, 0.f);
            const int e1 = __ldg(aptr + aa + 1);
            for (int e = __ldg(aptr + aa); e < e1; ++e) {
                const int2 en = __ldg(a.ant_ent + e);
                const float2 qv = RX[en.y];
                // conj(w) * q
                const float wr = __int_as_float(en.x), wi = a.ant_wim ? __ldg(a.ant_wim + e) : 0.f;
                s.x = fmaf(wr, qv.x, fmaf(wi, qv.y, s.x));
                s.y = fmaf(wr, qv.y, fmaf(-wi, qv.x, s.y));
            }
            const float2 v = VR[aa];
            // conj(v) * s
            GA[aa].x += v.x * s.x + v.y * s.y;
            GA[aa].y += v.x * s.y - v.y * s.x;
        }
    }
    if (cur >= 0) flush(cur);
}

template <int NP, int VDT>
cudaError_t launch_bwd_t(const BwdArgs& a, int n_sm, cudaStream_t st) {
    using G = Geo<NP>;
    auto kern = moff_bwd_kernel<NP, VDT>;
    const size_t smem = BwdLayout<NP>::smem_bytes(a.n_ant);
    cudaError_t e = ensure_smem<moff_bwd_kernel<NP, VDT>>(smem);
    if (e != cudaSuccess) return e;
    if (a.n_items == 0) return cudaSuccess;
    if constexpr (G::Q == 1) {
        int per_sm = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, G::NT, smem);
        if (e != cudaSuccess) return e;
        if (per_sm < 1) return cudaErrorInvalidConfiguration;
        long long grid = (long long)per_sm * n_sm;
        if (grid > a.n_items) grid = a.n_items;
        kern<<<(unsigned)grid, G::NT, smem, st>>>(a);
        return cudaGetLastError();
    } else {
        cudaLaunchConfig_t cfg = {};
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = G::Q;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.blockDim = dim3(G::NT);
        cfg.dynamicSmemBytes = smem;
        cfg.stream = st;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        cfg.gridDim = dim3(G::Q * n_sm);
        if constexpr (G::Q > 8) {
            e = cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
            if (e != cudaSuccess) return e;
        }
        int n_cl = 0;
        e = cudaOccupancyMaxActiveClusters(&n_cl, kern, &cfg);
        if (e != cudaSuccess) return e;
        if (n_cl < 1) return cudaErrorInvalidConfiguration;
        long long ncl = n_cl;
        if (ncl > a.n_items) ncl = a.n_items;
        cfg.gridDim = dim3((unsigned)(ncl * G::Q));
        e = cudaLaunchKernelEx(&cfg, kern, a);
        if (e != cudaSuccess) return e;
        return cudaGetLastError();
    }
}

}  // namespace epic
