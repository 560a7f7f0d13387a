// Forward MOFF kernel: for every (channel, pol, time) item, gain -> gridding ->
// zero-padded 2-D spatial transform -> |.|^2 -> accumulation over time
// (Eq. "dirty-image-MOFF"; Sec. 3 "Gridding Convolution", "Spatial Fourier Transform",
// "Time-averaging").
//
// Persistent: each CTA (or cluster of Q CTAs for N_p = 256) walks a contiguous range of
// items in (channel*pol)-major, time-minor order, keeping its share of the N_p x N_p
// image of the current (channel, pol) in float32 registers, and adds it into the float64
// accumulator with atomics when the (channel, pol) changes, every `flush_every`
// samples, and at the end.
//
// Per item, inside one CTA:
//   decode + gain    owner thread a % NT turns voltage a into g_a V_a in shared memory
//                    (next item's raw voltages are prefetched into registers);
//   row pass         thread (row y, n1) gathers its N_g/S cells E(y, n1 + S n2) from the
//                    cell-major CSR of M(r, a) (atomics-free), runs the first-stage
//                    sub-transform, twiddles, exchanges through shared memory within its
//                    warp, runs the second stage, and writes row y of the row-transformed
//                    grid (to the owning CTA of the cluster for Q > 1);
//   column pass      thread (column, n1) reads the N_g non-zero rows of its column, does
//                    the same two stages along y, squares and accumulates.
// One CTA: two CTA barriers per item; everything else is warp-synchronous.
// Cluster (Q > 1): the row pass sends its outputs with `st.async`, whose bytes complete a
// transaction count on the receiving CTA's mbarrier, so each CTA waits for its own column data
// only (a bounded wait) instead of a cluster barrier.  With two row-pass output buffers (used
// alternately by consecutive items) the item needs no cluster barrier at all: a CTA writes a
// peer's buffer for item i + 2 only after it has received that peer's item-(i + 1) data, which
// the peer sends after its column pass of item i has read the buffer.  With one buffer a
// cluster barrier after the decode keeps the peers' column pass ahead of the next writes.
//
// Cross-polarisation variant (XP): the sub-array has two pols and its (channel, pol) index
// runs over 4 C virtual pols v = 0..3 per channel, v = 0: X, 1: Y, 2: X + Y, 3: X + iY, whose
// gridded fields are g_X V_X (+ phi_v g_Y V_Y), phi_2 = 1, phi_3 = i.  Since the transform is
// linear, the sums of |F_v|^2 give the cross power F_X conj(F_Y) through the polarisation
// identity (Re = (S_2 - S_0 - S_1) / 2, Im = (S_3 - S_0 - S_1) / 2), evaluated in the epilogue.
#pragma once
#include "moff_common.cuh"
#include "tcgen05.cuh"

namespace epic {

// Address in the shared memory of cluster rank q of this CTA's shared address p (volatile: it is
// recomputed at each use instead of being held in registers across the row pass).
__device__ __forceinline__ uint32_t mapa_u32(uint32_t p, int q) {
    uint32_t r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(p), "r"(q));
    return r;
}

// Asynchronous 8-byte store into (possibly another CTA's) shared memory; its bytes complete
// the transaction count of the mbarrier at mbar (in the destination CTA).
__device__ __forceinline__ void st_async_f2(uint32_t addr, float2 v, uint32_t mbar) {
    asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.v2.f32 [%0], {%1, %2}, [%3];"
                 :: "r"(addr), "f"(v.x), "f"(v.y), "r"(mbar) : "memory");
}

// Bounded wait for an mbarrier phase completed by stores of other CTAs of the cluster
// (acquire at cluster scope); false on timeout.  Each try suspends the thread for up to 1 ms.
__device__ __forceinline__ bool mbar_wait_cluster(uint32_t addr, uint32_t parity, int tries) {
    for (int i = 0; i < tries; ++i) {
        uint32_t done;
        asm volatile("{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2, %3;\n\t"
                     "selp.u32 %0, 1, 0, p;\n\t}" : "=r"(done) : "r"(addr), "r"(parity), "r"(1000000u) : "memory");
        if (done) return true;
    }
    return false;
}

// First item whose cost position is >= c: items of sub-array s occupy the cost interval
// [cost[s] + i w_s, cost[s] + (i + 1) w_s); consecutive workers' ranges tile the items exactly.
__device__ __forceinline__ int item_at_cost(const SegList& L, long long c) {
    int s = 0;
    while (s + 1 < L.n_seg && L.cost[s + 1] <= c) ++s;
    const long long off = c - L.cost[s];
    const long long i = (off + L.weight[s] - 1) / L.weight[s];
    const long long n_s = L.first[s + 1] - L.first[s];
    return L.first[s] + (int)(i < n_s ? i : n_s);
}

template <int NP, int VDT, bool XP, int NB>
__global__ void __launch_bounds__(Geo<NP>::NT, Geo<NP>::MINB)
moff_fwd_kernel(const __grid_constant__ SegList L) {
    using G = Geo<NP>;
    constexpr int S = G::S, R1 = G::R1, NI = G::NI, KP = G::KP, NT = G::NT, NG = G::NG;
    constexpr int Q = G::Q, VPT = G::VPT;
    using VT = typename Volt<VDT>::T;

    extern __shared__ __align__(16) unsigned char smem_raw[];
    float2* RX = reinterpret_cast<float2*>(smem_raw);        // [ROWS][RXS] exchange
    float2* RB0 = RX + G::ROWS * G::RXS;                     // [NB][NG][RBS] row-pass output
    float2* TW = RB0 + NB * NG * G::RBS;                     // [S][TWS] exp(+2 pi i n1 k2 / NP)
    uint64_t* MB = reinterpret_cast<uint64_t*>(TW + G::TWN); // [2] exchange mbarriers (Q > 1)
    float2* VB = TW + G::TWN + G::MBF;                       // [A] g_a V_a
    float2* GN = VB + L.max_ant;                             // [A] gains
    float* PW = reinterpret_cast<float*>(GN + L.max_ant);    // [A] partial sum |g V|^2
    float2* GY = reinterpret_cast<float2*>(PW + ((L.max_ant + 1) & ~1));   // XP: [A] phi_v g_Y

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int n1 = lane % S;
    const int r = tid / S;
    const int cc = lane / S;
    int rank = 0, wid = blockIdx.x, nw = gridDim.x;     // worker = CTA (or cluster)
    if constexpr (Q > 1) {
        rank = blockIdx.x % Q;
        wid = blockIdx.x / Q;
        nw = gridDim.x / Q;
    }
    const int y = rank * G::ROWS + r;

    static_assert(NB == 1 || (NB == 2 && Q > 1), "two row-pass buffers serve the cluster forms");
    G::load_twiddles(TW, L.seg[0].twiddle, tid, NT);
    for (int aa = tid; aa < L.max_ant; aa += NT) PW[aa] = 0.f;   // owner-thread entries
    bool lost = false;          // a bounded exchange wait of this thread ran out
    if constexpr (Q > 1) {
        if (tid == 0) {
            tc::mbar_init(tc::smem_u32(MB), 1);
            tc::mbar_init(tc::smem_u32(MB + 1), 1);
            asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        }
        cg::this_cluster().sync();      // every CTA's mbarriers exist before the first exchange
    }

    // global items [0, first[n_seg]) of all sub-arrays, split over the workers in equal shares of
    // estimated cost (equal item counts for a single sub-array)
    const int beg = L.n_seg == 1 ? (int)((long long)L.first[1] * wid / nw) : item_at_cost(L, L.cost[L.n_seg] / nw * wid + L.cost[L.n_seg] % nw * wid / nw);
    const int end = L.n_seg == 1 ? (int)((long long)L.first[1] * (wid + 1) / nw)
                                 : item_at_cost(L, L.cost[L.n_seg] / nw * (wid + 1) + L.cost[L.n_seg] % nw * (wid + 1) / nw);
    int sg = 0;
    while (sg + 1 < L.n_seg && L.first[sg + 1] <= beg) ++sg;
    const FwdArgs* ap = &L.seg[sg];
    int A = ap->n_ant, T = ap->n_time, seg_first = L.first[sg], seg_end = L.first[sg + 1];
    const VT* V = static_cast<const VT*>(ap->volt);
#define a (*ap)

    float acc[2][R1];
#pragma unroll
    for (int s = 0; s < 2; ++s)
#pragma unroll
        for (int i = 0; i < R1; ++i) acc[s][i] = 0.f;

    // voltage row of (channel*pol cp, time t) of sub-array sp (volt = its voltages): for XP,
    // cp is virtual and the row is that of pol X of the channel (pol Y follows it), or of
    // pol Y for v = 1
    auto volt_row = [&](const FwdArgs* sp, const VT* volt, int cp, int t) -> const VT* {
        if constexpr (XP) {
            const int c = cp >> 2, p = (cp & 3) == 1 ? 1 : 0;
            return volt + ((long long)t * (sp->n_cp >> 1) + 2 * c + p) * (long long)sp->n_ant;
        } else {
            return volt + ((long long)t * sp->n_cp + cp) * (long long)sp->n_ant;
        }
    };

    VT raw[VPT], rawy[XP ? VPT : 1];
    // raw voltages of global item g (which may belong to the next sub-array)
    auto prefetch = [&](int g) {
        const FwdArgs* sp = (g < seg_end) ? ap : ap + 1;
        const int li = g - ((g < seg_end) ? seg_first : seg_end);
        const int Tq = sp->n_time, Aq = sp->n_ant;
        const int cp = li / Tq, t = li - cp * Tq;
        const VT* base = volt_row(sp, static_cast<const VT*>(sp->volt), cp, t);
#pragma unroll
        for (int i = 0; i < VPT; ++i) {
            const int aa = tid + NT * i;
            if (aa < Aq) raw[i] = __ldg(base + aa);
            if constexpr (XP) {
                if (aa < Aq && (cp & 3) >= 2) rawy[i] = __ldg(base + Aq + aa);
            }
        }
    };

    auto flush = [&](int cp, bool with_power) {
        double* dst = a.accum + (size_t)cp * NP * NP;
#pragma unroll
        for (int s = 0; s < 2; ++s) {
            const int kx = rank * G::COLS + G::col(s, warp, cc);
            const int ix = (kx + NP / 2) & (NP - 1);
#pragma unroll
            for (int q = 0; q < KP; ++q)
#pragma unroll
                for (int k1 = 0; k1 < S; ++k1) {
                    const int ky = n1 * KP + q + R1 * k1;
                    const int iy = (ky + NP / 2) & (NP - 1);
                    atomicAdd(dst + iy * NP + ix, (double)acc[s][q * S + k1]);
                    acc[s][q * S + k1] = 0.f;
                }
        }
        if (with_power) {
            for (int aa = tid; aa < A; aa += NT) {
                if (a.power != nullptr && rank == 0) atomicAdd(a.power + (size_t)cp * A + aa, (double)PW[aa]);
                PW[aa] = 0.f;
            }
        }
    };

    int cur = -1, since = 0;
    if (beg < end) prefetch(beg);
    for (int g = beg; g < end; ++g) {
        if (g == seg_end) {          // next sub-array: flush, then switch tables and sizes
            if (cur >= 0) flush(cur, true);
            cur = -1;
            ++ap;
            A = ap->n_ant;
            T = ap->n_time;
            V = static_cast<const VT*>(ap->volt);
            seg_first = seg_end;
            seg_end += ap->n_cp * T;
        }
        const int item = g - seg_first;
        const int cp = item / T;
        const int t = item - cp * T;
        if (cp != cur || since == a.flush_every) {
            if (cur >= 0) flush(cur, true);
            if (cp != cur) {
                if constexpr (XP) {
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
            }
            cur = cp;
            since = 0;
        }
        ++since;

        // ---- decode + gain (owner threads), prefetch the next item ----
        {
            const VT* base = XP ? volt_row(ap, V, cp, t) : V + ((long long)t * a.n_cp + cp) * (long long)A;
            const bool two = XP && (cp & 3) >= 2;     // virtual pol combining X and Y
#pragma unroll
            for (int i = 0; i < VPT; ++i) {
                const int aa = tid + NT * i;
                if (aa < A) {
                    float2 vp = cmul(GN[aa], Volt<VDT>::dec(raw[i]));
                    if constexpr (XP) {
                        if (two) {
                            const float2 w = cmul(GY[aa], Volt<VDT>::dec(rawy[i]));
                            vp.x += w.x;
                            vp.y += w.y;
                        }
                    }
                    VB[aa] = vp;
                    PW[aa] += cnorm(vp);
                }
            }
            for (int aa = tid + NT * VPT; aa < A; aa += NT) {
                float2 vp = cmul(GN[aa], Volt<VDT>::dec(__ldg(base + aa)));
                if (two) {
                    const float2 w = cmul(GY[aa], Volt<VDT>::dec(__ldg(base + A + aa)));
                    vp.x += w.x;
                    vp.y += w.y;
                }
                VB[aa] = vp;
                PW[aa] += cnorm(vp);
            }
            if (g + 1 < end) prefetch(g + 1);
        }
        // this worker's item j uses row-pass buffer j % NB, whose mbarrier phase has parity (j / NB) & 1
        const int jb = NB == 2 ? (g - beg) & 1 : 0;
        const uint32_t par = (uint32_t)(((g - beg) / NB) & 1);
        float2* RB = RB0 + jb * (NG * G::RBS);
        if constexpr (NB == 2) {
            __syncthreads();
        } else {
            block_or_cluster_sync<Q>();
        }
        if constexpr (Q > 1) {      // this CTA receives N_g rows x COLS columns of the row pass
            if (tid == 0 && !lost) tc::mbar_expect_tx(tc::smem_u32(MB + jb), NG * G::COLS * (int)sizeof(float2));
        }

        // ---- row pass: gridding + 1-D transform along x of row y ----
        {
            float2 x[NI];
            if constexpr (Cfg<NP>::RR) {
                gather_cells<NI, true>(x, a.cell_ptr, y * NG + n1, S, a.cell_ent, a.cell_wim, VB);
            } else {
                static_assert(Q == 1, "the interleaved mapping assumes one CTA per image");
                gather_interleaved<NI>(x, a.wlane, a.wbase, a.went, a.wwim, (y / G::LPC) * NI, lane, VB);
            }
            float2 Y[R1];
            dft_halfzero_in<R1, +1>(x, Y);
            float2* rx = RX + r * G::RXS;
            G::twiddle_store(rx, Y, TW, n1);
            __syncwarp();
            const uint32_t rb_s = tc::smem_u32(RB), mb_s = tc::smem_u32(MB + jb);
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
                        // after a timeout this thread stops sending: its peers' waits then run
                        // out too (bounded), and no transaction count grows without end
                        const int dst = (R1 * k1) / G::COLS;     // CTA owning column kx
                        if (!lost)
                            st_async_f2(mapa_u32(rb_s + (uint32_t)(y * G::RBS + kx % G::COLS) * (uint32_t)sizeof(float2), dst),
                                        z[k1], mapa_u32(mb_s, dst));
                    } else {
                        RB[y * G::RBS + kx] = z[k1];
                    }
                }
            }
        }
        if constexpr (Q > 1) {      // wait for this CTA's columns from every CTA of the cluster
            if (!lost && !mbar_wait_cluster(tc::smem_u32(MB + jb), par, tc::kWaitTries)) {
                lost = true;
                if (a.status) atomicOr(a.status, kStatusClusterTimeout);
            }
        } else {
            __syncthreads();
        }

        // ---- column pass: 1-D transform along y of two columns, |.|^2, accumulate ----
#pragma unroll
        for (int s = 0; s < 2; ++s) {
            const int c = G::col(s, warp, cc);
            float2 x[NI];
#pragma unroll
            for (int n2 = 0; n2 < NI; ++n2) x[n2] = RB[(n1 + S * n2) * G::RBS + c];
            float2 Y[R1];
            dft_halfzero_in<R1, +1>(x, Y);
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
                for (int k1 = 0; k1 < S; ++k1) acc_norm(acc[s][q * S + k1], z[k1]);
            }
            __syncwarp();
        }
    }
    if (cur >= 0) flush(cur, true);
    // no CTA leaves while a peer may still store into its shared memory (after a timeout)
    if constexpr (Q > 1) cg::this_cluster().sync();
#undef a
}

// Row-pass output buffers of the forward kernel for sub-arrays of up to max_ant antennas: two
// where the form has them and they fit this device's shared memory, else one.
template <int NP, bool XP>
int fwd_buffers(int max_ant) {
    using G = Geo<NP>;
    if constexpr (Cfg<NP>::NB < 2) {
        return 1;
    } else {
        int dev = 0, optin = 0;
        if (cudaGetDevice(&dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess)
            return 1;
        const size_t need = XP ? G::smem_bytes_xpol(max_ant, 2) : G::smem_bytes(max_ant, 2);
        return need <= (size_t)optin ? 2 : 1;
    }
}

template <int NP, int VDT, bool XP, int NB>
cudaError_t launch_fwd_nb(const SegList& L, int n_sm, cudaStream_t st) {
    using G = Geo<NP>;
    auto kern = moff_fwd_kernel<NP, VDT, XP, NB>;
    const size_t smem = XP ? G::smem_bytes_xpol(L.max_ant, NB) : G::smem_bytes(L.max_ant, NB);
    cudaError_t e = ensure_smem<moff_fwd_kernel<NP, VDT, XP, NB>>(smem);
    if (e != cudaSuccess) return e;
    const long long n_items = L.first[L.n_seg];
    if (n_items == 0) return cudaSuccess;
    if constexpr (G::Q == 1) {
        int per_sm = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, G::NT, smem);
        if (e != cudaSuccess) return e;
        if (per_sm < 1) return cudaErrorInvalidConfiguration;
        long long grid = (long long)per_sm * n_sm;
        if (L.max_workers > 0 && grid > L.max_workers) grid = L.max_workers;
        if (grid > n_items) grid = n_items;
        kern<<<(unsigned)grid, G::NT, smem, st>>>(L);
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
        if (L.max_workers > 0 && ncl > L.max_workers) ncl = L.max_workers;
        if (ncl > n_items) ncl = n_items;
        cfg.gridDim = dim3((unsigned)(ncl * G::Q));
        e = cudaLaunchKernelEx(&cfg, kern, L);
        if (e != cudaSuccess) return e;
        return cudaGetLastError();
    }
}

template <int NP, int VDT, bool XP = false>
cudaError_t launch_fwd_t(const SegList& L, int n_sm, cudaStream_t st) {
    if constexpr (Cfg<NP>::NB == 2) {
        if (L.max_buffers != 1 && fwd_buffers<NP, XP>(L.max_ant) == 2) return launch_fwd_nb<NP, VDT, XP, 2>(L, n_sm, st);
    }
    return launch_fwd_nb<NP, VDT, XP, 1>(L, n_sm, st);
}

template <int NP, int VDT, int NB>
int resident_fwd_workers_nb(int max_ant, int n_sm) {
    using G = Geo<NP>;
    auto kern = moff_fwd_kernel<NP, VDT, false, NB>;
    const size_t smem = G::smem_bytes(max_ant, NB);
    if (ensure_smem<moff_fwd_kernel<NP, VDT, false, NB>>(smem) != cudaSuccess) return 0;
    if constexpr (G::Q == 1) {
        int per_sm = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, G::NT, smem) != cudaSuccess) return 0;
        return per_sm * n_sm;
    } else {
        cudaLaunchConfig_t cfg = {};
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = G::Q;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.blockDim = dim3(G::NT);
        cfg.dynamicSmemBytes = smem;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        cfg.gridDim = dim3(G::Q * n_sm);
        if constexpr (G::Q > 8) cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
        int n_cl = 0;
        if (cudaOccupancyMaxActiveClusters(&n_cl, kern, &cfg) != cudaSuccess) return 0;
        return n_cl;
    }
}

template <int NP, int VDT>
int resident_fwd_workers_t(int max_ant, int n_sm) {
    if constexpr (Cfg<NP>::NB == 2) {
        if (fwd_buffers<NP, false>(max_ant) == 2) return resident_fwd_workers_nb<NP, VDT, 2>(max_ant, n_sm);
    }
    return resident_fwd_workers_nb<NP, VDT, 1>(max_ant, n_sm);
}

}  // namespace epic
