// C ABI of the MOFF imaging library: plan construction (the antenna-to-grid mapping of
// Sec. 3, built once in float64 on the host), argument validation and launches.
#include <algorithm>
#include <cmath>
#include <complex>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>
#include <cuda_fp16.h>

#include "../../include/epic.h"
#include "epic_internal.h"
#include "epic_plan.h"
#include "epic_trace.h"

namespace {
thread_local std::string g_err;
bool is_pow2_size(int n) { return n == 32 || n == 64 || n == 128 || n == 256 || n == 512; }
}  // namespace

void epic_clear_error() { g_err.clear(); }

epic_status epic_fail(epic_status st, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_err = buf;
    return st;
}

epic_status epic_cuda_fail(cudaError_t e, const char* what) {
    return epic_fail(EPIC_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

epic_status epic_check_alignment(std::initializer_list<EpicAlign> arrays) {
    for (const EpicAlign& x : arrays)
        if (x.ptr && reinterpret_cast<uintptr_t>(x.ptr) % x.bytes != 0)
            return epic_fail(EPIC_EINVAL, "%s must be %zu-byte aligned", x.name, x.bytes);
    return EPIC_OK;
}

size_t epic_volt_bytes(int vdt) { return vdt == EPIC_VOLT_C64 ? 8 : vdt == EPIC_VOLT_F16 ? 4 : 1; }

namespace {

void free_plan(epic_plan* p) {
    if (!p) return;
    cudaFree(p->cell_ptr);
    cudaFree(p->cell_ent);
    cudaFree(p->cell_wim);
    cudaFree(p->fx_ptr);
    cudaFree(p->fx_ent);
    cudaFree(p->fx_wim);
    cudaFree(p->wlane);
    cudaFree(p->wbase);
    cudaFree(p->went);
    cudaFree(p->wwim);
    cudaFree(p->ant_ptr);
    cudaFree(p->ant_ent);
    cudaFree(p->ant_wim);
    cudaFree(p->twiddle);
    cudaFree(p->lag_tab);
    cudaFree(p->dg_tab);
    cudaFree(p->dg_lane);
    cudaFree(p->dg_base);
    cudaFree(p->dg_wre);
    cudaFree(p->dg_wim);
    cudaFree(p->dg_ant);
    cudaFree(p->dg_wpk);
    cudaFree(p->status);
    cudaFree(p->tp_scratch);
    cudaFree(p->fx_lag_ptr);
    cudaFree(p->fx_lag_ent);
    cudaFree(p->fx_vis_t);
    cudaFree(p->fx_u);
    delete p;
}

template <typename T>
cudaError_t upload(T** dst, const std::vector<T>& src) {
    const size_t bytes = std::max<size_t>(src.size(), 1) * sizeof(T);
    cudaError_t e = cudaMalloc(reinterpret_cast<void**>(dst), bytes);
    if (e != cudaSuccess) return e;
    if (!src.empty()) e = cudaMemcpy(*dst, src.data(), src.size() * sizeof(T), cudaMemcpyHostToDevice);
    return e;
}

int2 pack_entry(std::complex<double> w, int idx) {
    const float wr = float(w.real());
    int2 e;
    std::memcpy(&e.x, &wr, 4);
    e.y = idx;
    return e;
}

struct MapEntry {
    int cell, ant, tap;
    std::complex<double> w;
};

}  // namespace

cudaError_t epic_launch_fwd_list(int n_pad, int vdt, const epic::SegList& L, int n_sm, cudaStream_t st, bool xpol) {
    switch (n_pad) {
        case 32: return epic::launch_fwd_32(vdt, L, n_sm, st, xpol);
        case 64: return epic::launch_fwd_64(vdt, L, n_sm, st, xpol);
        case 128: return epic::launch_fwd_128(vdt, L, n_sm, st, xpol);
        case 256: return epic::launch_fwd_256(vdt, L, n_sm, st, xpol);
        case 512: return epic::launch_fwd_512(vdt, L, n_sm, st, xpol);
        default: return cudaErrorInvalidValue;
    }
}

int epic_resident_workers(int n_pad, int vdt, const std::vector<epic_plan*>& plans, const std::vector<int>& members,
                          int n_sm) {
    int max_ant = 0;
    for (int i : members) max_ant = std::max(max_ant, plans[i]->n_ant);
    return epic::resident_fwd_workers(n_pad, vdt, max_ant, n_sm);
}

epic::FwdArgs epic_plan_fwd_args(const epic_plan* plan, const void* volt, int n_time, const float2* gains,
                                 double* accum, double* power) {
    epic::FwdArgs a;
    a.volt = volt;
    a.n_time = n_time;
    a.n_cp = plan->n_chan * plan->n_pol;
    a.n_ant = plan->n_ant;
    a.gains = gains;
    a.cell_ptr = plan->cell_ptr;
    a.cell_ent = plan->cell_ent;
    a.cell_wim = plan->cell_wim;
    a.wlane = plan->wlane;
    a.wbase = plan->wbase;
    a.went = plan->went;
    a.wwim = plan->wwim;
    a.twiddle = plan->twiddle;
    a.accum = accum;
    a.power = power;
    a.n_items = (long long)a.n_cp * n_time;
    a.flush_every = 1024;
    a.wsum_max = plan->wsum_max;
    a.status = plan->status;
    a.wait_tries = plan->wait_tries;
    return a;
}

namespace {

epic_status launch_fwd(const epic_plan* p, const epic::FwdArgs& a, cudaStream_t st, bool xpol = false) {
    epic::SegList L;
    L.seg[0] = a;
    L.first[0] = 0;
    L.first[1] = (int)a.n_items;
    L.weight[0] = 1;
    L.cost[0] = 0;
    L.cost[1] = a.n_items;
    L.n_seg = 1;
    L.max_ant = a.n_ant;
    L.max_workers = 0;
    const cudaError_t e = epic_launch_fwd_list(p->n_pad, p->vdt, L, p->n_sm, st, xpol);
    return e == cudaSuccess ? EPIC_OK : epic_cuda_fail(e, "imaging kernel launch");
}

epic_status launch_bwd(const epic_plan* p, const epic::BwdArgs& a, cudaStream_t st) {
    cudaError_t e;
    switch (p->n_pad) {
        case 32: e = epic::launch_bwd_32(p->vdt, a, p->n_sm, st); break;
        case 64: e = epic::launch_bwd_64(p->vdt, a, p->n_sm, st); break;
        case 128: e = epic::launch_bwd_128(p->vdt, a, p->n_sm, st); break;
        case 256: e = epic::launch_bwd_256(p->vdt, a, p->n_sm, st); break;
        case 512: e = epic::launch_bwd_512(p->vdt, a, p->n_sm, st); break;
        default: return epic_fail(EPIC_EUNSUPPORTED, "n_pad %d", p->n_pad);
    }
    return e == cudaSuccess ? EPIC_OK : epic_cuda_fail(e, "adjoint kernel launch");
}

}  // namespace

extern "C" {

const char* epic_last_error(void) { return g_err.c_str(); }


epic_status epic_create(epic_plan** plan, int n_ant, const double* pos_xy, const int* kern_ptr,
                        const double* kern_dxdy, const double* kern_w, double dx,
                        const double* origin_xy, int n_grid, int n_pad, int n_chan, int n_pol,
                        int volt_dtype, int device) {
    EpicRange range("epic_create");
    epic_clear_error();
    if (!plan) return epic_fail(EPIC_EINVAL, "plan out-pointer is NULL");
    *plan = nullptr;
    if (n_ant < 1 || n_ant > 4096) return epic_fail(EPIC_EINVAL, "n_ant = %d outside 1..4096", n_ant);
    if (!pos_xy || !kern_ptr || !origin_xy) return epic_fail(EPIC_EINVAL, "NULL host array");
    if (!(dx > 0.0) || !std::isfinite(dx)) return epic_fail(EPIC_EINVAL, "grid spacing must be finite and > 0");
    if (!std::isfinite(origin_xy[0]) || !std::isfinite(origin_xy[1])) return epic_fail(EPIC_EINVAL, "origin not finite");
    if (!is_pow2_size(n_pad)) return epic_fail(EPIC_EUNSUPPORTED, "n_pad = %d (supported: 32, 64, 128, 256, 512)", n_pad);
    if (n_grid < 1 || 2 * n_grid > n_pad)
        return epic_fail(EPIC_EINVAL, "n_grid = %d must be in 1..n_pad/2 (2x zero padding)", n_grid);
    if (n_chan < 1 || n_pol < 1) return epic_fail(EPIC_EINVAL, "n_chan and n_pol must be >= 1");
    if (volt_dtype < EPIC_VOLT_C64 || volt_dtype > EPIC_VOLT_CI4) return epic_fail(EPIC_EINVAL, "volt_dtype %d", volt_dtype);
    if (kern_ptr[0] != 0) return epic_fail(EPIC_EINVAL, "kern_ptr[0] must be 0");
    for (int a = 0; a < n_ant; ++a)
        if (kern_ptr[a + 1] < kern_ptr[a]) return epic_fail(EPIC_EINVAL, "kern_ptr not non-decreasing at antenna %d", a);
    const int n_taps = kern_ptr[n_ant];
    if (n_taps > 0 && (!kern_dxdy || !kern_w)) return epic_fail(EPIC_EINVAL, "NULL footprint table");

    const int NG = n_pad / 2;   // the kernels work on the N_p/2 grid; cells >= n_grid stay empty
    const double ox = origin_xy[0], oy = origin_xy[1];
    std::vector<MapEntry> ents;
    ents.reserve(n_taps);
    for (int a = 0; a < n_ant; ++a) {
        const double px = pos_xy[2 * a], py = pos_xy[2 * a + 1];
        if (!std::isfinite(px) || !std::isfinite(py)) return epic_fail(EPIC_EINVAL, "antenna %d position not finite", a);
        for (int k = kern_ptr[a]; k < kern_ptr[a + 1]; ++k) {
            const double x = px + kern_dxdy[2 * k];
            const double y = py + kern_dxdy[2 * k + 1];
            const double ux = (x - ox) / dx + 0.5;
            const double uy = (y - oy) / dx + 0.5;
            if (!std::isfinite(ux) || !std::isfinite(uy))
                return epic_fail(EPIC_EINVAL, "footprint sample %d of antenna %d not finite", k, a);
            const double fx = std::floor(ux), fy = std::floor(uy);
            if (fx < 0 || fy < 0 || fx >= n_grid || fy >= n_grid)
                return epic_fail(EPIC_EINVAL, "footprint sample %d of antenna %d maps to cell (%g, %g) outside the %d x %d grid",
                            k, a, fy, fx, n_grid, n_grid);
            const std::complex<double> w(kern_w[2 * k], kern_w[2 * k + 1]);
            if (!std::isfinite(w.real()) || !std::isfinite(w.imag()))
                return epic_fail(EPIC_EINVAL, "footprint weight %d not finite", k);
            ents.push_back({int(fy) * NG + int(fx), a, k, w});
        }
    }
    // M(r, a): sum the weights of samples of the same antenna landing in the same cell,
    // in tap order.
    std::stable_sort(ents.begin(), ents.end(), [](const MapEntry& l, const MapEntry& r) {
        return l.cell != r.cell ? l.cell < r.cell : (l.ant != r.ant ? l.ant < r.ant : l.tap < r.tap);
    });
    std::vector<MapEntry> m;
    for (const MapEntry& e : ents) {
        if (!m.empty() && m.back().cell == e.cell && m.back().ant == e.ant)
            m.back().w += e.w;
        else
            m.push_back(e);
    }

    epic_plan* p = new epic_plan;
    p->n_ant = n_ant;
    p->n_grid = n_grid;
    p->n_pad = n_pad;
    p->n_chan = n_chan;
    p->n_pol = n_pol;
    p->vdt = volt_dtype;
    p->device = device;
    p->nnz = (int64_t)m.size();

    // cell-major CSR (gather side of the gridding)
    std::vector<int> cptr((size_t)NG * NG + 1, 0);
    std::vector<int2> cent;
    std::vector<float> cwim;
    cent.reserve(m.size());
    cwim.reserve(m.size());
    bool complex_w = false;
    for (const MapEntry& e : m) {
        cptr[e.cell + 1]++;
        cent.push_back(pack_entry(e.w, e.ant));
        cwim.push_back(float(e.w.imag()));
        complex_w = complex_w || (float(e.w.imag()) != 0.0f);
    }
    for (size_t i = 0; i + 1 < cptr.size(); ++i) {
        if (cptr[i + 1] > 0) p->n_cells++;
        cptr[i + 1] += cptr[i];
    }
    {
        std::vector<double> wsum((size_t)NG * NG, 0.0);
        for (const MapEntry& e : m) wsum[e.cell] += std::abs(e.w);
        double wm = 0.0;
        for (double v : wsum) wm = std::max(wm, v);
        p->wsum_max = float(wm * (1.0 + 1e-6));
    }

    // warp-interleaved copy of the cell-major mapping for the forward kernels that gather cell
    // by cell: group (row block yb, n2) serves the warp whose lane l owns cell
    // (yb * 32/S + l / S, l % S + S * n2); the lanes are ranked by decreasing entry count, and
    // step k stores the k-th entry of the lanes of rank 0 .. n_k - 1 (those with more than k
    // entries), so the active lanes of a step read one contiguous run.
    std::vector<int> wlane, wbase;
    std::vector<int2> went;
    std::vector<float> wwim;
    const int SL = epic::fwd_interleave_lanes(n_pad);
    if (SL > 0) {
        const int LPC = 32 / SL, NI = NG / SL, n_blk = NG / LPC;
        wlane.resize((size_t)n_blk * NI * 32);
        wbase.resize((size_t)n_blk * NI);
        went.reserve(m.size());
        wwim.reserve(m.size());
        for (int yb = 0; yb < n_blk; ++yb) {
            for (int n2 = 0; n2 < NI; ++n2) {
                const int g = yb * NI + n2;
                int cell[32], cnt[32], order[32], rank[32];
                for (int l = 0; l < 32; ++l) {
                    cell[l] = (yb * LPC + l / SL) * NG + (l % SL) + SL * n2;
                    cnt[l] = cptr[cell[l] + 1] - cptr[cell[l]];
                    order[l] = l;
                }
                std::stable_sort(order, order + 32, [&](int x, int y) { return cnt[x] > cnt[y]; });
                for (int i = 0; i < 32; ++i) rank[order[i]] = i;
                wbase[g] = (int)went.size();
                for (int l = 0; l < 32; ++l) wlane[(size_t)g * 32 + l] = cnt[l] | (rank[l] << 16);
                for (int k = 0; k < cnt[order[0]]; ++k) {
                    for (int i = 0; i < 32 && cnt[order[i]] > k; ++i) {
                        const int e = cptr[cell[order[i]]] + k;
                        went.push_back(cent[e]);
                        wwim.push_back(cwim[e]);
                    }
                }
            }
        }
    }

    // gridding slot tables of the tensor-core forms (N_p = 128 and 256)
    std::vector<int2> dlane;
    std::vector<int> dbase;
    std::vector<float> dwre, dwim;
    std::vector<uint16_t> dant;
    const bool dg_ok = (n_pad == 128 && epic::dftgemm_gather_tables(cptr, cent, cwim, dlane, dbase, dwre, dwim, dant)) ||
                       (n_pad == 256 &&
                        epic::dftgemm_gather_tables_ng(128, epic::kDg256GridWarps, cptr, cent, cwim, dlane, dbase,
                                                       dwre, dwim, dant));
    // N_p = 256 with real weights: the same entries packed one word each for the FP16-gridding
    // form, (FP16 weight, rounded to nearest) << 16 | antenna
    std::vector<uint32_t> dwpk;
    if (dg_ok && n_pad == 256 && !complex_w) {
        dwpk.resize(dwre.size());
        for (size_t q = 0; q < dwre.size(); ++q)
            dwpk[q] = ((uint32_t)__half_as_ushort(__float2half_rn(dwre[q])) << 16) | (uint32_t)dant[q];
    }

    // antenna-major CSR per row block (degridding side of the adjoint); cells are stored as
    // offsets into the adjoint kernel's shared-memory row buffer
    const int rows = epic::grid_rows_per_block(n_pad);
    const int nq = NG / rows;
    const int rxs = epic::exchange_row_stride(n_pad);
    std::vector<std::vector<std::pair<int2, float>>> per_ant((size_t)nq * n_ant);
    for (const MapEntry& e : m) {
        const int gy = e.cell / NG, gx = e.cell % NG;
        const int q = gy / rows;
        per_ant[(size_t)q * n_ant + e.ant].push_back({pack_entry(e.w, (gy - q * rows) * rxs + gx), float(e.w.imag())});
    }
    std::vector<int> aptr((size_t)nq * (n_ant + 1), 0);
    std::vector<int2> aent;
    std::vector<float> awim;
    aent.reserve(m.size());
    awim.reserve(m.size());
    for (int q = 0; q < nq; ++q) {
        aptr[(size_t)q * (n_ant + 1)] = (int)aent.size();
        for (int a = 0; a < n_ant; ++a) {
            for (auto& pe : per_ant[(size_t)q * n_ant + a]) {
                aent.push_back(pe.first);
                awim.push_back(pe.second);
            }
            aptr[(size_t)q * (n_ant + 1) + a + 1] = (int)aent.size();
        }
    }

    // per-antenna footprint auto-correlation R_a(d) on the L x L lag window
    std::vector<std::vector<const MapEntry*>> by_ant(n_ant);
    for (const MapEntry& e : m) by_ant[e.ant].push_back(&e);
    int ext = 1;
    for (int a = 0; a < n_ant; ++a) {
        if (by_ant[a].empty()) continue;
        int x0 = 1 << 30, x1 = -1, y0 = 1 << 30, y1 = -1;
        for (const MapEntry* e : by_ant[a]) {
            const int gy = e->cell / NG, gx = e->cell % NG;
            x0 = std::min(x0, gx); x1 = std::max(x1, gx);
            y0 = std::min(y0, gy); y1 = std::max(y1, gy);
        }
        ext = std::max(ext, std::max(x1 - x0 + 1, y1 - y0 + 1));
    }
    const int L = 2 * ext - 1;
    // antenna-major copy of the mapping with (gy, gx) packed, for the FX route's gridding of
    // visibilities with the antenna-pair kernels (N_p <= 128)
    std::vector<int> fxptr;
    std::vector<int2> fxent;
    std::vector<float> fxwim;
    if (n_pad <= 128) {
        fxptr.assign((size_t)n_ant + 1, 0);
        fxent.reserve(m.size());
        fxwim.reserve(m.size());
        for (int a = 0; a < n_ant; ++a) {
            for (const MapEntry* e : by_ant[a]) {
                fxent.push_back(pack_entry(e->w, ((e->cell / NG) << 16) | (e->cell % NG)));
                fxwim.push_back(float(e->w.imag()));
            }
            fxptr[(size_t)a + 1] = (int)fxent.size();
        }
    }
    std::vector<float2> lag;
    int smem_optin_ac = 0;
    cudaDeviceGetAttribute(&smem_optin_ac, cudaDevAttrMaxSharedMemoryPerBlockOptin, device);
    if (L <= 63 && epic::autocorr_smem_bytes(L, n_pad, n_ant) <= (size_t)smem_optin_ac) {
        p->lag_side = L;
        const int h = ext - 1;
        lag.assign((size_t)n_ant * L * L, make_float2(0.f, 0.f));
        std::vector<std::complex<double>> acc((size_t)L * L);
        for (int a = 0; a < n_ant; ++a) {
            std::fill(acc.begin(), acc.end(), std::complex<double>(0.0, 0.0));
            for (const MapEntry* e : by_ant[a])
                for (const MapEntry* f : by_ant[a]) {
                    const int dy = e->cell / NG - f->cell / NG, dxl = e->cell % NG - f->cell % NG;
                    acc[(size_t)(dy + h) * L + (dxl + h)] += e->w * std::conj(f->w);
                }
            for (size_t j = 0; j < acc.size(); ++j)
                lag[(size_t)a * L * L + j] = make_float2(float(acc[j].real()), float(acc[j].imag()));
        }
    }

    std::vector<float2> tw(n_pad);
    for (int j = 0; j < n_pad; ++j) {
        const double ang = 2.0 * M_PI * double(j) / double(n_pad);
        tw[j] = make_float2(float(std::cos(ang)), float(std::sin(ang)));
    }

    EpicDeviceGuard guard(device);
    if (!guard.ok) {
        delete p;
        return epic_fail(EPIC_ECUDA, "cannot select CUDA device %d", device);
    }
    cudaError_t e = cudaDeviceGetAttribute(&p->n_sm, cudaDevAttrMultiProcessorCount, device);
    if (e != cudaSuccess) {
        delete p;
        return epic_cuda_fail(e, "cudaDeviceGetAttribute");
    }
    int smem_optin = 0;
    cudaDeviceGetAttribute(&smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, device);
    const size_t need = epic::fwd_smem_bytes(n_pad, n_ant);   // the adjoint's own need is checked by its call
    if (need > (size_t)smem_optin) {
        delete p;
        return epic_fail(EPIC_EUNSUPPORTED, "%d antennas need %zu bytes of shared memory per block (device limit %d)",
                    n_ant, need, smem_optin);
    }
    if ((e = upload(&p->cell_ptr, cptr)) != cudaSuccess || (e = upload(&p->cell_ent, cent)) != cudaSuccess ||
        (e = upload(&p->ant_ptr, aptr)) != cudaSuccess || (e = upload(&p->ant_ent, aent)) != cudaSuccess ||
        (e = upload(&p->twiddle, tw)) != cudaSuccess || (e = upload(&p->lag_tab, lag)) != cudaSuccess ||
        (complex_w && ((e = upload(&p->cell_wim, cwim)) != cudaSuccess || (e = upload(&p->ant_wim, awim)) != cudaSuccess)) ||
        (n_pad <= 128 && ((e = upload(&p->fx_ptr, fxptr)) != cudaSuccess || (e = upload(&p->fx_ent, fxent)) != cudaSuccess ||
                          (complex_w && (e = upload(&p->fx_wim, fxwim)) != cudaSuccess))) ||
        (SL > 0 && ((e = upload(&p->wlane, wlane)) != cudaSuccess || (e = upload(&p->wbase, wbase)) != cudaSuccess ||
                    (e = upload(&p->went, went)) != cudaSuccess ||
                    (complex_w && (e = upload(&p->wwim, wwim)) != cudaSuccess))) ||
        (dg_ok && ((e = upload(&p->dg_lane, dlane)) != cudaSuccess || (e = upload(&p->dg_base, dbase)) != cudaSuccess ||
                   (e = upload(&p->dg_wre, dwre)) != cudaSuccess || (e = upload(&p->dg_ant, dant)) != cudaSuccess ||
                   (complex_w && (e = upload(&p->dg_wim, dwim)) != cudaSuccess) ||
                   (!dwpk.empty() && (e = upload(&p->dg_wpk, dwpk)) != cudaSuccess)))) {
        free_plan(p);
        return e == cudaErrorMemoryAllocation ? epic_fail(EPIC_ENOMEM, "plan tables: %s", cudaGetErrorString(e))
                                              : epic_cuda_fail(e, "plan upload");
    }
    p->fx_ptr_h = fxptr;
    p->fx_ent_h = fxent;
    p->fx_wim_h = fxwim;
    if ((e = upload(&p->status, std::vector<int>(1, 0))) != cudaSuccess) {
        free_plan(p);
        return e == cudaErrorMemoryAllocation ? epic_fail(EPIC_ENOMEM, "status word: %s", cudaGetErrorString(e))
                                              : epic_cuda_fail(e, "status word");
    }
    *plan = p;
    return EPIC_OK;
}

namespace {

std::mutex g_fx_lag_mu;
constexpr int64_t kMaxFxLagEntries = 1LL << 27;   // 2 GB of device tables at most

// The FX route's antenna-pair kernels of every ordered pair (autocorrelations included),
// B_ab(d) = sum over mapping entries e of a and f of b with g_e - g_f = d of w_e conj(w_f)
// (Eq. "e-field-conv": the cross-correlation of the two sampled footprints), summed per pair in
// float64 and grouped by wrapped lag cell d into a CSR, uploaded to the plan.  Built once, by the
// first epic_fx_image call.
epic_status build_fx_lag_table(const epic_plan* p) {
    const int A = p->n_ant, NP = p->n_pad, MSK = NP - 1;
    int lg = 0;
    while ((1 << lg) < NP) ++lg;
    const std::vector<int>& ptr = p->fx_ptr_h;
    const std::vector<int2>& ent = p->fx_ent_h;
    const bool cw = p->fx_wim != nullptr;
    std::vector<int> y0(A, 1 << 30), y1(A, -1), x0(A, 1 << 30), x1(A, -1);
    for (int a = 0; a < A; ++a)
        for (int e = ptr[a]; e < ptr[a + 1]; ++e) {
            const int gy = ent[e].y >> 16, gx = ent[e].y & 0xFFFF;
            y0[a] = std::min(y0[a], gy); y1[a] = std::max(y1[a], gy);
            x0[a] = std::min(x0[a], gx); x1[a] = std::max(x1[a], gx);
        }
    int64_t bound = 0;
    for (int a = 0; a < A; ++a)
        for (int b = 0; b < A; ++b)
            if (y1[a] >= 0 && y1[b] >= 0)
                bound += (int64_t)(y1[a] - y0[a] + y1[b] - y0[b] + 1) * (x1[a] - x0[a] + x1[b] - x0[b] + 1);
    if (bound > kMaxFxLagEntries)
        return epic_fail(EPIC_EUNSUPPORTED, "the antenna-pair lag table would hold up to %lld entries (limit %lld)",
                         (long long)bound, (long long)kMaxFxLagEntries);
    if ((int64_t)A * A * p->n_chan * p->n_pol > 2147483647LL)
        return epic_fail(EPIC_EUNSUPPORTED, "A^2 * C * P = %lld visibilities: the FX imaging indexes them in 32 bits",
                         (long long)A * A * p->n_chan * p->n_pol);
    std::vector<int> lag, pair;
    std::vector<float2> w;
    lag.reserve((size_t)bound);
    pair.reserve((size_t)bound);
    w.reserve((size_t)bound);
    std::vector<std::complex<double>> win;
    auto weight = [&](int e) {
        float re;
        std::memcpy(&re, &ent[e].x, sizeof(float));
        return std::complex<double>(re, cw ? p->fx_wim_h[e] : 0.0);
    };
    for (int a = 0; a < A; ++a) {
        if (y1[a] < 0) continue;
        for (int b = 0; b < A; ++b) {
            if (y1[b] < 0) continue;
            const int dy0 = y0[a] - y1[b], dx0 = x0[a] - x1[b];
            const int H = y1[a] - y0[a] + y1[b] - y0[b] + 1, W = x1[a] - x0[a] + x1[b] - x0[b] + 1;
            win.assign((size_t)H * W, std::complex<double>(0.0, 0.0));
            for (int e = ptr[a]; e < ptr[a + 1]; ++e) {
                const std::complex<double> we = weight(e);
                const int gye = ent[e].y >> 16, gxe = ent[e].y & 0xFFFF;
                for (int f = ptr[b]; f < ptr[b + 1]; ++f) {
                    const int dy = gye - (ent[f].y >> 16), dx = gxe - (ent[f].y & 0xFFFF);
                    win[(size_t)(dy - dy0) * W + (dx - dx0)] += we * std::conj(weight(f));
                }
            }
            for (int i = 0; i < H; ++i)
                for (int j = 0; j < W; ++j) {
                    const std::complex<double> v = win[(size_t)i * W + j];
                    if (v == std::complex<double>(0.0, 0.0)) continue;
                    lag.push_back((((dy0 + i) & MSK) << lg) | ((dx0 + j) & MSK));
                    pair.push_back(a * A + b);
                    w.push_back(make_float2(float(v.real()), float(v.imag())));
                }
        }
    }
    // counting sort by lag cell
    std::vector<int> lptr((size_t)NP * NP + 1, 0);
    for (int l : lag) lptr[(size_t)l + 1]++;
    for (size_t i = 0; i + 1 < lptr.size(); ++i) lptr[i + 1] += lptr[i];
    std::vector<int> fill(lptr.begin(), lptr.end() - 1);
    const int cp = p->n_chan * p->n_pol;
    std::vector<int4> sent(pair.size());
    for (size_t i = 0; i < lag.size(); ++i) {
        int wr, wi;
        std::memcpy(&wr, &w[i].x, sizeof(float));
        std::memcpy(&wi, &w[i].y, sizeof(float));
        sent[fill[lag[i]]++] = make_int4(wr, wi, pair[i] * cp, 0);
    }
    cudaError_t e;
    if ((e = upload(&p->fx_lag_ptr, lptr)) != cudaSuccess || (e = upload(&p->fx_lag_ent, sent)) != cudaSuccess ||
        (e = cudaMalloc(&p->fx_vis_t, (size_t)A * A * cp * sizeof(float2))) != cudaSuccess ||
        (e = cudaMalloc(&p->fx_u, (size_t)cp * NP * NP * sizeof(float2))) != cudaSuccess) {
        cudaFree(p->fx_lag_ptr);
        cudaFree(p->fx_lag_ent);
        cudaFree(p->fx_vis_t);
        cudaFree(p->fx_u);
        p->fx_lag_ptr = nullptr;
        p->fx_lag_ent = nullptr;
        p->fx_vis_t = nullptr;
        p->fx_u = nullptr;
        return e == cudaErrorMemoryAllocation ? epic_fail(EPIC_ENOMEM, "FX lag table and scratch: %s", cudaGetErrorString(e))
                                              : epic_cuda_fail(e, "FX lag table upload");
    }
    p->fx_lag_n = (int64_t)sent.size();
    return EPIC_OK;
}

}  // namespace

epic_status epic_set_wait_limit(epic_plan* plan, int tries) {
    epic_clear_error();
    if (!plan) return epic_fail(EPIC_EINVAL, "plan is NULL");
    if (tries < 0 || tries > 1000000) return epic_fail(EPIC_EINVAL, "tries = %d outside 0..1000000", tries);
    plan->wait_tries = tries;
    return EPIC_OK;
}

epic_status epic_sync(const epic_plan* plan, void* stream) {
    EpicRange range("epic_sync");
    epic_clear_error();
    if (!plan) return epic_fail(EPIC_EINVAL, "plan is NULL");
    EpicDeviceGuard guard(plan->device);
    if (!guard.ok) return epic_fail(EPIC_ECUDA, "cannot select CUDA device %d", plan->device);
    cudaError_t e = cudaStreamSynchronize(static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return epic_cuda_fail(e, "stream synchronize");
    int word = 0;
    if ((e = cudaMemcpy(&word, plan->status, sizeof(int), cudaMemcpyDeviceToHost)) != cudaSuccess)
        return epic_cuda_fail(e, "status word read");
    if (word == 0) return EPIC_OK;
    if ((e = cudaMemset(plan->status, 0, sizeof(int))) != cudaSuccess) return epic_cuda_fail(e, "status word clear");
    std::string where;
    if (word & epic::kStatusImageTimeout) where += "tensor-core imaging kernel";
    if (word & epic::kStatusCorrelateTimeout) where += std::string(where.empty() ? "" : " and the ") + "correlator";
    if (word & epic::kStatusClusterTimeout)
        where += std::string(where.empty() ? "" : " and the ") + "cluster exchange of the FFT imaging kernel";
    return epic_fail(EPIC_ETIMEOUT, "a bounded wait ran out in the %s (its outputs are undefined)", where.c_str());
}

epic_status epic_set_transform(epic_plan* plan, int xform) {
    epic_clear_error();
    if (!plan) return epic_fail(EPIC_EINVAL, "plan is NULL");
    if (xform == EPIC_XFORM_FFT) {
        plan->xform = xform;
        return EPIC_OK;
    }
    if (xform == EPIC_XFORM_FFT_TWOPASS) {
        if (plan->n_pad != 512)
            return epic_fail(EPIC_EUNSUPPORTED, "the two-pass FFT form exists for n_pad 512 only (plan: %d)", plan->n_pad);
        EpicDeviceGuard guard(plan->device);
        if (!guard.ok) return epic_fail(EPIC_ECUDA, "cannot select CUDA device %d", plan->device);
        int smem_optin = 0;
        cudaDeviceGetAttribute(&smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, plan->device);
        if (epic::twopass_rows_smem_bytes(plan->n_ant) > (size_t)smem_optin)
            return epic_fail(EPIC_EUNSUPPORTED, "%d antennas do not fit the two-pass row kernel's shared memory",
                             plan->n_ant);
        if (!plan->tp_scratch) {
            const int chunk = 4 * plan->n_sm;
            cudaError_t e = cudaMalloc(reinterpret_cast<void**>(&plan->tp_scratch), epic::twopass_scratch_bytes(chunk));
            if (e != cudaSuccess) {
                plan->tp_scratch = nullptr;
                return e == cudaErrorMemoryAllocation ? epic_fail(EPIC_ENOMEM, "two-pass scratch: %s", cudaGetErrorString(e))
                                                      : epic_cuda_fail(e, "two-pass scratch");
            }
            plan->tp_chunk = chunk;
        }
        plan->xform = xform;
        return EPIC_OK;
    }
    if (xform != EPIC_XFORM_DFTGEMM && xform != EPIC_XFORM_DFTGEMM_FP16 && xform != EPIC_XFORM_DFTGEMM_FP16_GRID)
        return epic_fail(EPIC_EINVAL, "xform %d", xform);
    if (plan->n_pad != 128 && plan->n_pad != 256)
        return epic_fail(EPIC_EUNSUPPORTED, "the tensor-core transform needs n_pad 128 or 256 (plan: %d)", plan->n_pad);
    if (xform == EPIC_XFORM_DFTGEMM_FP16 && plan->n_pad != 128)
        return epic_fail(EPIC_EUNSUPPORTED, "the reduced-precision tensor-core form exists for n_pad 128 only (plan: %d)",
                         plan->n_pad);
    if (xform == EPIC_XFORM_DFTGEMM_FP16_GRID && plan->n_pad != 256)
        return epic_fail(EPIC_EUNSUPPORTED, "the FP16-gridding tensor-core form exists for n_pad 256 only (plan: %d)",
                         plan->n_pad);
    if (!plan->dg_lane)
        return epic_fail(EPIC_EUNSUPPORTED, "a pair of grid cells has more than 65535 mapping entries, or more than "
                                            "65536 antennas");
    if (xform == EPIC_XFORM_DFTGEMM_FP16_GRID && !plan->dg_wim && !plan->dg_wpk)
        return epic_fail(EPIC_EUNSUPPORTED, "the plan has no packed FP16 gather entries");
    EpicDeviceGuard guard(plan->device);
    if (!guard.ok) return epic_fail(EPIC_ECUDA, "cannot select CUDA device %d", plan->device);
    int smem_optin = 0;
    cudaDeviceGetAttribute(&smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, plan->device);
    const size_t dg_need = plan->n_pad == 128
                               ? epic::dftgemm_smem_bytes(plan->n_ant, false, xform == EPIC_XFORM_DFTGEMM_FP16)
                               : epic::dftgemm256_smem_bytes(plan->n_ant);
    if (dg_need > (size_t)smem_optin)
        return epic_fail(EPIC_EUNSUPPORTED, "%d antennas do not fit the tensor-core kernel's shared memory", plan->n_ant);
    if (!plan->dg_tab) {
        std::vector<uint16_t> tab;
        if (plan->n_pad == 128)
            epic::dftgemm_tables(tab);
        else
            epic::dftgemm256_tables(tab);
        cudaError_t e = upload(&plan->dg_tab, tab);
        if (e != cudaSuccess) {
            cudaFree(plan->dg_tab);
            plan->dg_tab = nullptr;
            return epic_cuda_fail(e, "DFT operand tables");
        }
    }
    plan->xform = xform;
    return EPIC_OK;
}

void epic_destroy(epic_plan* plan) {
    if (!plan) return;
    EpicDeviceGuard guard(plan->device);
    free_plan(plan);
}

epic_status epic_plan_info(const epic_plan* plan, int64_t* nnz, int64_t* n_cells, int* lag_side) {
    epic_clear_error();
    if (!plan) return epic_fail(EPIC_EINVAL, "plan is NULL");
    if (nnz) *nnz = plan->nnz;
    if (n_cells) *n_cells = plan->n_cells;
    if (lag_side) *lag_side = plan->lag_side;
    return EPIC_OK;
}

epic_status epic_image(const epic_plan* plan, const void* volt, int n_time, const float* gains,
                       double* accum, double* power, int64_t t_prev, float* image, float* autocorr,
                       void* stream) {
    EpicRange range("epic_image");
    epic_clear_error();
    if (!plan) return epic_fail(EPIC_EINVAL, "plan is NULL");
    if (n_time < 1) return epic_fail(EPIC_EINVAL, "n_time = %d must be >= 1", n_time);
    if (!volt) return epic_fail(EPIC_EINVAL, "volt is NULL");
    if (!accum) return epic_fail(EPIC_EINVAL, "accum is NULL");
    if (t_prev < 0) return epic_fail(EPIC_EINVAL, "t_prev must be >= 0");
    if (autocorr && !power) return epic_fail(EPIC_EINVAL, "autocorr needs the power accumulator");
    if (autocorr && plan->lag_side == 0)
        return epic_fail(EPIC_EUNSUPPORTED, "footprints too wide for the auto-correlation tables");
    {
        const epic_status al = epic_check_alignment({{"volt", volt, epic_volt_bytes(plan->vdt)}, {"gains", gains, 8},
                                                     {"accum", accum, 8}, {"power", power, 8}, {"image", image, 4},
                                                     {"autocorr", autocorr, 4}});
        if (al != EPIC_OK) return al;
    }
    if ((long long)plan->n_chan * plan->n_pol * n_time > 2147483647LL)
        return epic_fail(EPIC_EUNSUPPORTED, "C * P * T must stay below 2^31 per call");
    EpicDeviceGuard guard(plan->device);
    if (!guard.ok) return epic_fail(EPIC_ECUDA, "cannot select CUDA device %d", plan->device);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int cp = plan->n_chan * plan->n_pol;
    const size_t npix = (size_t)cp * plan->n_pad * plan->n_pad;
    cudaError_t e;
    if (t_prev == 0) {
        if ((e = cudaMemsetAsync(accum, 0, npix * sizeof(double), st)) != cudaSuccess) return epic_cuda_fail(e, "memset accum");
        if (power && (e = cudaMemsetAsync(power, 0, (size_t)cp * plan->n_ant * sizeof(double), st)) != cudaSuccess)
            return epic_cuda_fail(e, "memset power");
    }
    const epic::FwdArgs a =
        epic_plan_fwd_args(plan, volt, n_time, reinterpret_cast<const float2*>(gains), accum, power);
    epic_status s;
    if (plan->xform == EPIC_XFORM_DFTGEMM || plan->xform == EPIC_XFORM_DFTGEMM_FP16 ||
        plan->xform == EPIC_XFORM_DFTGEMM_FP16_GRID) {
        const epic::DgGather g{plan->dg_lane, plan->dg_base, plan->dg_wre, plan->dg_wim, plan->dg_ant, (int)plan->nnz,
                               plan->dg_wpk};
        e = plan->n_pad == 128 ? epic::launch_dftgemm(plan->vdt, a, plan->dg_tab, g, plan->n_sm, st, false,
                                                      plan->xform == EPIC_XFORM_DFTGEMM_FP16)
                               : epic::launch_dftgemm256(plan->vdt, a, plan->dg_tab, g, plan->n_sm, st,
                                                         plan->xform == EPIC_XFORM_DFTGEMM_FP16_GRID);
        s = e == cudaSuccess ? EPIC_OK : epic_cuda_fail(e, "tensor-core imaging kernel launch");
    } else if (plan->xform == EPIC_XFORM_FFT_TWOPASS) {
        epic::SegList L;
        L.seg[0] = a;
        L.first[0] = 0;
        L.first[1] = (int)a.n_items;
        L.weight[0] = 1;
        L.cost[0] = 0;
        L.cost[1] = a.n_items;
        L.n_seg = 1;
        L.max_ant = a.n_ant;
        L.max_workers = 0;
        e = epic::launch_fwd512_twopass(plan->vdt, L, plan->n_sm, st, plan->tp_scratch, plan->tp_chunk);
        s = e == cudaSuccess ? EPIC_OK : epic_cuda_fail(e, "two-pass imaging kernels launch");
    } else {
        s = launch_fwd(plan, a, st);
    }
    if (s != EPIC_OK) return s;
    const double inv_t = 1.0 / double(t_prev + n_time);
    if (image && (e = epic::launch_finalize_image(accum, image, (long long)npix, inv_t, st)) != cudaSuccess)
        return epic_cuda_fail(e, "image epilogue");
    if (autocorr && (e = epic::launch_autocorr(power, plan->lag_tab, cp, plan->n_ant, plan->lag_side, plan->n_pad,
                                               inv_t, autocorr, st)) != cudaSuccess)
        return epic_cuda_fail(e, "auto-correlation epilogue");
    return EPIC_OK;
}

epic_status epic_image_backward(const epic_plan* plan, const void* volt, int n_time, const float* gains,
                                const float* grad_image, float* grad_gains, void* stream) {
    EpicRange range("epic_image_backward");
    epic_clear_error();
    if (!plan) return epic_fail(EPIC_EINVAL, "plan is NULL");
    if (n_time < 1) return epic_fail(EPIC_EINVAL, "n_time = %d must be >= 1", n_time);
    if (!volt || !grad_image || !grad_gains) return epic_fail(EPIC_EINVAL, "NULL device array");
    {
        const epic_status al = epic_check_alignment({{"volt", volt, epic_volt_bytes(plan->vdt)}, {"gains", gains, 8},
                                                     {"grad_image", grad_image, 4}, {"grad_gains", grad_gains, 8}});
        if (al != EPIC_OK) return al;
    }
    if ((long long)plan->n_chan * plan->n_pol * n_time > 2147483647LL)
        return epic_fail(EPIC_EUNSUPPORTED, "C * P * T must stay below 2^31 per call");
    EpicDeviceGuard guard(plan->device);
    if (!guard.ok) return epic_fail(EPIC_ECUDA, "cannot select CUDA device %d", plan->device);
    int smem_optin = 0;
    cudaDeviceGetAttribute(&smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, plan->device);
    if (epic::bwd_smem_bytes(plan->n_pad, plan->n_ant) > (size_t)smem_optin)
        return epic_fail(EPIC_EUNSUPPORTED, "%d antennas do not fit the adjoint kernel's shared memory at n_pad %d",
                         plan->n_ant, plan->n_pad);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int cp = plan->n_chan * plan->n_pol;
    cudaError_t e = cudaMemsetAsync(grad_gains, 0, (size_t)cp * plan->n_ant * 2 * sizeof(float), st);
    if (e != cudaSuccess) return epic_cuda_fail(e, "memset grad_gains");
    epic::BwdArgs a;
    a.volt = volt;
    a.n_time = n_time;
    a.n_cp = cp;
    a.n_ant = plan->n_ant;
    a.gains = reinterpret_cast<const float2*>(gains);
    a.cell_ptr = plan->cell_ptr;
    a.cell_ent = plan->cell_ent;
    a.cell_wim = plan->cell_wim;
    a.ant_ptr = plan->ant_ptr;
    a.ant_ent = plan->ant_ent;
    a.ant_wim = plan->ant_wim;
    a.twiddle = plan->twiddle;
    a.grad_image = grad_image;
    a.grad_gains = reinterpret_cast<float2*>(grad_gains);
    a.n_items = (long long)cp * n_time;
    a.scale = float(2.0 / double(n_time));
    return launch_bwd(plan, a, st);
}

epic_status epic_image_xpol(const epic_plan* plan, const void* volt, int n_time, const float* gains,
                            double* accum4, int64_t t_prev, float* image, float* cross, void* stream) {
    EpicRange range("epic_image_xpol");
    epic_clear_error();
    if (!plan) return epic_fail(EPIC_EINVAL, "plan is NULL");
    if (plan->n_pol != 2) return epic_fail(EPIC_EINVAL, "cross-polarisation images need a plan with 2 pols (has %d)", plan->n_pol);
    if (n_time < 1) return epic_fail(EPIC_EINVAL, "n_time = %d must be >= 1", n_time);
    if (!volt || !accum4) return epic_fail(EPIC_EINVAL, "NULL device array");
    {
        const epic_status al = epic_check_alignment({{"volt", volt, epic_volt_bytes(plan->vdt)}, {"gains", gains, 8},
                                                     {"accum4", accum4, 8}, {"image", image, 4}, {"cross", cross, 8}});
        if (al != EPIC_OK) return al;
    }
    if (t_prev < 0) return epic_fail(EPIC_EINVAL, "t_prev must be >= 0");
    if ((long long)plan->n_chan * 4 * n_time > 2147483647LL)
        return epic_fail(EPIC_EUNSUPPORTED, "4 * C * T must stay below 2^31 per call");
    EpicDeviceGuard guard(plan->device);
    if (!guard.ok) return epic_fail(EPIC_ECUDA, "cannot select CUDA device %d", plan->device);
    int smem_optin = 0;
    cudaDeviceGetAttribute(&smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, plan->device);
    if (plan->xform == EPIC_XFORM_DFTGEMM_FP16 || plan->xform == EPIC_XFORM_FFT_TWOPASS ||
        plan->xform == EPIC_XFORM_DFTGEMM_FP16_GRID)
        return epic_fail(EPIC_EUNSUPPORTED, "the %s form has no cross-polarisation variant; use EPIC_XFORM_FFT%s",
                         plan->xform == EPIC_XFORM_FFT_TWOPASS ? "two-pass" : "reduced-precision tensor-core",
                         plan->xform == EPIC_XFORM_FFT_TWOPASS ? "" : " or EPIC_XFORM_DFTGEMM");
    const bool dg = plan->xform == EPIC_XFORM_DFTGEMM;
    if (dg && plan->n_pad != 128)
        return epic_fail(EPIC_EUNSUPPORTED, "the tensor-core cross-polarisation form exists for n_pad 128 only; "
                                            "use the FFT form (epic_set_transform) at n_pad %d", plan->n_pad);
    if ((dg ? epic::dftgemm_smem_bytes(plan->n_ant, true) : epic::fwd_xpol_smem_bytes(plan->n_pad, plan->n_ant)) >
        (size_t)smem_optin)
        return epic_fail(EPIC_EUNSUPPORTED, "%d antennas do not fit the %s cross-polarisation kernel's shared memory",
                         plan->n_ant, dg ? "tensor-core" : "FFT");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const long long npix = (long long)plan->n_pad * plan->n_pad;
    cudaError_t e;
    if (t_prev == 0 && (e = cudaMemsetAsync(accum4, 0, (size_t)plan->n_chan * 4 * npix * sizeof(double), st)) != cudaSuccess)
        return epic_cuda_fail(e, "memset accum4");
    epic::FwdArgs a = epic_plan_fwd_args(plan, volt, n_time, reinterpret_cast<const float2*>(gains), accum4, nullptr);
    a.n_cp = plan->n_chan * 4;          // virtual pols X, Y, X + Y, X + iY per channel
    a.n_items = (long long)a.n_cp * n_time;
    epic_status s;
    if (dg) {
        const epic::DgGather g{plan->dg_lane, plan->dg_base, plan->dg_wre, plan->dg_wim, plan->dg_ant, (int)plan->nnz};
        e = epic::launch_dftgemm(plan->vdt, a, plan->dg_tab, g, plan->n_sm, st, true);
        s = e == cudaSuccess ? EPIC_OK : epic_cuda_fail(e, "tensor-core cross-polarisation kernel launch");
    } else {
        s = launch_fwd(plan, a, st, true);
    }
    if (s != EPIC_OK) return s;
    if ((e = epic::launch_finalize_xpol(accum4, image, reinterpret_cast<float2*>(cross), plan->n_chan, npix,
                                        1.0 / double(t_prev + n_time), st)) != cudaSuccess)
        return epic_cuda_fail(e, "cross-polarisation epilogue");
    return EPIC_OK;
}

epic_status epic_fengine(int n_ant, int n_pol, int n_chan, int n_time, int in_dtype, const void* raw, int out_dtype,
                         void* volt, int device, void* stream) {
    EpicRange range("epic_fengine");
    epic_clear_error();
    if (n_ant < 1 || n_pol < 1 || n_time < 0) return epic_fail(EPIC_EINVAL, "bad sizes");
    if (n_chan != 32 && n_chan != 64 && n_chan != 128 && n_chan != 256 && n_chan != 512)
        return epic_fail(EPIC_EUNSUPPORTED, "n_chan = %d (supported: 32, 64, 128, 256, 512)", n_chan);
    if (in_dtype < EPIC_VOLT_C64 || in_dtype > EPIC_VOLT_CI4) return epic_fail(EPIC_EINVAL, "in_dtype %d", in_dtype);
    if (out_dtype != EPIC_VOLT_C64 && out_dtype != EPIC_VOLT_F16)
        return epic_fail(EPIC_EINVAL, "out_dtype %d (complex64 or FP16 pairs)", out_dtype);
    if (n_time == 0) return EPIC_OK;
    if (!raw || !volt) return epic_fail(EPIC_EINVAL, "NULL device array");
    {
        const epic_status al = epic_check_alignment({{"raw", raw, epic_volt_bytes(in_dtype)},
                                                     {"volt", volt, epic_volt_bytes(out_dtype)}});
        if (al != EPIC_OK) return al;
    }
    EpicDeviceGuard guard(device);
    if (!guard.ok) return epic_fail(EPIC_ECUDA, "cannot select CUDA device %d", device);
    int n_sm = 0;
    cudaError_t e = cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, device);
    if (e != cudaSuccess) return epic_cuda_fail(e, "cudaDeviceGetAttribute");
    epic::FengArgs a;
    a.raw = raw;
    a.volt = volt;
    a.n_time = n_time;
    a.n_pol = n_pol;
    a.n_ant = n_ant;
    e = epic::launch_fengine(n_chan, in_dtype, out_dtype == EPIC_VOLT_F16 ? 1 : 0, a, n_sm,
                             static_cast<cudaStream_t>(stream));
    return e == cudaSuccess ? EPIC_OK : epic_cuda_fail(e, "F-engine kernel launch");
}

epic_status epic_weff(const epic_plan* plan, float* weff, void* stream) {
    EpicRange range("epic_weff");
    epic_clear_error();
    if (!plan) return epic_fail(EPIC_EINVAL, "plan is NULL");
    if (!weff) return epic_fail(EPIC_EINVAL, "weff is NULL");
    if (epic_check_alignment({{"weff", weff, 4}}) != EPIC_OK) return EPIC_EINVAL;
    if (plan->n_ant < 2) return epic_fail(EPIC_EINVAL, "the effective weighting needs at least two antennas");
    if (plan->lag_side == 0)
        return epic_fail(EPIC_EUNSUPPORTED, "footprints too wide for the auto-correlation tables");
    EpicDeviceGuard guard(plan->device);
    if (!guard.ok) return epic_fail(EPIC_ECUDA, "cannot select CUDA device %d", plan->device);
    int smem_optin = 0;
    cudaDeviceGetAttribute(&smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, plan->device);
    if (epic::weff_smem_bytes(plan->lag_side, plan->n_pad) > (size_t)smem_optin)
        return epic_fail(EPIC_EUNSUPPORTED, "lag window %d does not fit the effective-weighting kernel", plan->lag_side);
    const cudaError_t e = epic::launch_weff(plan->lag_tab, plan->n_ant, plan->lag_side, plan->n_pad, weff,
                                            static_cast<cudaStream_t>(stream));
    return e == cudaSuccess ? EPIC_OK : epic_cuda_fail(e, "effective-weighting kernel launch");
}

epic_status epic_isotropic(const epic_plan* plan, const float* image, const float* autocorr, const float* weff,
                           float rel_floor, float* iso, void* stream) {
    EpicRange range("epic_isotropic");
    epic_clear_error();
    if (!plan) return epic_fail(EPIC_EINVAL, "plan is NULL");
    if (!image || !autocorr || !weff || !iso) return epic_fail(EPIC_EINVAL, "NULL device array");
    {
        const epic_status al = epic_check_alignment({{"image", image, 4}, {"autocorr", autocorr, 4},
                                                     {"weff", weff, 4}, {"iso", iso, 4}});
        if (al != EPIC_OK) return al;
    }
    if (plan->n_ant < 2) return epic_fail(EPIC_EINVAL, "the isotropic estimate needs at least two antennas");
    if (!(rel_floor >= 0.f) || !(rel_floor < 1.f)) return epic_fail(EPIC_EINVAL, "rel_floor must be in [0, 1)");
    EpicDeviceGuard guard(plan->device);
    if (!guard.ok) return epic_fail(EPIC_ECUDA, "cannot select CUDA device %d", plan->device);
    const int npix = plan->n_pad * plan->n_pad;
    const long long n = (long long)plan->n_chan * plan->n_pol * npix;
    const cudaError_t e = epic::launch_isotropic(image, autocorr, weff, rel_floor, plan->n_ant, n, npix, iso,
                                                 static_cast<cudaStream_t>(stream));
    return e == cudaSuccess ? EPIC_OK : epic_cuda_fail(e, "isotropic-estimate kernel launch");
}

epic_status epic_correlate(const epic_plan* plan, const void* volt, int n_time, const float* gains, float* vis,
                           void* stream) {
    EpicRange range("epic_correlate");
    epic_clear_error();
    if (!plan) return epic_fail(EPIC_EINVAL, "plan is NULL");
    if (n_time < 1) return epic_fail(EPIC_EINVAL, "n_time = %d must be >= 1", n_time);
    if (!volt || !vis) return epic_fail(EPIC_EINVAL, "NULL device array");
    {
        const epic_status al = epic_check_alignment({{"volt", volt, epic_volt_bytes(plan->vdt)}, {"gains", gains, 8},
                                                     {"vis", vis, 8}});
        if (al != EPIC_OK) return al;
    }
    if (plan->vdt == EPIC_VOLT_C64)
        return epic_fail(EPIC_EUNSUPPORTED, "the correlator takes FP16 or 4+4-bit voltages (exact FP16 operands)");
    if (n_time > 131072) return epic_fail(EPIC_EUNSUPPORTED, "n_time = %d: at most 131072 samples per call", n_time);
    EpicDeviceGuard guard(plan->device);
    if (!guard.ok) return epic_fail(EPIC_ECUDA, "cannot select CUDA device %d", plan->device);
    int smem_optin = 0;
    cudaDeviceGetAttribute(&smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, plan->device);
    if (epic::xeng_smem_bytes() > (size_t)smem_optin) return epic_fail(EPIC_EUNSUPPORTED, "shared memory");
    epic::XengArgs a;
    a.volt = volt;
    a.n_time = n_time;
    a.n_cp = plan->n_chan * plan->n_pol;
    a.n_ant = plan->n_ant;
    a.gains = reinterpret_cast<const float2*>(gains);
    a.vis = reinterpret_cast<float2*>(vis);
    a.status = plan->status;
    a.wait_tries = plan->wait_tries;
    const cudaError_t e = epic::launch_xeng(plan->vdt, a, plan->n_sm, static_cast<cudaStream_t>(stream));
    return e == cudaSuccess ? EPIC_OK : epic_cuda_fail(e, "correlator kernel launch");
}

epic_status epic_fx_image(const epic_plan* plan, const float* vis, float* image, void* stream) {
    EpicRange range("epic_fx_image");
    epic_clear_error();
    if (!plan) return epic_fail(EPIC_EINVAL, "plan is NULL");
    if (!vis || !image) return epic_fail(EPIC_EINVAL, "NULL device array");
    {
        const epic_status al = epic_check_alignment({{"vis", vis, 8}, {"image", image, 4}});
        if (al != EPIC_OK) return al;
    }
    if (plan->n_pad > 128 || !plan->fx_ptr)
        return epic_fail(EPIC_EUNSUPPORTED, "the FX imaging kernel holds the lag plane in shared memory: n_pad <= 128");
    EpicDeviceGuard guard(plan->device);
    if (!guard.ok) return epic_fail(EPIC_ECUDA, "cannot select CUDA device %d", plan->device);
    {
        std::lock_guard<std::mutex> lock(g_fx_lag_mu);
        if (plan->fx_lag_n < 0) {
            const epic_status st = build_fx_lag_table(plan);
            if (st != EPIC_OK) return st;
        }
    }
    epic::FxArgs a;
    a.vis = reinterpret_cast<const float2*>(vis);
    a.n_cp = plan->n_chan * plan->n_pol;
    a.n_ant = plan->n_ant;
    a.lag_ptr = plan->fx_lag_ptr;
    a.lag_ent = plan->fx_lag_ent;
    a.vis_t = plan->fx_vis_t;
    a.u = plan->fx_u;
    a.image = image;
    const cudaError_t e = epic::launch_fx_image(plan->n_pad, a, static_cast<cudaStream_t>(stream));
    return e == cudaSuccess ? EPIC_OK : epic_cuda_fail(e, "FX imaging kernel launch");
}

epic_status epic_grid(const epic_plan* plan, const void* volt, int n_time, const float* gains, float* grid,
                      void* stream) {
    EpicRange range("epic_grid");
    epic_clear_error();
    if (!plan) return epic_fail(EPIC_EINVAL, "plan is NULL");
    if (n_time < 1) return epic_fail(EPIC_EINVAL, "n_time = %d must be >= 1", n_time);
    if (!volt || !grid) return epic_fail(EPIC_EINVAL, "NULL device array");
    {
        const epic_status al = epic_check_alignment({{"volt", volt, epic_volt_bytes(plan->vdt)}, {"gains", gains, 8},
                                                     {"grid", grid, 8}});
        if (al != EPIC_OK) return al;
    }
    if ((long long)plan->n_chan * plan->n_pol * n_time > 2147483647LL)
        return epic_fail(EPIC_EUNSUPPORTED, "C * P * T must stay below 2^31 per call");
    EpicDeviceGuard guard(plan->device);
    if (!guard.ok) return epic_fail(EPIC_ECUDA, "cannot select CUDA device %d", plan->device);
    int smem_optin = 0;
    cudaDeviceGetAttribute(&smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, plan->device);
    const int tb = epic::grid_samples_per_unit(plan->n_ant, (size_t)smem_optin);
    if (epic::grid_smem_bytes(plan->n_ant, tb) > (size_t)smem_optin)
        return epic_fail(EPIC_EUNSUPPORTED, "%d antennas do not fit the gridder's shared memory", plan->n_ant);
    epic::GridArgs a;
    a.volt = volt;
    a.n_time = n_time;
    a.n_cp = plan->n_chan * plan->n_pol;
    a.n_ant = plan->n_ant;
    a.gains = reinterpret_cast<const float2*>(gains);
    a.cell_ptr = plan->cell_ptr;
    a.cell_ent = plan->cell_ent;
    a.cell_wim = plan->cell_wim;
    a.nnz = (int)plan->nnz;
    a.csr_width = plan->n_pad / 2;
    a.n_grid = plan->n_grid;
    a.out = reinterpret_cast<float2*>(grid);
    const cudaError_t e = epic::launch_grid(plan->vdt, tb, a, plan->n_sm, static_cast<cudaStream_t>(stream));
    return e == cudaSuccess ? EPIC_OK : epic_cuda_fail(e, "gridding kernel launch");
}

}  // extern "C"
