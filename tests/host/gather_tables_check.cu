// Host-only check of the tensor-core kernels' gridding slot tables (no GPU): builds them with the
// library's own builder from a cell-major mapping read from a text file (on the 64 x 64 grid of
// N_p = 128 with 16 warps, or the 128 x 128 grid of N_p = 256 with the warp count given as the
// second argument), then walks them the
// way the kernel's warps do (step k: lanes with more than k entries, contiguous run, start of
// step k + 1 = start of step k + active lanes) and checks that
//   every index stays inside the tables and every antenna inside the array,
//   every cell pair (x, y), (x, y + 1) is stored exactly once, at an in-range even offset,
//   the 32 lanes of a slot store to 32 distinct shared-memory banks,
//   lanes are in decreasing entry count, every slot is held by one position of some warp (a warp
//   holds at most ceil(slots / warps) of them: positions per warp; the rest have all-zero lanes
//   and base -1, the mark that makes the kernel skip them instead of storing their zero sums
//   over the cell pair at offset 0),
//   every cell's walked entries are a permutation of its mapping entries (the builder orders a
//   cell's entries to spread the antennas read at one step over shared-memory banks), and its
//   sum equals the sum of the same entries in the CSR order within FP32 rounding (a few units in
//   the last place of the sum of |w| |v|).
// Exit status 0 when every check holds.
#include "../../paper_1510_08318_gb300/csrc/moff_dftgemm.cu"
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <fstream>
#include <random>
#include <set>
#include <tuple>

int main(int argc, char** argv) {
    if (argc < 2) return 2;
    std::ifstream f(argv[1]);
    int ncell = 0, nnz = 0;
    f >> ncell >> nnz;
    const int NG = ncell == 64 * 64 ? 64 : ncell == 128 * 128 ? 128 : 0;   // the form's grid side
    if (NG == 0) return 2;
    const int NW = argc > 2 ? std::atoi(argv[2]) : 16;                       // gridding warps
    std::vector<int> cptr(ncell + 1), ant(nnz);
    std::vector<float> wr(nnz), wi(nnz);
    for (auto& v : cptr) f >> v;
    for (auto& v : ant) f >> v;
    for (auto& v : wr) f >> v;
    for (auto& v : wi) f >> v;
    std::vector<int2> cent(nnz);
    for (int i = 0; i < nnz; ++i) {
        int b;
        std::memcpy(&b, &wr[i], 4);
        cent[i] = int2{b, ant[i]};
    }
    int A = 1;
    for (int a : ant) A = std::max(A, a + 1);
    std::vector<int2> lane;
    std::vector<int> base;
    std::vector<float> wre, wim;
    std::vector<uint16_t> an;
    const bool ok = NG == 64 && NW == 16 ? epic::dftgemm_gather_tables(cptr, cent, wi, lane, base, wre, wim, an)
                                         : epic::dftgemm_gather_tables_ng(NG, NW, cptr, cent, wi, lane, base, wre,
                                                                          wim, an);
    if (!ok) {
        std::printf("builder refused the mapping\n");
        return 1;
    }
    const int ETAB = NG * NG, NSLOT = NG * NG / 64, PER = (NSLOT + NW - 1) / NW, NPOS = NW * PER;
    int bad = 0;
    if ((int)lane.size() != NPOS * 32 || (int)base.size() != NPOS || (int)wre.size() != nnz ||
        wim.size() != wre.size() || an.size() != wre.size()) {
        std::printf("table sizes\n");
        return 1;
    }
    std::mt19937 rng(7);
    std::uniform_real_distribution<float> U(-1.f, 1.f);
    std::vector<float2> VB(A);
    for (auto& v : VB) v = make_float2(U(rng), U(rng));
    std::vector<float2> E(ETAB, make_float2(0.f, 0.f));
    std::vector<int> seen(ETAB, 0);
    std::vector<std::vector<int>> walked(ETAB);   // table entries summed into each E^T element
    int used = 0;
    for (int slot = 0; slot < NPOS; ++slot) {
        // positions no slot took (when the slots do not divide evenly over the warps) carry base -1,
        // which the kernels skip, and all-zero lanes; every other position a base >= 0
        bool empty = true;
        for (int l = 0; l < 32; ++l) empty = empty && lane[slot * 32 + l].x == 0 && lane[slot * 32 + l].y == 0;
        if (base[slot] < 0) {
            if (!empty || base[slot] != -1) ++bad;
            continue;
        }
        if (empty) ++bad;
        ++used;
        int c0[32], cnt[32], e[32];
        unsigned banks = 0;
        for (int l = 0; l < 32; ++l) {
            const unsigned x = (unsigned)lane[slot * 32 + l].x;
            c0[l] = x & 0xffff;
            cnt[l] = x >> 16;
            if (c0[l] > cnt[l] || (l > 0 && cnt[l] > cnt[l - 1])) ++bad;
            const int off = lane[slot * 32 + l].y;
            if (off < 0 || off + 1 >= ETAB || (off & 1)) { ++bad; continue; }
            banks |= 1u << ((off / 2) % 32);
            e[l] = base[slot] + l;
        }
        if (banks != 0xffffffffu) ++bad;
        float2 s0[32], s1[32];
        std::vector<int> w0s[32], w1s[32];
        for (int l = 0; l < 32; ++l) s0[l] = s1[l] = make_float2(0.f, 0.f);
        for (int k = 0; k < cnt[0]; ++k) {
            int nk = 0;
            for (int l = 0; l < 32; ++l) nk += k < cnt[l];
            for (int l = 0; l < nk; ++l) {
                if (e[l] < 0 || e[l] >= (int)wre.size() || an[e[l]] >= A) { ++bad; continue; }
                const float w0 = k < c0[l] ? wre[e[l]] : 0.f, w1 = wre[e[l]] - w0;   // as the kernel
                const float wi0 = k < c0[l] ? wim[e[l]] : 0.f, wi1 = wim[e[l]] - wi0;
                const float2 v = VB[an[e[l]]];
                float2& s = k < c0[l] ? s0[l] : s1[l];
                const float w = k < c0[l] ? w0 : w1, wq = k < c0[l] ? wi0 : wi1;
                s.x = fmaf(w, v.x, fmaf(-wq, v.y, s.x));
                s.y = fmaf(w, v.y, fmaf(wq, v.x, s.y));
                (k < c0[l] ? w0s[l] : w1s[l]).push_back(e[l]);
            }
            for (int l = 0; l < 32; ++l) e[l] += nk;
        }
        for (int l = 0; l < 32; ++l) {
            const int off = lane[slot * 32 + l].y;
            if (off < 0 || off + 1 >= ETAB) continue;
            E[off] = s0[l];
            E[off + 1] = s1[l];
            seen[off] += 1;
            seen[off + 1] += 1;
            walked[off] = w0s[l];
            walked[off + 1] = w1s[l];
        }
    }
    if (used != NSLOT) ++bad;
    // the reference: each cell's entries as a multiset (antenna, weight), and its sum in the order
    // of the CSR, which the walked sum must match within FP32 rounding of the absolute sum
    int miss = 0, perm = 0, far = 0;
    double maxrel = 0.0;
    auto key = [](int a, float r, float i) {
        unsigned br, bi;
        std::memcpy(&br, &r, 4);
        std::memcpy(&bi, &i, 4);
        return std::make_tuple(a, br, bi);
    };
    for (int y = 0; y < NG; ++y)
        for (int x = 0; x < NG; ++x) {
            const int c = y * NG + x, off = epic::tc::koff(x, y, NG);
            if (seen[off] != 1) { ++miss; continue; }
            std::vector<std::tuple<int, unsigned, unsigned>> want, got;
            for (int i = cptr[c]; i < cptr[c + 1]; ++i) want.push_back(key(ant[i], wr[i], wi[i]));
            for (int e : walked[off]) got.push_back(key(an[e], wre[e], wim[e]));
            std::sort(want.begin(), want.end());
            std::sort(got.begin(), got.end());
            if (want != got) ++perm;
            float2 s = make_float2(0.f, 0.f);
            double mag = 0.0;
            for (int i = cptr[c]; i < cptr[c + 1]; ++i) {
                const float2 v = VB[ant[i]];
                s.x = fmaf(wr[i], v.x, fmaf(-wi[i], v.y, s.x));
                s.y = fmaf(wr[i], v.y, fmaf(wi[i], v.x, s.y));
                mag += std::hypot((double)wr[i], (double)wi[i]) * std::hypot((double)v.x, (double)v.y);
            }
            const double d = std::max(std::fabs(E[off].x - s.x), std::fabs(E[off].y - s.y));
            // each FMA rounds once (relative 2^-24): 2 per entry and component, so 4 n 2^-24 of
            // the absolute sum bounds any reordering's difference
            const double bound = 4.0 * (cptr[c + 1] - cptr[c]) * std::ldexp(mag, -24);
            if (d > bound) ++far;
            if (mag > 0) maxrel = std::max(maxrel, d / mag);
        }
    std::printf("bad %d missing %d not-a-permutation %d beyond-rounding %d max |diff| / sum|w v| %g\n", bad, miss,
                perm, far, maxrel);
    return (bad || miss || perm || far) ? 1 : 0;
}
