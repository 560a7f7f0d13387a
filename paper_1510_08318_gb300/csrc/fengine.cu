// F-engine (Sec. 3 "Temporal Fourier transform"): the time samples of every antenna are
// Fourier transformed, block by block, into electric-field spectra that feed the imaging:
//   V[t][c][p][a] = sum_{j < C} x[(t C + j)][p][a] exp(-2 pi i j c / C),   c = 0 .. C-1,
// an unnormalised forward DFT of each block of C consecutive samples (bins in FFT order:
// c > C/2 are the negative frequencies), no window.
//
// One CTA per (block t, pol, tile of 32 antennas) at a time, transformed along time with
// C = R1 R2 (Cooley-Tukey): thread (antenna, n1) loads samples n1 + R2 n2 of its antenna into
// registers (coalesced: antennas contiguous; the next unit's while this one is processed),
// does their R1-point DFT there, twiddles by exp(-2 pi i n1 k2 / C) and writes the results to
// shared memory; then each thread does R2-point DFTs of (antenna, k2) and writes bins
// k2 + R1 k1 with coalesced stores.  HBM-bound: it reads the raw samples once and writes the
// spectra once; shared memory sees one write and one read per value.  For C <= 128 and an even
// antenna count a thread takes two adjacent antennas as packed FP32 pairs (fengine2_kernel).
#include <cuda_fp16.h>
#include "moff_common.cuh"

namespace epic {
namespace fe {

constexpr int TA = 32;   // antennas per tile

template <int C> struct Split;
template <> struct Split<32>  { static constexpr int R2 = 4; };
template <> struct Split<64>  { static constexpr int R2 = 8; };
template <> struct Split<128> { static constexpr int R2 = 8; };
template <> struct Split<256> { static constexpr int R2 = 16; };
template <> struct Split<512> { static constexpr int R2 = 16; };

template <int C>
constexpr size_t smem_bytes() { return sizeof(float2) * ((size_t)C * TA + C); }

template <int OUT> struct Out;
template <> struct Out<0> {       // complex64
    using T = float2;
    static __device__ __forceinline__ T enc(float2 v) { return v; }
};
template <> struct Out<1> {       // FP16 pair
    using T = __half2;
    static __device__ __forceinline__ T enc(float2 v) { return __floats2half2_rn(v.x, v.y); }
};

template <int C, int VIN, int OUT>
__global__ void __launch_bounds__(TA * Split<C>::R2, (TA * Split<C>::R2 <= 256) ? 3 : 1) fengine_kernel(const FengArgs a) {
    constexpr int R2 = Split<C>::R2, R1 = C / R2, NT = TA * R2;
    static_assert(R1 >= R2 && R1 <= 64 && R1 % R2 == 0, "split");
    using VT = typename Volt<VIN>::T;
    using OT = typename Out<OUT>::T;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float2* X = reinterpret_cast<float2*>(smem_raw);     // [C][TA]
    float2* TW = X + C * TA;                             // [C] exp(-2 pi i j / C)
    const int tid = threadIdx.x, al = tid % TA, n1 = tid / TA;
    for (int j = tid; j < C; j += NT) {
        double s, c;
        sincospi(-2.0 * j / C, &s, &c);
        TW[j] = make_float2(float(c), float(s));
    }
    const int A = a.n_ant, P = a.n_pol;
    const int n_tiles = (A + TA - 1) / TA;
    const int n_units = a.n_time * P * n_tiles;   // < 2^31 (checked by the caller)
    const VT* raw = static_cast<const VT*>(a.raw);
    OT* out = static_cast<OT*>(a.volt);
    const long long row = (long long)P * A;       // elements from one sample (or bin) to the next
    // raw samples of a unit (rows n1 + R2 q of its block): the next unit's are loaded into
    // registers while the current one is transformed and stored.  Unit u = (t, p, tile) with
    // the tile fastest, kept as 32-bit coordinates: a step of gridDim.x units adds the stride's
    // own coordinates with carries (no divisions per unit).
    const int G = gridDim.x, g_tile = G % n_tiles, g_p = (G / n_tiles) % P, g_t = G / (n_tiles * P);
    auto step = [&](int& tile, int& p, int& t) {
        tile += g_tile;
        const int c1 = tile >= n_tiles;
        tile -= c1 ? n_tiles : 0;
        p += g_p + c1;
        const int c2 = p >= P;
        p -= c2 ? P : 0;
        t += g_t + c2;
    };
    VT nxt[R1];
    auto load_unit = [&](int tile, int p, int t) {
        const int ant = tile * TA + al;
        const VT* src = raw + ((long long)t * C + n1) * row + (long long)p * A + ant;
#pragma unroll
        for (int q = 0; q < R1; ++q) nxt[q] = ant < A ? __ldg(src + q * R2 * row) : VT{};
    };
    const int u0 = blockIdx.x;
    int tile = u0 % n_tiles, p = (u0 / n_tiles) % P, t = u0 / (n_tiles * P);
    if (u0 < n_units) load_unit(tile, p, t);
    for (int u = u0; u < n_units; u += G) {
        int ntile = tile, np = p, nt = t;         // coordinates of unit u + G
        step(ntile, np, nt);
        const int ant = tile * TA + al;
        // stage 1: R1-point DFT of samples n1 + R2 n2 (the rows this thread loaded, straight from
        // registers), then the twiddle exp(-2 pi i n1 k2 / C) on the way into shared memory
        {
            float2 x[R1];
#pragma unroll
            for (int q = 0; q < R1; ++q) x[q] = Volt<VIN>::dec(nxt[q]);
            if (u + G < n_units) load_unit(ntile, np, nt);
            dft<R1, -1>(x);
            __syncthreads();                              // previous unit's stage-2 reads are done
#pragma unroll
            for (int k2 = 0; k2 < R1; ++k2) X[(n1 + R2 * k2) * TA + al] = cmul(x[k2], TW[n1 * k2]);   // n1 k2 < C
        }
        __syncthreads();
        // stage 2: for k2 = n1, n1 + R2, ...: R2-point DFT over n1' of the row n1' + R2 k2, bins
        // c = k2 + R1 k1
#pragma unroll
        for (int q = 0; q < R1 / R2; ++q) {
            const int k2 = n1 + R2 * q;
            float2 z[R2];
#pragma unroll
            for (int m = 0; m < R2; ++m) z[m] = X[(m + R2 * k2) * TA + al];
            dft<R2, -1>(z);
            if (ant < A) {
                OT* dst = out + ((long long)t * C + k2) * row + (long long)p * A + ant;
#pragma unroll
                for (int k1 = 0; k1 < R2; ++k1) dst[k1 * R1 * row] = Out<OUT>::enc(z[k1]);
            }
        }
        tile = ntile;
        p = np;
        t = nt;
    }
}

// ---- two antennas per thread (C <= 128, even antenna count) ----------------------------------
// The complex values of two adjacent antennas as packed FP32 pairs, re = (re_0, re_1) and
// im = (im_0, im_1), so that one f32x2 instruction does an operation for both antennas and the
// loads, stores, address arithmetic and twiddle loads of a thread serve two antennas.
struct P2 { unsigned long long re, im; };

__device__ __forceinline__ unsigned long long f2add(unsigned long long a, unsigned long long b) {
    unsigned long long r;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ unsigned long long f2sub(unsigned long long a, unsigned long long b) {
    unsigned long long r;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ unsigned long long f2mul(unsigned long long a, unsigned long long b) {
    unsigned long long r;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
// a * b + c, each lane rounded once
__device__ __forceinline__ unsigned long long f2fma(unsigned long long a, unsigned long long b, unsigned long long c) {
    unsigned long long r;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(a), "l"(b), "l"(c));
    return r;
}
__device__ __forceinline__ unsigned long long f2dup(float c) { return pack2(make_float2(c, c)); }

// (a - b) * exp(SIGN 2 pi i m / M) for a compile-time rotation; the half and quarter turns cost
// no multiplies (the swap and the sign go into the subtraction).
template <int SIGN>
__device__ __forceinline__ P2 sub_rot(const P2& a, const P2& b, int m, int M) {
    const int r = ((m % M) + M) % M;
    P2 d;
    if (r == 0) {
        d.re = f2sub(a.re, b.re);
        d.im = f2sub(a.im, b.im);
    } else if (2 * r == M) {
        d.re = f2sub(b.re, a.re);
        d.im = f2sub(b.im, a.im);
    } else if (4 * r == M || 4 * r == 3 * M) {
        if ((SIGN > 0) == (4 * r == M)) {      // times +i: (-(a - b).im, (a - b).re)
            d.re = f2sub(b.im, a.im);
            d.im = f2sub(a.re, b.re);
        } else {                               // times -i: ((a - b).im, -(a - b).re)
            d.re = f2sub(a.im, b.im);
            d.im = f2sub(b.re, a.re);
        }
    } else {
        const int idx = r * (64 / M);
        const float c = kTw64.c[idx], s = SIGN > 0 ? kTw64.s[idx] : -kTw64.s[idx];
        const unsigned long long dre = f2sub(a.re, b.re), dim = f2sub(a.im, b.im);
        d.re = f2fma(dre, f2dup(c), f2mul(dim, f2dup(-s)));
        d.im = f2fma(dre, f2dup(s), f2mul(dim, f2dup(c)));
    }
    return d;
}

// In-place x[k] <- sum_n x[n] exp(SIGN 2 pi i n k / N) for both antennas of every pair, N a power
// of two <= 64: radix-2 decimation in frequency, then a compile-time permutation.
template <int N, int SIGN>
__device__ __forceinline__ void dft2(P2 (&x)[N]) {
    if constexpr (N > 1) {
#pragma unroll
        for (int half = N / 2; half >= 1; half >>= 1) {
#pragma unroll
            for (int blk = 0; blk < N; blk += 2 * half) {
#pragma unroll
                for (int j = 0; j < half; ++j) {
                    const P2 a = x[blk + j], b = x[blk + j + half];
                    x[blk + j].re = f2add(a.re, b.re);
                    x[blk + j].im = f2add(a.im, b.im);
                    x[blk + j + half] = sub_rot<SIGN>(a, b, j, 2 * half);
                }
            }
        }
        P2 y[N];
#pragma unroll
        for (int k = 0; k < N; ++k) y[k] = x[bitrev<N>(k)];
#pragma unroll
        for (int k = 0; k < N; ++k) x[k] = y[k];
    }
}

// Raw samples of two adjacent antennas and their decode into a pair.
template <int VIN> struct Pair;
template <> struct Pair<0> {      // complex64: (re_0, im_0, re_1, im_1)
    using T = float4;
    static __device__ __forceinline__ P2 dec(T v) {
        return P2{pack2(make_float2(v.x, v.z)), pack2(make_float2(v.y, v.w))};
    }
};
template <> struct Pair<1> {      // FP16 pairs: (re_0, im_0), (re_1, im_1)
    using T = uint2;
    static __device__ __forceinline__ P2 dec(T v) {
        const float2 f0 = __half22float2(*reinterpret_cast<const __half2*>(&v.x));
        const float2 f1 = __half22float2(*reinterpret_cast<const __half2*>(&v.y));
        return P2{pack2(make_float2(f0.x, f1.x)), pack2(make_float2(f0.y, f1.y))};
    }
};
template <> struct Pair<2> {      // two 4+4-bit bytes (antenna 0 in the low byte), real part high
    using T = unsigned short;
    // as in the single-antenna decode: a two's-complement nibble n is (n ^ 8) - 8, and (n ^ 8) in
    // the mantissa of 2^23 minus 2^23 + 8 (one packed subtraction for both antennas) leaves n
    static __device__ __forceinline__ P2 dec(T v) {
        const unsigned w = (unsigned)v ^ 0x8888u;
        const float r0 = __uint_as_float(0x4B000000u | ((w >> 4) & 0xFu)), i0 = __uint_as_float(0x4B000000u | (w & 0xFu));
        const float r1 = __uint_as_float(0x4B000000u | (w >> 12)), i1 = __uint_as_float(0x4B000000u | ((w >> 8) & 0xFu));
        const unsigned long long off = f2dup(8388616.0f);
        return P2{f2sub(pack2(make_float2(r0, r1)), off), f2sub(pack2(make_float2(i0, i1)), off)};
    }
};

// Spectra of two adjacent antennas at one bin, stored with one 16- or 8-byte store.
template <int OUT> struct Out2;
template <> struct Out2<0> {      // complex64
    using T = float4;
    static __device__ __forceinline__ T enc(const P2& z) {
        const float2 re = unpack2(z.re), im = unpack2(z.im);
        return make_float4(re.x, im.x, re.y, im.y);
    }
};
template <> struct Out2<1> {      // FP16 pairs
    using T = uint2;
    static __device__ __forceinline__ T enc(const P2& z) {
        const float2 re = unpack2(z.re), im = unpack2(z.im);
        const __half2 h0 = __floats2half2_rn(re.x, im.x), h1 = __floats2half2_rn(re.y, im.y);
        return make_uint2(*reinterpret_cast<const unsigned*>(&h0), *reinterpret_cast<const unsigned*>(&h1));
    }
};

template <int C>
constexpr size_t smem_bytes2() { return (size_t)C * (2 * 2 * TA * sizeof(float) + sizeof(float4) + sizeof(float2)); }

// The same transform with 64-antenna tiles: thread (l, n1) takes antennas 2l, 2l + 1 of the
// tile.  Shared memory holds the real and imaginary parts in separate [C][64] planes, so that a
// pair is one 8-byte access and a warp's accesses are contiguous.  Needs an even antenna count
// (every pair starts at an even element of every row) and pair-aligned arrays.
template <int C, int VIN, int OUT>
__global__ void __launch_bounds__(32 * Split<C>::R2, 2) fengine2_kernel(const FengArgs a) {
    constexpr int R2 = Split<C>::R2, R1 = C / R2, NT = 32 * R2, TA2 = 2 * TA;
    static_assert(R1 >= R2 && R1 <= 64 && R1 % R2 == 0, "split");
    using VT = typename Pair<VIN>::T;
    using OT = typename Out2<OUT>::T;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float* XR = reinterpret_cast<float*>(smem_raw);              // [C][TA2] real parts
    float* XI = XR + C * TA2;                                     // [C][TA2] imaginary parts
    float4* TWP = reinterpret_cast<float4*>(XI + C * TA2);        // [C] (c, c, s, s) of exp(-2 pi i j / C)
    float2* TWN = reinterpret_cast<float2*>(TWP + C);             // [C] (-s, -s)
    const int tid = threadIdx.x, l = tid % 32, n1 = tid / 32;
    for (int j = tid; j < C; j += NT) {
        double s, c;
        sincospi(-2.0 * j / C, &s, &c);
        TWP[j] = make_float4(float(c), float(c), float(s), float(s));
        TWN[j] = make_float2(-float(s), -float(s));
    }
    const int A = a.n_ant, P = a.n_pol;
    const int n_tiles = (A + TA2 - 1) / TA2;
    const int n_units = a.n_time * P * n_tiles;   // < 2^31 (checked by the caller)
    const VT* raw = static_cast<const VT*>(a.raw);
    OT* out = static_cast<OT*>(a.volt);
    const long long row = (long long)P * A / 2;   // pairs from one sample (or bin) to the next
    // unit u = (t, p, tile), tile fastest, kept as coordinates: a step of gridDim.x units adds
    // the stride's own coordinates with carries (no divisions per unit)
    const int G = gridDim.x, g_tile = G % n_tiles, g_p = (G / n_tiles) % P, g_t = G / (n_tiles * P);
    auto step = [&](int& tile, int& p, int& t) {
        tile += g_tile;
        const int c1 = tile >= n_tiles;
        tile -= c1 ? n_tiles : 0;
        p += g_p + c1;
        const int c2 = p >= P;
        p -= c2 ? P : 0;
        t += g_t + c2;
    };
    VT nxt[R1];
    auto load_unit = [&](int tile, int p, int t) {
        const int ant = tile * TA2 + 2 * l;
        const VT* src = raw + ((long long)t * C + n1) * row + (p * A + ant) / 2;
#pragma unroll
        for (int q = 0; q < R1; ++q) nxt[q] = ant < A ? __ldg(src + q * R2 * row) : VT{};
    };
    const int u0 = blockIdx.x;
    int tile = u0 % n_tiles, p = (u0 / n_tiles) % P, t = u0 / (n_tiles * P);
    if (u0 < n_units) load_unit(tile, p, t);
    for (int u = u0; u < n_units; u += G) {
        int ntile = tile, np = p, nt = t;         // coordinates of unit u + G
        step(ntile, np, nt);
        const int ant = tile * TA2 + 2 * l;
        // stage 1: R1-point DFTs of samples n1 + R2 n2 (registers), twiddle exp(-2 pi i n1 k2 / C)
        {
            P2 x[R1];
#pragma unroll
            for (int q = 0; q < R1; ++q) x[q] = Pair<VIN>::dec(nxt[q]);
            dft2<R1, -1>(x);
            // the next unit's samples load under this unit's twiddle, exchange and stage 2 (not
            // under the DFT above, whose registers they would add to)
            if (u + G < n_units) load_unit(ntile, np, nt);
            __syncthreads();                              // previous unit's stage-2 reads are done
#pragma unroll
            for (int k2 = 0; k2 < R1; ++k2) {
                P2 y = x[k2];
                if (k2 > 0) {
                    const float4 w = TWP[n1 * k2];        // n1 k2 < C
                    const unsigned long long cc = pack2(make_float2(w.x, w.y)), ss = pack2(make_float2(w.z, w.w));
                    const unsigned long long nss = pack2(TWN[n1 * k2]);
                    y.re = f2fma(x[k2].re, cc, f2mul(x[k2].im, nss));
                    y.im = f2fma(x[k2].re, ss, f2mul(x[k2].im, cc));
                }
                const int o = (n1 + R2 * k2) * TA2 + 2 * l;
                *reinterpret_cast<unsigned long long*>(XR + o) = y.re;
                *reinterpret_cast<unsigned long long*>(XI + o) = y.im;
            }
        }
        __syncthreads();
        // stage 2: for k2 = n1, n1 + R2, ...: R2-point DFTs over n1' of rows n1' + R2 k2, bins
        // c = k2 + R1 k1
#pragma unroll
        for (int q = 0; q < R1 / R2; ++q) {
            const int k2 = n1 + R2 * q;
            P2 z[R2];
#pragma unroll
            for (int m = 0; m < R2; ++m) {
                const int o = (m + R2 * k2) * TA2 + 2 * l;
                z[m].re = *reinterpret_cast<const unsigned long long*>(XR + o);
                z[m].im = *reinterpret_cast<const unsigned long long*>(XI + o);
            }
            dft2<R2, -1>(z);
            if (ant < A) {
                OT* dst = out + ((long long)t * C + k2) * row + (p * A + ant) / 2;
#pragma unroll
                for (int k1 = 0; k1 < R2; ++k1) dst[k1 * R1 * row] = Out2<OUT>::enc(z[k1]);
            }
        }
        tile = ntile;
        p = np;
        t = nt;
    }
}

// the pair form: C <= 128 (complex64 input: C <= 64, where its registers suffice), an even
// antenna count and arrays aligned to two elements
template <int C, int VIN, int OUT>
bool use_pairs(const FengArgs& a) {
    if constexpr (C > 128 || (VIN == 0 && C > 64)) {
        return false;
    } else {
        return a.n_ant % 2 == 0 && reinterpret_cast<uintptr_t>(a.raw) % sizeof(typename Pair<VIN>::T) == 0 &&
               reinterpret_cast<uintptr_t>(a.volt) % sizeof(typename Out2<OUT>::T) == 0;
    }
}

template <int C, int VIN, int OUT>
cudaError_t launch_pairs(const FengArgs& a, int n_sm, cudaStream_t st) {
    constexpr int NT = 32 * Split<C>::R2;
    auto kern = fengine2_kernel<C, VIN, OUT>;
    const size_t smem = smem_bytes2<C>();
    cudaError_t e = ensure_smem<fengine2_kernel<C, VIN, OUT>>(smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, NT, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    const long long n_units = (long long)a.n_time * a.n_pol * ((a.n_ant + 2 * TA - 1) / (2 * TA));
    if (n_units > 2147483647LL) return cudaErrorInvalidValue;
    const long long grid = n_units < (long long)per_sm * n_sm ? n_units : (long long)per_sm * n_sm;
    if (grid == 0) return cudaSuccess;
    kern<<<(unsigned)grid, NT, smem, st>>>(a);
    return cudaGetLastError();
}

template <int C, int VIN, int OUT>
cudaError_t launch_t(const FengArgs& a, int n_sm, cudaStream_t st) {
    if constexpr (C <= 128 && !(VIN == 0 && C > 64)) {
        if (use_pairs<C, VIN, OUT>(a)) return launch_pairs<C, VIN, OUT>(a, n_sm, st);
    }
    constexpr int NT = TA * Split<C>::R2;
    const size_t smem = smem_bytes<C>();
    cudaError_t e = ensure_smem<fengine_kernel<C, VIN, OUT>>(smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fengine_kernel<C, VIN, OUT>, NT, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    const long long n_units = (long long)a.n_time * a.n_pol * ((a.n_ant + TA - 1) / TA);
    if (n_units > 2147483647LL) return cudaErrorInvalidValue;
    const long long grid = n_units < (long long)per_sm * n_sm ? n_units : (long long)per_sm * n_sm;
    if (grid == 0) return cudaSuccess;
    fengine_kernel<C, VIN, OUT><<<(unsigned)grid, NT, smem, st>>>(a);
    return cudaGetLastError();
}

template <int C>
cudaError_t launch_c(int vin, int vout, const FengArgs& a, int n_sm, cudaStream_t st) {
    switch (vin * 2 + vout) {
        case 0: return launch_t<C, 0, 0>(a, n_sm, st);
        case 1: return launch_t<C, 0, 1>(a, n_sm, st);
        case 2: return launch_t<C, 1, 0>(a, n_sm, st);
        case 3: return launch_t<C, 1, 1>(a, n_sm, st);
        case 4: return launch_t<C, 2, 0>(a, n_sm, st);
        case 5: return launch_t<C, 2, 1>(a, n_sm, st);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace fe

// vin: EPIC_VOLT_* of the raw samples; vout: 0 = complex64, 1 = FP16 pairs
cudaError_t launch_fengine(int n_chan, int vin, int vout, const FengArgs& a, int n_sm, cudaStream_t st) {
    switch (n_chan) {
        case 32: return fe::launch_c<32>(vin, vout, a, n_sm, st);
        case 64: return fe::launch_c<64>(vin, vout, a, n_sm, st);
        case 128: return fe::launch_c<128>(vin, vout, a, n_sm, st);
        case 256: return fe::launch_c<256>(vin, vout, a, n_sm, st);
        case 512: return fe::launch_c<512>(vin, vout, a, n_sm, st);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace epic
