// Register-resident small DFTs used by the MOFF spatial transform.
//
// The 2-D transform of the zero-padded grid (Sec. 3 "Spatial Fourier Transform",
// Eq. "dirty-image-MOFF") is split into 1-D transforms of length N_p whose upper half
// of inputs is zero; each of those is factored N_p = S * R1 (Cooley-Tukey) into
// R1-point sub-transforms with half-zero input, a twiddle by exp(+-2 pi i n1 k2 / N_p)
// and S-point sub-transforms.  The sub-transforms (lengths 2..32) are done here, fully
// unrolled in registers, with compile-time twiddle constants.
#pragma once
#include <cuda_runtime.h>

namespace epic {

// ---- compile-time cos / sin of 2 pi m / 64 (Taylor series, float64, reduced to [-pi, pi]) ----
constexpr double kPi = 3.14159265358979323846264338327950288;

constexpr double taylor_sin(double x) {
    double term = x, sum = x;
    for (int n = 1; n < 24; ++n) {
        term *= -x * x / double((2 * n) * (2 * n + 1));
        sum += term;
    }
    return sum;
}
constexpr double taylor_cos(double x) {
    double term = 1.0, sum = 1.0;
    for (int n = 1; n < 24; ++n) {
        term *= -x * x / double((2 * n - 1) * (2 * n));
        sum += term;
    }
    return sum;
}
// angle 2 pi m / M with m reduced into (-M/2, M/2]
constexpr double turn_angle(int m, int M) {
    int r = ((m % M) + M) % M;
    if (2 * r > M) r -= M;
    return 2.0 * kPi * double(r) / double(M);
}
// Table of exp(2 pi i m / 64), m in [0, 64), built by the compiler (constant-evaluated), so
// that every rotation below with a compile-time (m, M) folds into immediate operands.
struct TwTable64 { float c[64]; float s[64]; };
constexpr TwTable64 make_tw64() {
    TwTable64 t{};
    for (int m = 0; m < 64; ++m) {
        t.c[m] = float(taylor_cos(turn_angle(m, 64)));
        t.s[m] = float(taylor_sin(turn_angle(m, 64)));
    }
    return t;
}
__device__ constexpr TwTable64 kTw64 = make_tw64();

// Complex add and subtract as one packed FP32 instruction (add.rn.f32x2 / sub.rn.f32x2: both
// lanes rounded to nearest like two scalar adds, so the results are the scalar ones bit for bit).
__device__ __forceinline__ unsigned long long pack2(float2 a) {
    unsigned long long r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a.x), "f"(a.y));
    return r;
}
__device__ __forceinline__ float2 unpack2(unsigned long long r) {
    float2 a;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(a.x), "=f"(a.y) : "l"(r));
    return a;
}
__device__ __forceinline__ float2 cadd(float2 a, float2 b) {
    unsigned long long r;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(pack2(a)), "l"(pack2(b)));
    return unpack2(r);
}
__device__ __forceinline__ float2 csub(float2 a, float2 b) {
    unsigned long long r;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(pack2(a)), "l"(pack2(b)));
    return unpack2(r);
}
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
// a * conj(b)
__device__ __forceinline__ float2 cmulc(float2 a, float2 b) {
    return make_float2(fmaf(a.x, b.x, a.y * b.y), fmaf(a.y, b.x, -a.x * b.y));
}
__device__ __forceinline__ float cnorm(float2 a) { return fmaf(a.x, a.x, a.y * a.y); }

// a * exp(SIGN * 2 pi i m / M) with m, M compile-time after unrolling; the trivial
// rotations (1, +-i, -1) cost no multiplies.
template <int SIGN>
__device__ __forceinline__ float2 rot(float2 a, int m, int M) {
    int r = ((m % M) + M) % M;
    if (r == 0) return a;
    if (4 * r == M) return SIGN > 0 ? make_float2(-a.y, a.x) : make_float2(a.y, -a.x);
    if (2 * r == M) return make_float2(-a.x, -a.y);
    if (4 * r == 3 * M) return SIGN > 0 ? make_float2(a.y, -a.x) : make_float2(-a.y, a.x);
    const int idx = r * (64 / M);
    const float c = kTw64.c[idx];
    const float s = SIGN > 0 ? kTw64.s[idx] : -kTw64.s[idx];
    return make_float2(fmaf(a.x, c, -a.y * s), fmaf(a.x, s, a.y * c));
}

template <int N>
__host__ __device__ constexpr int bitrev(int k) {
    int r = 0;
    for (int b = 1; b < N; b <<= 1) { r = (r << 1) | (k & 1); k >>= 1; }
    return r;
}

// In-place x[k] <- sum_n x[n] exp(SIGN 2 pi i n k / N), N a power of two <= 64.
// Radix-2 decimation in frequency (natural input, bit-reversed output), then a
// compile-time permutation (register renaming).
template <int N, int SIGN>
__device__ __forceinline__ void dft(float2 (&x)[N]) {
    if constexpr (N > 1) {
#pragma unroll
        for (int half = N / 2; half >= 1; half >>= 1) {
#pragma unroll
            for (int blk = 0; blk < N; blk += 2 * half) {
#pragma unroll
                for (int j = 0; j < half; ++j) {
                    const float2 a = x[blk + j], b = x[blk + j + half];
                    x[blk + j] = cadd(a, b);
                    x[blk + j + half] = rot<SIGN>(csub(a, b), j, 2 * half);
                }
            }
        }
        float2 y[N];
#pragma unroll
        for (int k = 0; k < N; ++k) y[k] = x[bitrev<N>(k)];
#pragma unroll
        for (int k = 0; k < N; ++k) x[k] = y[k];
    }
}

// Y[k] = sum_{n < N/2} x[n] exp(SIGN 2 pi i n k / N) for k < N: an N-point DFT whose upper
// half of inputs is zero.  Even outputs are the N/2-point DFT of x, odd outputs the
// N/2-point DFT of x[n] exp(SIGN 2 pi i n / N).
template <int N, int SIGN>
__device__ __forceinline__ void dft_halfzero_in(const float2 (&x)[N / 2], float2 (&Y)[N]) {
    float2 e[N / 2], o[N / 2];
#pragma unroll
    for (int n = 0; n < N / 2; ++n) { e[n] = x[n]; o[n] = rot<SIGN>(x[n], n, N); }
    dft<N / 2, SIGN>(e);
    dft<N / 2, SIGN>(o);
#pragma unroll
    for (int m = 0; m < N / 2; ++m) { Y[2 * m] = e[m]; Y[2 * m + 1] = o[m]; }
}

// Adjoint of dft_halfzero_in with the opposite sign: x[n] = sum_{k < N} Y[k] exp(SIGN 2 pi i n k / N)
// for n < N/2 only.
template <int N, int SIGN>
__device__ __forceinline__ void dft_halfzero_out(const float2 (&Y)[N], float2 (&x)[N / 2]) {
    float2 e[N / 2], o[N / 2];
#pragma unroll
    for (int m = 0; m < N / 2; ++m) { e[m] = Y[2 * m]; o[m] = Y[2 * m + 1]; }
    dft<N / 2, SIGN>(e);
    dft<N / 2, SIGN>(o);
#pragma unroll
    for (int n = 0; n < N / 2; ++n) x[n] = cadd(e[n], rot<SIGN>(o[n], n, N));
}

}  // namespace epic
