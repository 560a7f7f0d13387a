// Once-per-integration epilogues of the MOFF imaging step, and host-visible geometry.
//
//   finalize_image   I = accum / T_total (Sec. 3 "Time-averaging").
//   weff, isotropic  the effective weighting of a heterogeneous array and the isotropic
//                    image estimate (Sec. 5).
//   autocorr         the antenna auto-correlation term of Sec. 4.2 in its per-antenna form
//                    (Sec. 4.3): A(k) = sum_a P_a |K_a(k)|^2 with K_a the spatial transform
//                    of antenna a's gridded footprint.  Since |K_a(k)|^2 is the transform of
//                    the footprint's auto-correlation R_a(d) = sum_g M[g,a] conj(M[g-d,a]),
//                    A(k) = sum_d U(d) exp(+2 pi i d.k / N_p) with U(d) = sum_a P_a R_a(d):
//                    a dense mat-vec over the small L x L lag window, then a separable sum
//                    onto the N_p x N_p pixels (U is Hermitian, so A is real).
#include "moff_common.cuh"
#include "moff_bwd.cuh"

namespace epic {

__global__ void finalize_image_kernel(const double* __restrict__ accum, float* __restrict__ image,
                                      long long n, double inv_t) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        image[i] = float(accum[i] * inv_t);
}

cudaError_t launch_finalize_image(const double* accum, float* image, long long n, double inv_t,
                                  cudaStream_t st) {
    if (n == 0) return cudaSuccess;
    long long blocks = (n + 255) / 256;
    if (blocks > 65536) blocks = 65536;
    finalize_image_kernel<<<(unsigned)blocks, 256, 0, st>>>(accum, image, n, inv_t);
    return cudaGetLastError();
}

// Cross-polarisation epilogue.  accum4 holds per channel the time sums S_v(k) of |F_v|^2 for
// the virtual pols v = X, Y, X + Y, X + iY; since |F_X + F_Y|^2 = |F_X|^2 + |F_Y|^2 +
// 2 Re(F_X conj F_Y) and |F_X + i F_Y|^2 = |F_X|^2 + |F_Y|^2 + 2 Im(F_X conj F_Y),
//   XX = S_0 / T, YY = S_1 / T, XY = ((S_2 - S_0 - S_1) + i (S_3 - S_0 - S_1)) / (2 T)
// in float64, then rounded.  image [C][2][npix] (may be null), cross [C][npix] complex.
__global__ void finalize_xpol_kernel(const double* __restrict__ accum4, float* __restrict__ image,
                                     float2* __restrict__ cross, int n_chan, long long npix, double inv_t) {
    const long long n = (long long)n_chan * npix;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const long long c = i / npix, k = i - c * npix;
        const double* s = accum4 + c * 4 * npix + k;
        const double s0 = s[0], s1 = s[npix], s2 = s[2 * npix], s3 = s[3 * npix];
        if (image) {
            image[(2 * c) * npix + k] = float(s0 * inv_t);
            image[(2 * c + 1) * npix + k] = float(s1 * inv_t);
        }
        if (cross) {
            const double h = 0.5 * inv_t;
            cross[c * npix + k] = make_float2(float((s2 - s0 - s1) * h), float((s3 - s0 - s1) * h));
        }
    }
}

cudaError_t launch_finalize_xpol(const double* accum4, float* image, float2* cross, int n_chan, long long npix,
                                 double inv_t, cudaStream_t st) {
    const long long n = (long long)n_chan * npix;
    if (n == 0 || (!image && !cross)) return cudaSuccess;
    long long blocks = (n + 255) / 256;
    if (blocks > 65536) blocks = 65536;
    finalize_xpol_kernel<<<(unsigned)blocks, 256, 0, st>>>(accum4, image, cross, n_chan, npix, inv_t);
    return cudaGetLastError();
}

constexpr int kAcThreads = 512;

// One block per (channel, pol).  Shared: U [L*L] float2, T1 [L][N_p] float2, twiddles
// [N_p] float2, P [A] float.  Three phases:
//   U(d)        = sum_a P_a R_a(d)                       (L^2 x A multiply-adds)
//   T1(dy, kx)  = sum_dx U(dy, dx) exp(+2 pi i dx kx / N_p) (L^2 x N_p)
//   A(ky, kx)   = Re sum_dy T1(dy, kx) exp(+2 pi i dy ky / N_p)  (N_p^2 x L)
// with k measured from the image centre (k = pixel - N_p/2; the exponent is periodic).
__global__ void __launch_bounds__(kAcThreads)
autocorr_kernel(const double* __restrict__ power, const float2* __restrict__ lag_tab,
                int n_ant, int L, int n_pad, double inv_t, float* __restrict__ out) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float2* U = reinterpret_cast<float2*>(smem_raw);
    float2* T1 = U + L * L;
    float2* TWs = T1 + L * n_pad;
    float* P = reinterpret_cast<float*>(TWs + n_pad);
    const int cp = blockIdx.x;
    const int LL = L * L, h = (L - 1) / 2, msk = n_pad - 1;
    for (int j = threadIdx.x; j < n_pad; j += blockDim.x) {
        double s, c;
        sincospi(2.0 * j / n_pad, &s, &c);
        TWs[j] = make_float2(float(c), float(s));
    }
    const double* pw = power + (size_t)cp * n_ant;
    for (int aa = threadIdx.x; aa < n_ant; aa += blockDim.x) P[aa] = float(pw[aa] * inv_t);
    __syncthreads();
    for (int j = threadIdx.x; j < LL; j += blockDim.x) {
        float2 u = make_float2(0.f, 0.f);
        for (int aa = 0; aa < n_ant; ++aa) {
            const float p = P[aa];
            const float2 rv = __ldg(lag_tab + (size_t)aa * LL + j);
            u.x = fmaf(p, rv.x, u.x);
            u.y = fmaf(p, rv.y, u.y);
        }
        U[j] = u;
    }
    __syncthreads();
    for (int j = threadIdx.x; j < L * n_pad; j += blockDim.x) {
        const int dy = j / n_pad, ix = j % n_pad, kx = ix - n_pad / 2;
        float2 acc = make_float2(0.f, 0.f);
        const float2* urow = U + dy * L;
        for (int dx = 0; dx < L; ++dx) {
            const float2 w = TWs[((dx - h) * kx) & msk];
            const float2 u = urow[dx];
            acc.x = fmaf(u.x, w.x, fmaf(-u.y, w.y, acc.x));
            acc.y = fmaf(u.x, w.y, fmaf(u.y, w.x, acc.y));
        }
        T1[j] = acc;
    }
    __syncthreads();
    const int npix = n_pad * n_pad;
    for (int pix = threadIdx.x; pix < npix; pix += blockDim.x) {
        const int iy = pix / n_pad, ix = pix % n_pad, ky = iy - n_pad / 2;
        float accr = 0.f;
        for (int dy = 0; dy < L; ++dy) {
            const float2 w = TWs[((dy - h) * ky) & msk];
            const float2 t = T1[dy * n_pad + ix];
            accr = fmaf(t.x, w.x, fmaf(-t.y, w.y, accr));
        }
        out[(size_t)cp * npix + pix] = accr;
    }
}

// Effective weighting of a heterogeneous array (Sec. 5, Eq. "effective-weighting-optimal"):
//   W_eff(k) = (1 / (A (A - 1))) sum_{a != b} |K_a(k)|^2 |K_b(k)|^2
//            = ((sum_a P_a)^2 - sum_a P_a^2) / (A (A - 1)),  P_a(k) = |K_a(k)|^2,
// with P_a the transform of the footprint auto-correlation R_a (the plan's lag tables),
// evaluated antenna by antenna (separably: rows of the lag window, then the pixels), image
// pixel order (k = 0 at the centre).  CTA b owns image rows kWeffRows b .. + kWeffRows - 1 and
// sums P_a and P_a^2 over the antennas in shared memory; every CTA redoes the row pass of each
// antenna (L x N_p values), which is small beside its share of the pixels.
constexpr int kWeffThreads = 512;
constexpr int kWeffRows = 16;

__global__ void __launch_bounds__(kWeffThreads)
weff_kernel(const float2* __restrict__ lag_tab, int n_ant, int L, int n_pad, float* __restrict__ out) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int rows = min(kWeffRows, n_pad), r0 = blockIdx.x * rows;
    const int npix = rows * n_pad, LL = L * L, h = (L - 1) / 2, msk = n_pad - 1;
    float* S2 = reinterpret_cast<float*>(smem_raw);        // [rows][n_pad]
    float* S4 = S2 + npix;
    float2* T1 = reinterpret_cast<float2*>(S4 + npix);     // [L][n_pad]
    float2* TWs = T1 + L * n_pad;
    for (int j = threadIdx.x; j < n_pad; j += blockDim.x) {
        double s, c;
        sincospi(2.0 * j / n_pad, &s, &c);
        TWs[j] = make_float2(float(c), float(s));
    }
    for (int pix = threadIdx.x; pix < npix; pix += blockDim.x) S2[pix] = S4[pix] = 0.f;
    __syncthreads();
    for (int a = 0; a < n_ant; ++a) {
        const float2* R = lag_tab + (size_t)a * LL;
        for (int j = threadIdx.x; j < L * n_pad; j += blockDim.x) {
            const int dy = j / n_pad, ix = j % n_pad, kx = ix - n_pad / 2;
            float2 acc = make_float2(0.f, 0.f);
            for (int dx = 0; dx < L; ++dx) {
                const float2 w = TWs[((dx - h) * kx) & msk];
                const float2 r = __ldg(R + dy * L + dx);
                acc.x = fmaf(r.x, w.x, fmaf(-r.y, w.y, acc.x));
                acc.y = fmaf(r.x, w.y, fmaf(r.y, w.x, acc.y));
            }
            T1[j] = acc;
        }
        __syncthreads();
        for (int pix = threadIdx.x; pix < npix; pix += blockDim.x) {
            const int iy = r0 + pix / n_pad, ix = pix % n_pad, ky = iy - n_pad / 2;
            float p = 0.f;
            for (int dy = 0; dy < L; ++dy) {
                const float2 w = TWs[((dy - h) * ky) & msk];
                const float2 t = T1[dy * n_pad + ix];
                p = fmaf(t.x, w.x, fmaf(-t.y, w.y, p));
            }
            S2[pix] += p;
            S4[pix] = fmaf(p, p, S4[pix]);
        }
        __syncthreads();
    }
    const float norm = 1.f / (float(n_ant) * float(n_ant - 1));
    for (int pix = threadIdx.x; pix < npix; pix += blockDim.x)
        out[(size_t)r0 * n_pad + pix] = fmaf(S2[pix], S2[pix], -S4[pix]) * norm;
}

size_t weff_smem_bytes(int lag_side, int n_pad) {
    const int rows = n_pad < kWeffRows ? n_pad : kWeffRows;
    return sizeof(float) * 2 * (size_t)rows * n_pad + sizeof(float2) * ((size_t)lag_side * n_pad + n_pad);
}

cudaError_t launch_weff(const float2* lag_tab, int n_ant, int lag_side, int n_pad, float* out, cudaStream_t st) {
    const size_t smem = weff_smem_bytes(lag_side, n_pad);
    cudaError_t e = ensure_smem<weff_kernel>(smem);
    if (e != cudaSuccess) return e;
    const int rows = n_pad < kWeffRows ? n_pad : kWeffRows;
    weff_kernel<<<n_pad / rows, kWeffThreads, smem, st>>>(lag_tab, n_ant, lag_side, n_pad, out);
    return cudaGetLastError();
}

// Isotropic image estimate (Sec. 5, Eq. "effective-weighting"): I_D^iso = I' / W_eff with
// I' = (image - autocorr) / (A (A - 1)) the mean weighted fringe over pairs a != b.  Pixels
// where W_eff is below rel_floor times its largest value are set to NaN (outside the beam).
__global__ void isotropic_kernel(const float* __restrict__ image, const float* __restrict__ autocorr,
                                 const float* __restrict__ weff, float rel_floor, float pair_norm,
                                 long long n, int npix, float* __restrict__ iso) {
    __shared__ float red[32];
    float m = 0.f;
    for (int i = threadIdx.x; i < npix; i += blockDim.x) m = fmaxf(m, weff[i]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x < 32) {
        m = threadIdx.x < (blockDim.x + 31) / 32 ? red[threadIdx.x] : 0.f;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
        if (threadIdx.x == 0) red[0] = m;
    }
    __syncthreads();
    const float floor_abs = rel_floor * red[0];
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const float w = weff[i % npix];
        iso[i] = (w >= floor_abs && w > 0.f) ? (image[i] - autocorr[i]) * pair_norm / w : __int_as_float(0x7fc00000);
    }
}

cudaError_t launch_isotropic(const float* image, const float* autocorr, const float* weff, float rel_floor,
                             int n_ant, long long n, int npix, float* iso, cudaStream_t st) {
    if (n == 0) return cudaSuccess;
    long long blocks = (n + 255) / 256;
    if (blocks > 4096) blocks = 4096;
    const float pair_norm = 1.f / (float(n_ant) * float(n_ant - 1));
    isotropic_kernel<<<(unsigned)blocks, 256, 0, st>>>(image, autocorr, weff, rel_floor, pair_norm, n, npix, iso);
    return cudaGetLastError();
}

size_t autocorr_smem_bytes(int lag_side, int n_pad, int n_ant) {
    return sizeof(float2) * ((size_t)lag_side * lag_side + (size_t)lag_side * n_pad + n_pad)
         + sizeof(float) * (size_t)n_ant;
}

cudaError_t launch_autocorr(const double* power, const float2* lag_tab, int n_cp, int n_ant,
                            int lag_side, int n_pad, double inv_t, float* out, cudaStream_t st) {
    const size_t smem = autocorr_smem_bytes(lag_side, n_pad, n_ant);
    cudaError_t e = ensure_smem<autocorr_kernel>(smem);
    if (e != cudaSuccess) return e;
    autocorr_kernel<<<n_cp, kAcThreads, smem, st>>>(power, lag_tab, n_ant, lag_side, n_pad, inv_t, out);
    return cudaGetLastError();
}

int resident_fwd_workers_32(int vdt, int max_ant, int n_sm);
int resident_fwd_workers_64(int vdt, int max_ant, int n_sm);
int resident_fwd_workers_128(int vdt, int max_ant, int n_sm);
int resident_fwd_workers_256(int vdt, int max_ant, int n_sm);
int resident_fwd_workers_512(int vdt, int max_ant, int n_sm);

int resident_fwd_workers(int n_pad, int vdt, int max_ant, int n_sm) {
    switch (n_pad) {
        case 32: return resident_fwd_workers_32(vdt, max_ant, n_sm);
        case 64: return resident_fwd_workers_64(vdt, max_ant, n_sm);
        case 128: return resident_fwd_workers_128(vdt, max_ant, n_sm);
        case 256: return resident_fwd_workers_256(vdt, max_ant, n_sm);
        case 512: return resident_fwd_workers_512(vdt, max_ant, n_sm);
        default: return 0;
    }
}

size_t fwd_smem_bytes(int n_pad, int n_ant) {
    switch (n_pad) {
        case 32: return Geo<32>::smem_bytes(n_ant);
        case 64: return Geo<64>::smem_bytes(n_ant);
        case 128: return Geo<128>::smem_bytes(n_ant);
        case 256: return Geo<256>::smem_bytes(n_ant);
        case 512: return Geo<512>::smem_bytes(n_ant);
        default: return 0;
    }
}

size_t fwd_xpol_smem_bytes(int n_pad, int n_ant) {
    switch (n_pad) {
        case 32: return Geo<32>::smem_bytes_xpol(n_ant);
        case 64: return Geo<64>::smem_bytes_xpol(n_ant);
        case 128: return Geo<128>::smem_bytes_xpol(n_ant);
        case 256: return Geo<256>::smem_bytes_xpol(n_ant);
        case 512: return Geo<512>::smem_bytes_xpol(n_ant);
        default: return 0;
    }
}

size_t bwd_smem_bytes(int n_pad, int n_ant) {
    switch (n_pad) {
        case 32: return BwdLayout<32>::smem_bytes(n_ant);
        case 64: return BwdLayout<64>::smem_bytes(n_ant);
        case 128: return BwdLayout<128>::smem_bytes(n_ant);
        case 256: return BwdLayout<256>::smem_bytes(n_ant);
        case 512: return BwdLayout<512>::smem_bytes(n_ant);
        default: return 0;
    }
}

int grid_rows_per_block(int n_pad) {
    switch (n_pad) {
        case 32: return Geo<32>::ROWS;
        case 64: return Geo<64>::ROWS;
        case 128: return Geo<128>::ROWS;
        case 256: return Geo<256>::ROWS;
        case 512: return Geo<512>::ROWS;
        default: return 0;
    }
}

int fwd_interleave_lanes(int n_pad) {
    switch (n_pad) {
        case 32: return Cfg<32>::RR ? 0 : Geo<32>::S;
        case 64: return Cfg<64>::RR ? 0 : Geo<64>::S;
        case 128: return Cfg<128>::RR ? 0 : Geo<128>::S;
        default: return 0;
    }
}

int exchange_row_stride(int n_pad) {
    switch (n_pad) {
        case 32: return Geo<32>::RXS;
        case 64: return Geo<64>::RXS;
        case 128: return Geo<128>::RXS;
        case 256: return Geo<256>::RXS;
        case 512: return Geo<512>::RXS;
        default: return 0;
    }
}

}  // namespace epic
