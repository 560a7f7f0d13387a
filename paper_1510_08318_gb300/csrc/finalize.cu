// Once-per-integration epilogues of the MOFF imaging step, and host-visible geometry.
//
//   finalize_image   I = accum / T_total (Sec. 3 "Time-averaging").
//   autocorr         the antenna auto-correlation term of Sec. 4.2 in its per-antenna form
//                    (Sec. 4.3): A(k) = sum_a P_a |K_a(k)|^2 with K_a the spatial transform
//                    of antenna a's gridded footprint.  Since |K_a(k)|^2 is the transform of
//                    the footprint's auto-correlation R_a(d) = sum_g M[g,a] conj(M[g-d,a]),
//                    A(k) = sum_d U(d) exp(+2 pi i d.k / N_p) with U(d) = sum_a P_a R_a(d):
//                    a dense mat-vec over the small L x L lag window, then a direct 2-D sum
//                    per output pixel (U is Hermitian, so A is real).
#include "moff_common.cuh"

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

constexpr int kAcThreads = 256;

// grid: (pixel blocks, CP).  Shared: U [L*L] float2, twiddles [N_p] float2.
__global__ void autocorr_kernel(const double* __restrict__ power, const float2* __restrict__ lag_tab,
                                int n_ant, int L, int n_pad, double inv_t, float* __restrict__ out) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float2* U = reinterpret_cast<float2*>(smem_raw);
    float2* TWs = U + L * L;
    const int cp = blockIdx.y;
    const int LL = L * L;
    for (int j = threadIdx.x; j < n_pad; j += blockDim.x) {
        double s, c;
        sincospi(2.0 * j / n_pad, &s, &c);
        TWs[j] = make_float2(float(c), float(s));
    }
    const double* pw = power + (size_t)cp * n_ant;
    for (int j = threadIdx.x; j < LL; j += blockDim.x) {
        float2 u = make_float2(0.f, 0.f);
        for (int aa = 0; aa < n_ant; ++aa) {
            const float p = float(pw[aa] * inv_t);
            const float2 rv = __ldg(lag_tab + (size_t)aa * LL + j);
            u.x = fmaf(p, rv.x, u.x);
            u.y = fmaf(p, rv.y, u.y);
        }
        U[j] = u;
    }
    __syncthreads();
    const int h = (L - 1) / 2;
    const int npix = n_pad * n_pad;
    const int pix = blockIdx.x * blockDim.x + threadIdx.x;
    if (pix >= npix) return;
    const int iy = pix / n_pad, ix = pix % n_pad;
    const int ky = iy - n_pad / 2, kx = ix - n_pad / 2;
    float accr = 0.f;
    for (int dy = -h; dy <= h; ++dy) {
        float2 inner = make_float2(0.f, 0.f);
        const float2* urow = U + (dy + h) * L;
        for (int dx = -h; dx <= h; ++dx) {
            const float2 w = TWs[((dx * kx) % n_pad + n_pad) % n_pad];
            const float2 u = urow[dx + h];
            inner.x = fmaf(u.x, w.x, fmaf(-u.y, w.y, inner.x));
            inner.y = fmaf(u.x, w.y, fmaf(u.y, w.x, inner.y));
        }
        const float2 w = TWs[((dy * ky) % n_pad + n_pad) % n_pad];
        accr = fmaf(inner.x, w.x, fmaf(-inner.y, w.y, accr));
    }
    out[(size_t)cp * npix + pix] = accr;
}

cudaError_t launch_autocorr(const double* power, const float2* lag_tab, int n_cp, int n_ant,
                            int lag_side, int n_pad, double inv_t, float* out, cudaStream_t st) {
    const int npix = n_pad * n_pad;
    dim3 grid((npix + kAcThreads - 1) / kAcThreads, n_cp);
    const size_t smem = sizeof(float2) * ((size_t)lag_side * lag_side + n_pad);
    autocorr_kernel<<<grid, kAcThreads, smem, st>>>(power, lag_tab, n_ant, lag_side, n_pad, inv_t, out);
    return cudaGetLastError();
}

size_t fwd_smem_bytes(int n_pad, int n_ant) {
    switch (n_pad) {
        case 32: return Geo<32>::smem_bytes(n_ant);
        case 64: return Geo<64>::smem_bytes(n_ant);
        case 128: return Geo<128>::smem_bytes(n_ant);
        case 256: return Geo<256>::smem_bytes(n_ant);
        default: return 0;
    }
}

size_t bwd_smem_bytes(int n_pad, int n_ant) {
    const size_t fixed_f = fwd_smem_bytes(n_pad, 0);
    return fixed_f == 0 ? 0 : fixed_f + size_t(n_ant) * 4 * sizeof(float2);
}

int grid_rows_per_block(int n_pad) {
    switch (n_pad) {
        case 32: return Geo<32>::ROWS;
        case 64: return Geo<64>::ROWS;
        case 128: return Geo<128>::ROWS;
        case 256: return Geo<256>::ROWS;
        default: return 0;
    }
}

int exchange_row_stride(int n_pad) {
    switch (n_pad) {
        case 32: return Geo<32>::RXS;
        case 64: return Geo<64>::RXS;
        case 128: return Geo<128>::RXS;
        case 256: return Geo<256>::RXS;
        default: return 0;
    }
}

}  // namespace epic
