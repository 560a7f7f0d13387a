"""FP64 CPU oracle for the MOFF imaging step -- TEST INFRASTRUCTURE ONLY.

Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline leg may import this
module.  It shares no code with the CUDA library and imports nothing from it.

Everything here is the plain definition from Thyagarajan et al. (2015), written out
in numpy/scipy float64, with no blocking, fusion or reordering:

  map_antennas   Sec. 3 "Antenna-to-Grid Mapping": nearest-grid-point mapping of every
                 footprint sample of every antenna; M(r, a) is the sparse N_g^2 x N_A
                 matrix of summed sample weights (stored CSR, as the paper does).
  grid_efields   Sec. 3 "Gridding Convolution": E(r) = M(r, a) E(a), with the complex
                 gains applied to E(a) first (Sec. 3 "Calibration").
  moff_image     Eq. "dirty-image-MOFF": zero-pad (Sec. 3 "Spatial Fourier Transform"),
                 2-D spatial DFT with the imaging sign exp(+2 pi i r.s / lambda)
                 (App. B, Eq. of the weighted fringe), squared per sample and
                 time-averaged (Sec. 3 "Time-averaging").
  autocorr_term  Sec. 4.2: the zero-spacing contribution of antenna auto-correlations,
                 A(k) = sum_a P_a |K_a(k)|^2 with P_a the mean antenna power and K_a
                 the spatial transform of antenna a's sampled footprint (the
                 per-antenna form Sec. 4.3 proposes).
  remove_autocorr_peak_scaled  Sec. 4.2 as the paper does it: the image taken back to the
                 uv plane, an estimated auto-correlation kernel scaled to the zero-spacing
                 value subtracted, and the result transformed back (uv_from_image and
                 image_from_uv_plane are the two transforms).
  fengine        Sec. 3 "Temporal Fourier transform": per-antenna spectra of blocks of
                 time samples (numpy's FFT as the library step).
  weff_opt, isotropic_image  Sec. 5: the effective weighting of the image of a
                 heterogeneous array and the isotropic dirty-image estimate I' / W_eff.
  moff_cross_image  the four cross-polarisation products mean_t F_p conj(F_q) of
                 dual-polarisation data (Sec. 3; App. A image module).
  grad_gains     derivative of a real loss L(I) with respect to the complex gains,
                 by the chain rule through Eq. "dirty-image-MOFF".

Conventions (readings of points the paper leaves open):
  * cell index per axis = floor((x - x0) / dx + 0.5) in float64, x = r_a + delta_k;
  * grid cell g = (gy, gx), flattened gy * N_g + gx; the N_g x N_g grid sits in the
    corner [0, N_g)^2 of the N_p x N_p zero-padded grid;
  * F(k) = sum_g E(g) exp(+2 pi i (g . k) / N_p), no normalisation;
  * the image is fftshifted: pixel (iy, ix) holds k = ((iy + N_p/2) mod N_p, ...),
    i.e. direction (l, m) = ((ix - N_p/2), (iy - N_p/2)) * lambda / (N_p dx);
  * time average = sum over samples / number of samples.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp


# ----------------------------------------------------------------------------------
# antenna-to-grid mapping (Sec. 3)
# ----------------------------------------------------------------------------------
def map_antennas(pos, kern_ptr, kern_dxdy, kern_w, dx, origin, n_grid):
    """Sparse M (N_g^2 x A, complex128, CSR).  Raises ValueError if a footprint sample
    falls outside the grid."""
    n_ant = pos.shape[0]
    rows, cols, vals = [], [], []
    for a in range(n_ant):
        for k in range(kern_ptr[a], kern_ptr[a + 1]):
            x = pos[a, 0] + kern_dxdy[k, 0]
            y = pos[a, 1] + kern_dxdy[k, 1]
            gx = int(np.floor((x - origin[0]) / dx + 0.5))
            gy = int(np.floor((y - origin[1]) / dx + 0.5))
            if not (0 <= gx < n_grid and 0 <= gy < n_grid):
                raise ValueError("footprint sample of antenna %d outside the grid" % a)
            rows.append(gy * n_grid + gx)
            cols.append(a)
            vals.append(complex(kern_w[k]))
    # duplicate (cell, antenna) entries are summed by the constructor
    M = sp.coo_matrix((np.array(vals, dtype=np.complex128), (rows, cols)),
                      shape=(n_grid * n_grid, n_ant)).tocsr()
    M.sum_duplicates()
    return M


def aperture_weights(M):
    """Eq. "gridding-convolution": W(r) = M(r, a) 1(a)."""
    return np.asarray(M @ np.ones(M.shape[1], dtype=np.complex128)).ravel()


# ----------------------------------------------------------------------------------
# the direct MOFF route
# ----------------------------------------------------------------------------------
def dft_matrix(n_pad, n_in):
    """D[k, g] = exp(+2 pi i g k / n_pad), k in [0, n_pad), g in [0, n_in)."""
    k = np.arange(n_pad)[:, None]
    g = np.arange(n_in)[None, :]
    return np.exp(2j * np.pi * ((k * g) % n_pad) / n_pad)


def grid_efields(M, volt_t, gain, n_grid):
    """E_t(g) for every sample: volt_t [T, A] complex, gain [A] complex.  -> [T, N_g, N_g]."""
    vp = volt_t * gain[None, :]
    E = (M @ vp.T).T
    return np.asarray(E).reshape(volt_t.shape[0], n_grid, n_grid)


def spatial_transform(E, n_pad):
    """Zero-padded 2-D DFT of each gridded field: [T, N_g, N_g] -> [T, N_p, N_p] (k order)."""
    n_grid = E.shape[-1]
    D = dft_matrix(n_pad, n_grid)
    return np.einsum("ky,tyx,jx->tkj", D, E, D, optimize=True)


def fftshift2(x):
    n = x.shape[-1]
    return np.roll(np.roll(x, n // 2, axis=-1), n // 2, axis=-2)


def moff_image_cp(M, volt_t, gain, n_grid, n_pad):
    """One (channel, pol): volt_t [T, A] -> (image [N_p, N_p] shifted, sum |F|^2 shifted)."""
    E = grid_efields(M, volt_t, gain, n_grid)
    F = spatial_transform(E, n_pad)
    s = (np.abs(F) ** 2).sum(0)
    s = fftshift2(s)
    return s / volt_t.shape[0], s


def moff_image(M, volt, gains, n_grid, n_pad):
    """Eq. "dirty-image-MOFF" for a cube: volt [T, C, P, A], gains [C, P, A] or None
    -> integrated image [C, P, N_p, N_p] float64."""
    T, C, P, A = volt.shape
    out = np.empty((C, P, n_pad, n_pad))
    for c in range(C):
        for p in range(P):
            g = np.ones(A, dtype=np.complex128) if gains is None else gains[c, p].astype(np.complex128)
            out[c, p] = moff_image_cp(M, volt[:, c, p, :], g, n_grid, n_pad)[0]
    return out


def moff_cross_image(M, volt, gains, n_grid, n_pad):
    """The four instrumental cross-polarisation images of a dual-polarisation cube (Sec. 3
    and the image module of App. A; Eq. "dirty-image-MOFF" with F_p conj(F_q) in place of
    |F_p|^2): volt [T, C, 2, A], gains [C, 2, A] or None ->
    I [C, 2, 2, N_p, N_p] complex128, I[c, p, q] = mean_t F_p(k) conj(F_q(k)), shifted.
    I[c, p, p] is moff_image's image; I[c, 1, 0] = conj(I[c, 0, 1])."""
    T, C, P, A = volt.shape
    if P != 2:
        raise ValueError("cross-polarisation images need two polarisations")
    out = np.empty((C, 2, 2, n_pad, n_pad), dtype=np.complex128)
    for c in range(C):
        F = []
        for p in range(2):
            g = np.ones(A, dtype=np.complex128) if gains is None else gains[c, p].astype(np.complex128)
            F.append(spatial_transform(grid_efields(M, volt[:, c, p, :], g, n_grid), n_pad))
        for p in range(2):
            for q in range(2):
                out[c, p, q] = fftshift2((F[p] * np.conj(F[q])).mean(0))
    return out


# ----------------------------------------------------------------------------------
# the antenna auto-correlation term (Sec. 4.2, per-antenna form of Sec. 4.3)
# ----------------------------------------------------------------------------------
def footprint_transforms(M, n_grid, n_pad):
    """K_a(k) = sum_g M[g, a] exp(+2 pi i g.k / N_p), shifted: [A, N_p, N_p] complex."""
    A = M.shape[1]
    Md = M.toarray().T.reshape(A, n_grid, n_grid)
    D = dft_matrix(n_pad, n_grid)
    K = np.einsum("ky,ayx,jx->akj", D, Md, D, optimize=True)
    return fftshift2(K)


def antenna_power(volt_t, gain):
    """P_a = mean_t |g_a V_a(t)|^2."""
    return (np.abs(volt_t * gain[None, :]) ** 2).mean(0)


def autocorr_term(M, volt, gains, n_grid, n_pad):
    """A[c, p, k] = sum_a P_a |K_a(k)|^2 (shifted), [C, P, N_p, N_p]."""
    T, C, P, A = volt.shape
    K2 = np.abs(footprint_transforms(M, n_grid, n_pad)) ** 2
    out = np.empty((C, P, n_pad, n_pad))
    for c in range(C):
        for p in range(P):
            g = np.ones(A, dtype=np.complex128) if gains is None else gains[c, p].astype(np.complex128)
            Pa = antenna_power(volt[:, c, p, :], g)
            out[c, p] = np.tensordot(Pa, K2, axes=(0, 0))
    return out


def uv_from_image(image, n_grid):
    """The uv plane of an image of the +i transform (Sec. 4.2: the squared image transformed
    back to the uv plane): image [N_p, N_p] shifted -> U(d) for lags d in (-N_g, N_g)^2,
    [2 N_g - 1, 2 N_g - 1] with lag (dy, dx) at (dy + N_g - 1, dx + N_g - 1).  Exact for
    N_p >= 2 N_g - 1 (no lag aliases); numpy's FFT is the library step."""
    n_pad = image.shape[-1]
    P = np.fft.fft2(np.fft.ifftshift(image)) / (n_pad * n_pad)
    lag = np.arange(-(n_grid - 1), n_grid) % n_pad
    return P[np.ix_(lag, lag)]


def image_from_uv_plane(U, n_grid, n_pad):
    """Inverse of uv_from_image: I(k) = sum_d U(d) exp(+2 pi i d.k / N_p), shifted."""
    P = np.zeros((n_pad, n_pad), dtype=np.complex128)
    lag = np.arange(-(n_grid - 1), n_grid) % n_pad
    P[np.ix_(lag, lag)] = U
    return np.fft.fftshift(np.fft.ifft2(P) * (n_pad * n_pad))


def remove_autocorr_peak_scaled(image, kernel_uv, n_grid):
    """The paper's removal of the antenna auto-correlations from a MOFF image (Sec. 4.2), in its
    order: transform the squared image back to the uv plane, subtract the estimated
    auto-correlation kernel (kernel_uv, on the lag plane of uv_from_image, peak at zero spacing)
    scaled so that its peak equals the uv plane's value at the zero-spacing pixel, and transform
    back.  Returns (image with the auto-correlations removed, its uv plane)."""
    U = uv_from_image(image, n_grid)
    z = n_grid - 1
    U = U - (U[z, z] / kernel_uv[z, z]) * kernel_uv
    return image_from_uv_plane(U, n_grid, image.shape[-1]).real, U


# ----------------------------------------------------------------------------------
# the F-engine (Sec. 3 "Temporal Fourier transform")
# ----------------------------------------------------------------------------------
def fengine(raw, n_chan):
    """Spectra of blocks of n_chan consecutive time samples of every antenna:
    raw [T n_chan, P, A] complex -> V [T, n_chan, P, A] with
    V[t, c] = sum_j raw[t n_chan + j] exp(-2 pi i j c / n_chan) (numpy's forward FFT)."""
    n_samp, P, A = raw.shape
    blocks = np.asarray(raw, dtype=np.complex128).reshape(n_samp // n_chan, n_chan, P, A)
    return np.fft.fft(blocks, axis=1)


# ----------------------------------------------------------------------------------
# heterogeneous arrays: effective weighting and the isotropic image estimate (Sec. 5)
# ----------------------------------------------------------------------------------
def weff_opt(M, n_grid, n_pad):
    """Eq. "effective-weighting-optimal" on the image pixels: the mean over ordered antenna
    pairs a != b of |K_a(k)|^2 |K_b(k)|^2, K_a the transform of antenna a's gridded footprint
    (the gridding weights equal to the instrument's, W^G = W^I), shifted: [N_p, N_p]."""
    K = footprint_transforms(M, n_grid, n_pad)
    P = np.abs(K) ** 2
    A = P.shape[0]
    total = np.zeros((n_pad, n_pad))
    for a in range(A):
        for b in range(A):
            if a != b:
                total += P[a] * P[b]
    return total / (A * (A - 1))


def isotropic_image(image, autocorr, weff, n_ant):
    """Eq. "effective-weighting": the estimate of the isotropically weighted dirty image,
    I_D^iso = I' / W_eff, with I' = (image - autocorr) / (N (N - 1)) the mean of the weighted
    fringes over antenna pairs a != b (Eq. "wt-dirty-image-EPIC")."""
    return (image - autocorr) / (n_ant * (n_ant - 1)) / weff


# ----------------------------------------------------------------------------------
# gradient of a real image-domain loss with respect to the complex gains
# ----------------------------------------------------------------------------------
def grad_gains(M, volt, gains, n_grid, n_pad, grad_image):
    """grad[c, p, a] = dL/dRe g + i dL/dIm g for a real loss L whose derivative with
    respect to the integrated image I[c, p] (shifted pixel order) is grad_image.

    With F_t(k) = sum_a g_a V_a(t) K_a(k) and I(k) = mean_t |F_t(k)|^2:
        dI(k)/d conj(g_a) = mean_t F_t(k) conj(V_a(t) K_a(k)),
        grad_a = 2 dL/d conj(g_a) = 2 sum_k G(k) mean_t F_t(k) conj(V_a(t) K_a(k)).
    """
    T, C, P, A = volt.shape
    K = footprint_transforms(M, n_grid, n_pad).reshape(A, -1)          # shifted k order
    out = np.empty((C, P, A), dtype=np.complex128)
    for c in range(C):
        for p in range(P):
            g = np.ones(A, dtype=np.complex128) if gains is None else gains[c, p].astype(np.complex128)
            V = volt[:, c, p, :]
            F = (V * g[None, :]) @ K                                   # [T, N_p^2] shifted
            G = grad_image[c, p].reshape(-1)
            # sum_k G(k) F_t(k) conj(K_a(k)) -> [T, A]
            S = (F * G[None, :]) @ np.conj(K).T
            out[c, p] = 2.0 * (np.conj(V) * S).mean(0)
    return out


def image_from_footprints(M, volt, gains, n_grid, n_pad):
    """The same image as moff_image, formed as mean_t |sum_a g_a V_a K_a(k)|^2 from the
    per-antenna footprint transforms (used to cross-check the gradient's forward model)."""
    T, C, P, A = volt.shape
    K = footprint_transforms(M, n_grid, n_pad).reshape(A, -1)
    out = np.empty((C, P, n_pad, n_pad))
    for c in range(C):
        for p in range(P):
            g = np.ones(A, dtype=np.complex128) if gains is None else gains[c, p].astype(np.complex128)
            F = (volt[:, c, p, :] * g[None, :]) @ K
            out[c, p] = (np.abs(F) ** 2).mean(0).reshape(n_pad, n_pad)
    return out
