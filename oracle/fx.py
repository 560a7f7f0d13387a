"""FP64 FX (visibility-based, software-holography) imaging route -- TEST INFRASTRUCTURE ONLY.

Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline leg may import this
module.  It shares no code with the CUDA library.

This is the second, independent route to the same image (Sec. 3, Fig. "FX-flowchart"):
  1. X-engine: V_ab = <E_a E_b^*>_t for every ordered antenna pair, autocorrelations
     included unless excluded (Eq. "cc-vis"; gains applied first, Sec. 3 "Calibration");
  2. gridding with the antenna-pair power response: U(d) = sum_ab V_ab B_ab(d), with
     B_ab(d) = sum_g M[g, a] conj(M[g - d, b]) the cross-correlation of the two sampled
     footprints (Eq. "e-field-conv": B^T N^-1 m equals the correlation of the gridded
     fields), d the integer lag on the grid;
  3. one spatial Fourier transform per integration (Eq. "dirty-image-FX") with the
     imaging sign exp(+2 pi i d.k / N_p), evaluated with numpy's FFT on the lag plane
     wrapped onto the N_p x N_p padded grid (with N_p >= 2 N_g no two lags alias).

Time-averaging happens before the transform here, and after squaring in the MOFF
route; the two agree exactly (Sec. 2: "mathematically equivalent").  The dense
grid-covariance form used in step 2 limits this route to small grids (N_g <= 32).

The paper's own visibility-based imager (Sec. 4.3) grids each baseline with the *directly
sampled* antenna-pair power response -- the analytic cross-correlation of the two aperture
illuminations, centred on the baseline -- instead of the correlation of the two gridded
footprints.  `uv_plane_analytic` and `square_pair_response` are that route, for arrays of
identical uniform square apertures (the simulation of Sec. 4.1); it agrees with MOFF only to
the gridding precision the paper reports.
"""
from __future__ import annotations

import numpy as np


def visibilities(volt_t, gain, exclude_auto=False):
    """V_ab = mean_t (g_a V_a)(g_b V_b)^*: [A, A]."""
    vp = volt_t * gain[None, :]
    V = vp.T @ np.conj(vp) / volt_t.shape[0]
    if exclude_auto:
        V = V - np.diag(np.diag(V))
    return V


def uv_plane(M, V, n_grid):
    """U(dy, dx) = sum_ab V_ab sum_g M[g, a] conj(M[g - d, b]) over lags in (-N_g, N_g)^2.

    Returned as [2 N_g - 1, 2 N_g - 1] with lag (dy, dx) at index (dy + N_g - 1, dx + N_g - 1).
    """
    Md = M.toarray()
    C = Md @ V @ np.conj(Md).T                       # grid covariance C[g, g']
    C = C.reshape(n_grid, n_grid, n_grid, n_grid)      # [gy, gx, gy', gx']
    g = np.arange(n_grid)
    dy = (g[:, None, None, None] - g[None, None, :, None]) + (n_grid - 1)
    dx = (g[None, :, None, None] - g[None, None, None, :]) + (n_grid - 1)
    dy = np.broadcast_to(dy, C.shape).ravel()
    dx = np.broadcast_to(dx, C.shape).ravel()
    U = np.zeros((2 * n_grid - 1, 2 * n_grid - 1), dtype=np.complex128)
    np.add.at(U, (dy, dx), C.ravel())
    return U


def image_from_uv(U, n_grid, n_pad):
    """I(k) = sum_d U(d) exp(+2 pi i d.k / N_p), shifted so k = 0 is at (N_p/2, N_p/2)."""
    if 2 * n_grid - 1 > n_pad:
        raise ValueError("lags alias on an N_p grid smaller than 2 N_g - 1")
    P = np.zeros((n_pad, n_pad), dtype=np.complex128)
    lag = np.arange(-(n_grid - 1), n_grid)
    iy = lag % n_pad
    P[np.ix_(iy, iy)] = U
    img = np.fft.ifft2(P) * (n_pad * n_pad)
    return np.fft.fftshift(img)


def fx_image(M, volt, gains, n_grid, n_pad, exclude_auto=False):
    """FX-route image cube [C, P, N_p, N_p] (complex; the imaginary part is roundoff)."""
    T, C, P, A = volt.shape
    out = np.empty((C, P, n_pad, n_pad), dtype=np.complex128)
    for c in range(C):
        for p in range(P):
            g = np.ones(A, dtype=np.complex128) if gains is None else gains[c, p].astype(np.complex128)
            V = visibilities(volt[:, c, p, :], g, exclude_auto)
            out[c, p] = image_from_uv(uv_plane(M, V, n_grid), n_grid, n_pad)
    return out


def cross_visibilities(volt_p, gain_p, volt_q, gain_q):
    """V^{pq}_ab = mean_t (g_ap V_ap)(g_bq V_bq)^*: [A, A] (all pairs, autos included)."""
    vp = volt_p * gain_p[None, :]
    vq = volt_q * gain_q[None, :]
    return vp.T @ np.conj(vq) / volt_p.shape[0]


def fx_cross_image(M, volt, gains, n_grid, n_pad):
    """FX-route cross-polarisation images [C, 2, 2, N_p, N_p]: I^{pq} from the visibilities
    V^{pq} of pol p of antenna a with pol q of antenna b, gridded and transformed as above."""
    T, C, P, A = volt.shape
    out = np.empty((C, 2, 2, n_pad, n_pad), dtype=np.complex128)
    for c in range(C):
        g = [np.ones(A, dtype=np.complex128) if gains is None else gains[c, p].astype(np.complex128)
             for p in range(2)]
        for p in range(2):
            for q in range(2):
                V = cross_visibilities(volt[:, c, p, :], g[p], volt[:, c, q, :], g[q])
                out[c, p, q] = image_from_uv(uv_plane(M, V, n_grid), n_grid, n_pad)
    return out


# ----------------------------------------------------------------------------------
# the paper's visibility-based route: directly sampled pair power responses (Sec. 4.3)
# ----------------------------------------------------------------------------------
def square_pair_response(u, v, side):
    """Cross-correlation of two identical uniform square apertures of the given side, each
    normalised to unit integral (1 / side^2 inside the square), at separation (u, v) metres:
    (side - |u|)(side - |v|) / side^4 inside |u|, |v| < side, else 0.  Integrates to 1."""
    return np.maximum(0.0, side - np.abs(u)) * np.maximum(0.0, side - np.abs(v)) / side ** 4


def uv_plane_analytic(pos, vis, side, dx, n_grid, exclude_auto=True):
    """U(d) = sum_ab V_ab dx^2 R(d dx - (r_a - r_b)), R = square_pair_response: every baseline
    gridded with its directly sampled pair power response, centred on the baseline (the lag
    d = g_a - g_b of the gridded route).  [2 N_g - 1, 2 N_g - 1] in the layout of uv_plane (lag
    (dy, dx) at index (dy + N_g - 1, dx + N_g - 1)); autocorrelations left out unless
    exclude_auto is False."""
    lag = np.arange(-(n_grid - 1), n_grid) * dx
    U = np.zeros((2 * n_grid - 1, 2 * n_grid - 1), dtype=np.complex128)
    A = pos.shape[0]
    for a in range(A):
        for b in range(A):
            if exclude_auto and a == b:
                continue
            bx, by = pos[a, 0] - pos[b, 0], pos[a, 1] - pos[b, 1]
            ix = np.nonzero(np.abs(lag - bx) < side)[0]
            iy = np.nonzero(np.abs(lag - by) < side)[0]
            if ix.size == 0 or iy.size == 0:
                continue
            R = square_pair_response(lag[ix][None, :] - bx, lag[iy][:, None] - by, side)
            U[np.ix_(iy, ix)] += vis[a, b] * dx * dx * R
    return U
