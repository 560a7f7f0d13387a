"""Pins for the FP64 oracle, against things other than itself (CPU only).

Each test names the passage of Thyagarajan et al. (2015) or the mathematical fact it
relies on.  Together they are chosen so that a dropped term, a wrong sign or index,
a transposed operand or a missing normalisation anywhere in the oracle fails one.
"""
import math
import os

import numpy as np
import pytest

from oracle import moff, fx
from paper_1510_08318_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden_rows(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append(line.split())
    return rows


def _cells(pos, n_grid, dx, origin):
    """Antennas at exact cell centres (integer cell coordinates -> metres)."""
    return origin[None, :] + dx * np.asarray(pos, dtype=np.float64)


# ----------------------------------------------------------------------------------
# the mapping and the input decoding against hand-derived fixtures
# ----------------------------------------------------------------------------------
def test_mapping_golden():
    pos = np.array([[1.2, 0.7], [2.5, 2.5], [0.1, 3.2]])
    ptr = np.array([0, 3, 5, 6])
    dxdy = np.array([[0, 0], [0.4, 0], [0.6, 0.1], [0, 0], [-1.0, -2.5], [-0.55, 0.2]])
    w = np.array([0.5, 0.25, 0.25j, 1.0, -2.0, 1 - 1j])
    M = moff.map_antennas(pos, ptr, dxdy, w, 1.0, np.zeros(2), 4).tocoo()
    got = {(int(r), int(c)): complex(v) for r, c, v in zip(M.row, M.col, M.data)}
    want = {(int(r[0]), int(r[1])): complex(float(r[2]), float(r[3])) for r in _golden_rows("mapping_small.txt")}
    assert set(got) == set(want)
    for k in want:
        assert abs(got[k] - want[k]) < 1e-15


def test_mapping_rejects_outside():
    with pytest.raises(ValueError):
        moff.map_antennas(np.array([[3.6, 0.0]]), np.array([0, 1]), np.zeros((1, 2)),
                          np.ones(1), 1.0, np.zeros(2), 4)


def test_ci4_decode_golden():
    for b, re, im in _golden_rows("ci4_decode.txt"):
        v = synth.decode_ci4(np.array([int(b, 16)], dtype=np.uint8))[0]
        assert v == complex(int(re), int(im))


def test_ci4_quantize_roundtrip():
    rng = np.random.default_rng(0)
    v = rng.integers(-7, 8, 100) + 1j * rng.integers(-7, 8, 100)
    b, _ = synth.quantize_ci4(v.astype(np.complex64), scale=1.0)
    assert np.array_equal(synth.decode_ci4(b), v)


# ----------------------------------------------------------------------------------
# closed forms
# ----------------------------------------------------------------------------------
def test_two_element_golden():
    """Textbook two-element fringe (Eq. "dirty-image-MOFF" with N_A = 2)."""
    n_grid, n_pad, dx = 8, 16, 1.0
    pos = _cells([[0, 0], [4, 0]], n_grid, dx, np.zeros(2))       # (x, y): g = (0,0), (0,4)
    M = moff.map_antennas(pos, np.array([0, 1, 2]), np.zeros((2, 2)), np.ones(2), dx, np.zeros(2), n_grid)
    rng = np.random.default_rng(0)
    phi = rng.uniform(0, 2 * np.pi, 5)
    S = 3.0
    v = (math.sqrt(S) * np.exp(1j * phi))[:, None, None, None] * np.ones((5, 1, 1, 2))
    img = moff.moff_image(M, v, None, n_grid, n_pad)[0, 0]
    for ix, val in _golden_rows("two_element.txt"):
        np.testing.assert_allclose(img[:, int(ix)], float(val), atol=1e-12)


@pytest.mark.parametrize("k0", [(0, 0), (3, -5), (-7, 2)])
def test_point_source_closed_form(k0):
    """One noiseless source at a pixel-centred direction, antennas on cell centres with
    single-sample kernels: I(k) = S |sum_a exp(+2 pi i g_a.(k - k0)/N_p)|^2 (the array
    factor), peak S N_A^2 at the source pixel.  Fixes the DFT sign (a source at +s
    appears at +s, Eq. 1 vs. App. B), the axis order, the padding and the 1/T."""
    rng = np.random.default_rng(11)
    n_grid, n_pad = 16, 32
    lam = 4.0
    dx = lam / 2
    origin = np.array([-13.0, 7.5])
    g = rng.choice(n_grid * n_grid, 9, replace=False)
    gy, gx = g // n_grid, g % n_grid
    pos = _cells(np.stack([gx, gy], 1), n_grid, dx, origin)
    A = pos.shape[0]
    M = moff.map_antennas(pos, np.arange(A + 1), np.zeros((A, 2)), np.ones(A), dx, origin, n_grid)
    k0y, k0x = k0
    l0, m0 = k0x * lam / (n_pad * dx), k0y * lam / (n_pad * dx)
    S, T = 2.5, 7
    sky = synth.Sky(np.array([l0]), np.array([m0]), np.array([S]))
    v = synth.voltages(rng, pos, [synth.C_LIGHT / lam], T, 1, sky, 0.0, dtype=np.complex128)
    img = moff.moff_image(M, v, None, n_grid, n_pad)[0, 0]
    iy, ix = np.meshgrid(np.arange(n_pad), np.arange(n_pad), indexing="ij")
    ky, kx = iy - n_pad // 2, ix - n_pad // 2
    af = np.zeros((n_pad, n_pad), dtype=np.complex128)
    for a in range(A):
        af += np.exp(2j * np.pi * (gy[a] * (ky - k0y) + gx[a] * (kx - k0x)) / n_pad)
    want = S * np.abs(af) ** 2
    np.testing.assert_allclose(img, want, rtol=1e-9, atol=1e-9 * want.max())
    assert abs(img[n_pad // 2 + k0y, n_pad // 2 + k0x] - S * A * A) < 1e-8 * S * A * A
    assert np.unravel_index(np.argmax(img), img.shape) == (n_pad // 2 + k0y, n_pad // 2 + k0x)


def test_parseval():
    """sum_k |F(k)|^2 = N_p^2 sum_g |E(g)|^2 for the unnormalised padded DFT, so the
    integrated image sums to N_p^2 times the mean gridded power."""
    wl = synth.workload_tiny(n_time=8)
    M = moff.map_antennas(wl.pos, wl.kern_ptr, wl.kern_dxdy, wl.kern_w, wl.dx, wl.origin, wl.n_grid)
    img = moff.moff_image(M, wl.volt, None, wl.n_grid, wl.n_pad)[0, 0]
    E = moff.grid_efields(M, wl.volt[:, 0, 0, :], np.ones(wl.n_ant), wl.n_grid)
    want = wl.n_pad ** 2 * (np.abs(E) ** 2).sum((1, 2)).mean()
    assert abs(img.sum() - want) < 1e-10 * want
    assert img.min() >= 0.0                       # |.|^2 averaged: non-negative


def test_gridding_is_sparse_matvec():
    """Eq. "gridding-convolution": W(r) = M 1 sums each antenna's (unit-sum) weights, so
    the array illumination integrates to N_A; E(r) = M E(a) for a single active antenna
    reproduces that antenna's footprint scaled by its voltage."""
    wl = synth.workload_tiny(n_time=2)
    M = moff.map_antennas(wl.pos, wl.kern_ptr, wl.kern_dxdy, wl.kern_w, wl.dx, wl.origin, wl.n_grid)
    W = moff.aperture_weights(M)
    assert abs(W.sum() - wl.n_ant) < 1e-12
    v = np.zeros((1, wl.n_ant), dtype=np.complex128)
    v[0, 3] = 2 - 1j
    E = moff.grid_efields(M, v, np.ones(wl.n_ant), wl.n_grid).ravel()
    col = np.asarray(M[:, 3].todense()).ravel()
    np.testing.assert_allclose(E, (2 - 1j) * col, atol=1e-15)


# ----------------------------------------------------------------------------------
# the two routes agree (Sec. 2, Eqs. "dirty-image-FX" and "dirty-image-MOFF")
# ----------------------------------------------------------------------------------
@pytest.fixture(scope="module")
def tiny():
    wl = synth.workload_tiny(n_time=16)
    M = moff.map_antennas(wl.pos, wl.kern_ptr, wl.kern_dxdy, wl.kern_w, wl.dx, wl.origin, wl.n_grid)
    rng = np.random.default_rng(4)
    gains = synth.random_gains(rng, (1, 1, wl.n_ant)).astype(np.complex128)
    return wl, M, gains


def test_moff_equals_fx_exact(tiny):
    wl, M, gains = tiny
    I_m = moff.moff_image(M, wl.volt, gains, wl.n_grid, wl.n_pad)
    I_x = fx.fx_image(M, wl.volt, gains, wl.n_grid, wl.n_pad)
    assert np.abs(I_x.imag).max() < 1e-9 * I_m.max()
    rel = np.linalg.norm(I_m - I_x.real) / np.linalg.norm(I_m)
    assert rel < 1e-12


def test_moff_minus_autocorr_equals_fx_cross(tiny):
    """Sec. 4.2: removing the antenna auto-correlation term from the MOFF image leaves the
    FX image formed from cross-correlations only (a != b)."""
    wl, M, gains = tiny
    I_m = moff.moff_image(M, wl.volt, gains, wl.n_grid, wl.n_pad)
    A = moff.autocorr_term(M, wl.volt, gains, wl.n_grid, wl.n_pad)
    I_x = fx.fx_image(M, wl.volt, gains, wl.n_grid, wl.n_pad, exclude_auto=True).real
    rel = np.linalg.norm((I_m - A) - I_x) / np.linalg.norm(I_m)
    assert rel < 1e-12
    assert A.min() >= 0.0


def test_brute_force_sky_dft():
    """Direct evaluation with no grid array and no DFT matrix: every footprint sample of
    every antenna contributes w g V exp(+2 pi i cell.k / N_p) at every pixel."""
    rng = np.random.default_rng(5)
    n_grid, n_pad, dx = 6, 12, 1.5
    origin = np.array([0.3, -0.2])
    A, T = 5, 4
    pos = origin + rng.uniform(1.0, (n_grid - 2) * dx, (A, 2))
    kerns = [(rng.uniform(-0.9, 0.9, (3, 2)), rng.standard_normal(3) + 1j * rng.standard_normal(3)) for _ in range(A)]
    ptr, dxdy, w = synth.pack_kernels(kerns)
    gains = (rng.standard_normal((1, 1, A)) + 1j * rng.standard_normal((1, 1, A)))
    v = rng.standard_normal((T, 1, 1, A)) + 1j * rng.standard_normal((T, 1, 1, A))
    M = moff.map_antennas(pos, ptr, dxdy, w, dx, origin, n_grid)
    img = moff.moff_image(M, v, gains, n_grid, n_pad)[0, 0]
    want = np.zeros((n_pad, n_pad))
    for iy in range(n_pad):
        for ix in range(n_pad):
            ky, kx = iy - n_pad // 2, ix - n_pad // 2
            acc = 0.0
            for t in range(T):
                f = 0j
                for a in range(A):
                    for k in range(ptr[a], ptr[a + 1]):
                        cx = math.floor((pos[a, 0] + dxdy[k, 0] - origin[0]) / dx + 0.5)
                        cy = math.floor((pos[a, 1] + dxdy[k, 1] - origin[1]) / dx + 0.5)
                        f += w[k] * gains[0, 0, a] * v[t, 0, 0, a] * np.exp(2j * np.pi * (cx * kx + cy * ky) / n_pad)
                acc += abs(f) ** 2
            want[iy, ix] = acc / T
    np.testing.assert_allclose(img, want, rtol=1e-10, atol=1e-12 * want.max())


# ----------------------------------------------------------------------------------
# invariants
# ----------------------------------------------------------------------------------
def test_invariants(tiny):
    wl, M, gains = tiny
    I0 = moff.moff_image(M, wl.volt, gains, wl.n_grid, wl.n_pad)
    # integer-cell translation of the whole array leaves |F| unchanged
    M2 = moff.map_antennas(wl.pos + np.array([2 * wl.dx, -3 * wl.dx]), wl.kern_ptr, wl.kern_dxdy,
                           wl.kern_w, wl.dx, wl.origin, wl.n_grid)
    I1 = moff.moff_image(M2, wl.volt, gains, wl.n_grid, wl.n_pad)
    assert np.linalg.norm(I1 - I0) < 1e-12 * np.linalg.norm(I0)
    # V -> c V scales the image by |c|^2
    c = 0.3 - 1.7j
    I2 = moff.moff_image(M, wl.volt * c, gains, wl.n_grid, wl.n_pad)
    assert np.linalg.norm(I2 - abs(c) ** 2 * I0) < 1e-12 * np.linalg.norm(I2)
    # a global gain phase is invisible; gains act as a per-antenna scaling of V
    I3 = moff.moff_image(M, wl.volt, gains * np.exp(0.7j), wl.n_grid, wl.n_pad)
    assert np.linalg.norm(I3 - I0) < 1e-12 * np.linalg.norm(I0)
    I4 = moff.moff_image(M, wl.volt * gains[0, 0][None, None, None, :], None, wl.n_grid, wl.n_pad)
    assert np.linalg.norm(I4 - I0) < 1e-12 * np.linalg.norm(I0)


def test_homogeneous_weighting():
    """Sec. 5, Eq. "wt-dirty-image-homogeneous": for identical antenna kernels the image is
    the kernel's power pattern |K(k)|^2 times the image of point-like antennas."""
    rng = np.random.default_rng(6)
    n_grid, n_pad, dx = 16, 32, 1.0
    origin = np.zeros(2)
    A, T = 7, 5
    cells = rng.choice(np.arange(3, n_grid - 3), (A, 2))
    pos = _cells(cells, n_grid, dx, origin) + 0.2          # identical sub-cell offset
    kd = np.array([[0.0, 0.0], [1.0, 0.0], [0.0, 1.0], [-1.1, 0.4], [0.6, -1.2]])
    kw = rng.standard_normal(5) + 1j * rng.standard_normal(5)
    v = rng.standard_normal((T, 1, 1, A)) + 1j * rng.standard_normal((T, 1, 1, A))
    ptr, dxdy, w = synth.pack_kernels([(kd, kw)] * A)
    M = moff.map_antennas(pos, ptr, dxdy, w, dx, origin, n_grid)
    M1 = moff.map_antennas(pos, np.arange(A + 1), np.zeros((A, 2)), np.ones(A), dx, origin, n_grid)
    I = moff.moff_image(M, v, None, n_grid, n_pad)[0, 0]
    I1 = moff.moff_image(M1, v, None, n_grid, n_pad)[0, 0]
    # kernel pattern relative to the antenna's own cell
    c0 = np.floor((pos[0] - origin) / dx + 0.5).astype(int)
    K = np.zeros((n_pad, n_pad), dtype=np.complex128)
    iy, ix = np.meshgrid(np.arange(n_pad), np.arange(n_pad), indexing="ij")
    for (ddx, ddy), ww in zip(kd, kw):
        cx = math.floor((pos[0, 0] + ddx - origin[0]) / dx + 0.5) - c0[0]
        cy = math.floor((pos[0, 1] + ddy - origin[1]) / dx + 0.5) - c0[1]
        K += ww * np.exp(2j * np.pi * (cx * (ix - n_pad // 2) + cy * (iy - n_pad // 2)) / n_pad)
    np.testing.assert_allclose(I, np.abs(K) ** 2 * I1, rtol=1e-9, atol=1e-10 * I.max())


def test_footprint_route_matches_direct(tiny):
    wl, M, gains = tiny
    I_m = moff.moff_image(M, wl.volt, gains, wl.n_grid, wl.n_pad)
    I_k = moff.image_from_footprints(M, wl.volt, gains, wl.n_grid, wl.n_pad)
    assert np.linalg.norm(I_k - I_m) < 1e-12 * np.linalg.norm(I_m)


# ----------------------------------------------------------------------------------
# the gradient against central finite differences
# ----------------------------------------------------------------------------------
def test_grad_gains_finite_difference():
    rng = np.random.default_rng(7)
    n_grid, n_pad, dx = 8, 16, 1.0
    A, T, C, P = 6, 5, 2, 1
    origin = np.zeros(2)
    pos = rng.uniform(1.5, n_grid - 2.5, (A, 2))
    kerns = [synth.kernel_square(1.5, 0.5) for _ in range(A)]
    ptr, dxdy, w = synth.pack_kernels(kerns)
    M = moff.map_antennas(pos, ptr, dxdy, w, dx, origin, n_grid)
    v = rng.standard_normal((T, C, P, A)) + 1j * rng.standard_normal((T, C, P, A))
    g = rng.standard_normal((C, P, A)) + 1j * rng.standard_normal((C, P, A))
    I_model = rng.uniform(0, 1, (C, P, n_pad, n_pad))

    def loss(gg):
        I = moff.moff_image(M, v, gg, n_grid, n_pad)
        return float(((I - I_model) ** 2).sum())

    I = moff.moff_image(M, v, g, n_grid, n_pad)
    grad = moff.grad_gains(M, v, g, n_grid, n_pad, 2 * (I - I_model))
    h = 1e-6
    fd = np.zeros_like(grad)
    for c in range(C):
        for a in range(A):
            for part in (1.0, 1j):
                gp, gm = g.copy(), g.copy()
                gp[c, 0, a] += h * part
                gm[c, 0, a] -= h * part
                d = (loss(gp) - loss(gm)) / (2 * h)
                fd[c, 0, a] += d * part
    np.testing.assert_allclose(grad, fd, rtol=1e-6, atol=1e-6 * np.abs(fd).max())


# ----------------------------------------------------------------------------------
# cross-polarisation products (Sec. 3; App. A image module)
# ----------------------------------------------------------------------------------
def _dual_pol(wl, alpha, seed):
    """[T, 1, 2, A]: pol X = the workload's voltages, pol Y = alpha X + independent noise."""
    rng = np.random.default_rng(seed)
    vx = wl.volt[:, :1, 0, :]
    noise = rng.standard_normal(vx.shape) + 1j * rng.standard_normal(vx.shape)
    return np.stack([vx, alpha * vx + 0.5 * noise], axis=2)


def test_cross_pol_equals_fx_exact(tiny):
    """MOFF cross-polarisation products equal the FX route with cross-polarised visibilities
    V^{pq}_ab = <E_ap E_bq^*> (Sec. 2 equivalence, per polarisation pair)."""
    wl, M, gains = tiny
    v = _dual_pol(wl, 0.6 - 0.3j, 11)
    g = np.stack([gains[:, 0], np.conj(gains[:, 0]) * 1.1], axis=1)     # [1, 2, A]
    I_m = moff.moff_cross_image(M, v, g, wl.n_grid, wl.n_pad)
    I_x = fx.fx_cross_image(M, v, g, wl.n_grid, wl.n_pad)
    rel = np.linalg.norm(I_m - I_x) / np.linalg.norm(I_m)
    assert rel < 1e-12
    assert np.linalg.norm(I_m[0, 0, 1]) > 0.1 * np.linalg.norm(I_m[0, 0, 0])   # a real XY signal


def test_cross_pol_special_cases(tiny):
    """Diagonal = the single-pol image; YX = conj(XY); for a fully polarised field E_Y = alpha E_X
    the products are XY = conj(alpha) XX and YY = |alpha|^2 XX (a swapped conjugate fails)."""
    wl, M, _ = tiny
    alpha = 0.7 + 0.4j
    vx = wl.volt[:, :1, 0, :]
    v = np.stack([vx, alpha * vx], axis=2)
    I = moff.moff_cross_image(M, v, None, wl.n_grid, wl.n_pad)
    xx = moff.moff_image(M, v, None, wl.n_grid, wl.n_pad)
    np.testing.assert_allclose(I[0, 0, 0].real, xx[0, 0], rtol=1e-12, atol=1e-12 * xx.max())
    np.testing.assert_allclose(I[0, 1, 1].real, xx[0, 1], rtol=1e-12, atol=1e-12 * xx.max())
    np.testing.assert_allclose(I[0, 1, 0], np.conj(I[0, 0, 1]), rtol=0, atol=1e-12 * xx.max())
    np.testing.assert_allclose(I[0, 0, 1], np.conj(alpha) * I[0, 0, 0], rtol=0, atol=1e-12 * xx.max())
    np.testing.assert_allclose(I[0, 1, 1], abs(alpha) ** 2 * I[0, 0, 0], rtol=0, atol=1e-12 * xx.max())


def test_cross_pol_parseval(tiny):
    """sum_k I_XY(k) = N_p^2 mean_t sum_g E_X(g) conj(E_Y(g)) (Parseval for the product)."""
    wl, M, _ = tiny
    v = _dual_pol(wl, -0.2 + 0.9j, 12)
    I = moff.moff_cross_image(M, v, None, wl.n_grid, wl.n_pad)
    one = np.ones(wl.n_ant, dtype=np.complex128)
    ex = moff.grid_efields(M, v[:, 0, 0, :], one, wl.n_grid)
    ey = moff.grid_efields(M, v[:, 0, 1, :], one, wl.n_grid)
    want = wl.n_pad ** 2 * (ex * np.conj(ey)).sum(axis=(1, 2)).mean()
    assert abs(I[0, 0, 1].sum() - want) < 1e-10 * abs(want)


# ----------------------------------------------------------------------------------
# heterogeneous arrays: effective weighting and the isotropic estimate (Sec. 5)
# ----------------------------------------------------------------------------------
def _on_grid_square(n_cells, dx):
    """Uniform square aperture whose samples sit exactly on cell centres (n_cells per side,
    odd), so the gridded footprint equals the aperture table."""
    c = (np.arange(n_cells) - (n_cells - 1) / 2) * dx
    xx, yy = np.meshgrid(c, c, indexing="xy")
    d = np.stack([xx.ravel(), yy.ravel()], axis=1)
    return d, np.full(d.shape[0], 1.0 / d.shape[0], dtype=np.complex128)


def _two_type_on_grid(n1, n2, n_grid=32, n_pad=64, dx=1.0, seed=2):
    rng = np.random.default_rng(seed)
    cells = rng.choice(np.arange(4, n_grid - 4), size=(n1 + n2, 2))
    origin = np.zeros(2)
    pos = _cells(cells, n_grid, dx, origin)
    kern = [_on_grid_square(1, dx)] * n1 + [_on_grid_square(5, dx)] * n2
    ptr, dxdy, w = synth.pack_kernels(kern)
    M = moff.map_antennas(pos, ptr, dxdy, w, dx, origin, n_grid)
    return pos, kern, ptr, dxdy, w, M, origin


def _brute_K(d, w, n_pad, dx):
    """|K(k)|^2 of one footprint table by a direct sum over its samples (shifted pixels)."""
    k = np.arange(n_pad) - n_pad // 2
    out = np.zeros((n_pad, n_pad), dtype=np.complex128)
    for (x, y), wt in zip(d, w):
        gx, gy = int(round(x / dx)), int(round(y / dx))
        out += wt * np.exp(2j * np.pi * (gy * k[:, None] + gx * k[None, :]) / n_pad)
    return np.abs(out) ** 2


def test_weff_closed_forms():
    """Sec. 5: homogeneous array -> W_eff = |K|^4; two types -> [n1 (n1-1) |K1|^4 +
    n2 (n2-1) |K2|^4 + 2 n1 n2 |K1|^2 |K2|^2] / (N (N-1)) (ordered pairs, so the mixed
    term counts twice); W_eff = 1 at k = 0 for unit-sum weights."""
    n1, n2 = 7, 5
    pos, kern, ptr, dxdy, w, M, origin = _two_type_on_grid(n1, n2)
    W = moff.weff_opt(M, 32, 64)
    P1 = _brute_K(*kern[0], 64, 1.0)
    P2 = _brute_K(*kern[-1], 64, 1.0)
    N = n1 + n2
    want = (n1 * (n1 - 1) * P1 ** 2 + n2 * (n2 - 1) * P2 ** 2 + 2 * n1 * n2 * P1 * P2) / (N * (N - 1))
    np.testing.assert_allclose(W, want, rtol=1e-10, atol=1e-13)
    assert abs(W[32, 32] - 1.0) < 1e-12
    Mh = moff.map_antennas(pos[:n2], ptr[:n2 + 1], dxdy, w, 1.0, origin, 32)   # first n2 antennas: type 1
    np.testing.assert_allclose(moff.weff_opt(Mh, 32, 64), P1 ** 2, rtol=1e-10, atol=1e-13)


def test_isotropic_estimate_recovers_flux():
    """Sec. 5 with W^G = W^I: a single noiseless source at a pixel centre seen by a two-type
    array whose apertures lie on the grid cells; the isotropic estimate at the source pixel
    equals the flux exactly (cross-only image / W_eff), and the all-pairs image does not."""
    n1, n2, n_grid, n_pad, dx = 6, 6, 32, 64, 1.0
    pos, kern, ptr, dxdy, w, M, origin = _two_type_on_grid(n1, n2, n_grid, n_pad, dx)
    lam = 4.0
    step = lam / (n_pad * dx)
    iy, ix = n_pad // 2 + 3, n_pad // 2 - 5
    sky = synth.Sky(np.array([(ix - n_pad // 2) * step]), np.array([(iy - n_pad // 2) * step]), np.array([7.5]))
    f = synth.C_LIGHT / lam
    v = synth.voltages(np.random.default_rng(0), pos, np.array([f]), 16, 1, sky, 0.0, dtype=np.complex128,
                       apertures=kern)
    img = moff.moff_image(M, v, None, n_grid, n_pad)[0, 0]
    ac = moff.autocorr_term(M, v, None, n_grid, n_pad)[0, 0]
    iso = moff.isotropic_image(img, ac, moff.weff_opt(M, n_grid, n_pad), n1 + n2)
    assert abs(iso[iy, ix] - 7.5) < 1e-9 * 7.5
    assert abs(img[iy, ix] / (n1 + n2) ** 2 - 7.5) > 0.05      # without the normalisation it is off


# ----------------------------------------------------------------------------------
# the F-engine (Sec. 3 "Temporal Fourier transform")
# ----------------------------------------------------------------------------------
def test_fengine_brute_force_tone_parseval():
    rng = np.random.default_rng(3)
    C, T, P, A = 16, 3, 2, 5
    raw = rng.standard_normal((T * C, P, A)) + 1j * rng.standard_normal((T * C, P, A))
    V = moff.fengine(raw, C)
    # brute-force DFT of every block
    j = np.arange(C)
    for t in range(T):
        for c in range(C):
            want = (raw[t * C:(t + 1) * C] * np.exp(-2j * np.pi * j * c / C)[:, None, None]).sum(0)
            np.testing.assert_allclose(V[t, c], want, rtol=1e-12, atol=1e-12)
    # Parseval per block and antenna
    np.testing.assert_allclose((np.abs(V) ** 2).sum(1), C * (np.abs(raw.reshape(T, C, P, A)) ** 2).sum(1),
                               rtol=1e-12)
    # a pure tone exp(+2 pi i c0 j / C) lands in bin c0 with value C (sign and bin order)
    c0 = 5
    tone = np.exp(2j * np.pi * c0 * np.arange(2 * C) / C)[:, None, None] * np.ones((1, 1, 2))
    Vt = moff.fengine(tone, C)
    assert np.allclose(Vt[:, c0], C) and np.abs(np.delete(Vt, c0, axis=1)).max() < 1e-9


# ----------------------------------------------------------------------------------
# the X-engine of the FX route (Sec. 3, Eq. "cc-vis")
# ----------------------------------------------------------------------------------
def test_visibilities_closed_form():
    """For antenna b carrying a scaled copy V_b = c V_a of antenna a's voltage,
    V_ab = g_a conj(g_b) conj(c) <|V_a|^2> and V_ba = conj(V_ab): fixes which side carries
    the conjugate and where the gains enter.  The diagonal is the antenna power, the matrix
    is Hermitian, and the cross-polarised form with q = p is the single-pol form."""
    rng = np.random.default_rng(21)
    T, A = 40, 4
    va = rng.standard_normal(T) + 1j * rng.standard_normal(T)
    c = 0.3 - 1.2j
    v = np.stack([va, c * va, rng.standard_normal(T) + 0j, 1j * va], axis=1)   # [T, A]
    g = np.array([1.0 + 0.5j, -0.4 + 0.8j, 0.9 + 0j, 0.2 - 0.7j])
    V = fx.visibilities(v, g)
    pa = (np.abs(va) ** 2).sum() / T
    assert abs(V[0, 1] - g[0] * np.conj(g[1]) * np.conj(c) * pa) < 1e-12 * pa
    assert abs(V[1, 0] - np.conj(V[0, 1])) < 1e-12 * pa
    assert abs(V[0, 3] - g[0] * np.conj(g[3]) * (-1j) * pa) < 1e-12 * pa
    np.testing.assert_allclose(np.diag(V).real, moff.antenna_power(v, g), rtol=1e-12)
    np.testing.assert_allclose(V, np.conj(V.T), rtol=0, atol=1e-12 * pa)
    Vx = fx.visibilities(v, g, exclude_auto=True)
    assert np.all(np.diag(Vx) == 0) and np.array_equal(Vx[0, 1:], V[0, 1:])
    np.testing.assert_allclose(fx.cross_visibilities(v, g, v, g), V, rtol=0, atol=1e-15 * pa)
