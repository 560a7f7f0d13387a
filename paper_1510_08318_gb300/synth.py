"""Seeded synthetic inputs for the MOFF imaging step.

This module produces *inputs* only: antenna layouts, sampled aperture-illumination
tables, point-source skies, channelised antenna voltages and their 4+4-bit / FP16
encodings, and complex gains.  It contains none of the imaging method's arithmetic
(no antenna-to-grid mapping, gridding, spatial transform, squaring or averaging), so
the FP64 oracle and the CUDA library can both be fed from it without sharing code.

Shapes follow the paper's workloads (Table 1: LWA1-like, HERA-331-like layouts) and
the measurement equation of Sec. 2 (Eq. "measured-E-field"): each antenna sees
    V_a(t) = sum_s A_s(t) exp(-2 pi i r_a . s_hat / lambda) + n_a(t)
with an isotropic element response, or, for the heterogeneous-array workload of Sec. 5,
each antenna's far-field pattern.  All generators take an explicit numpy Generator
(PCG64) so every input is reproducible from a seed.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

C_LIGHT = 299792458.0


# ----------------------------------------------------------------------------------
# layouts (metres, [A, 2] float64: x, y)
# ----------------------------------------------------------------------------------
def layout_rect(rng, n_ant, width, height):
    return np.stack([rng.uniform(-width / 2, width / 2, n_ant),
                     rng.uniform(-height / 2, height / 2, n_ant)], axis=1)


def layout_ellipse(rng, n_ant, diam_x, diam_y):
    """Uniform inside an ellipse of the given full axes."""
    out = np.empty((0, 2))
    while out.shape[0] < n_ant:
        p = np.stack([rng.uniform(-1, 1, 4 * n_ant), rng.uniform(-1, 1, 4 * n_ant)], axis=1)
        p = p[(p ** 2).sum(1) <= 1.0]
        out = np.concatenate([out, p])
    out = out[:n_ant]
    return out * np.array([diam_x / 2, diam_y / 2])


def layout_disk(rng, n_ant, diameter):
    return layout_ellipse(rng, n_ant, diameter, diameter)


def layout_rect_min_sep(rng, n_ant, width, height, min_sep):
    """Uniform in a width x height box, drawn one by one and rejected closer than min_sep to an
    earlier antenna (tiles that do not overlap)."""
    pts = []
    while len(pts) < n_ant:
        p = np.array([rng.uniform(-width / 2, width / 2), rng.uniform(-height / 2, height / 2)])
        if all(math.hypot(p[0] - q[0], p[1] - q[1]) >= min_sep for q in pts):
            pts.append(p)
    return np.array(pts, dtype=np.float64)


def layout_hex(n_side, spacing):
    """Hexagonal close-packed core with n_side antennas per side (3 n (n-1) + 1 total)."""
    pts = []
    r = n_side - 1
    for q in range(-r, r + 1):
        for s in range(max(-r, -q - r), min(r, -q + r) + 1):
            x = spacing * (q + s / 2.0)
            y = spacing * (s * math.sqrt(3) / 2.0)
            pts.append((x, y))
    return np.array(pts, dtype=np.float64)


# ----------------------------------------------------------------------------------
# sampled aperture illumination tables: offsets [K, 2] (m) and weights [K] complex,
# normalised to sum 1 (Sec. 4.2: auto-correlation weights normalised to unit sum)
# ----------------------------------------------------------------------------------
def _lattice(half, h):
    n = max(1, int(math.ceil(2 * half / h - 1e-9)))
    hh = 2 * half / n
    c = (np.arange(n) + 0.5) * hh - half
    xx, yy = np.meshgrid(c, c, indexing="xy")
    return np.stack([xx.ravel(), yy.ravel()], axis=1)


def kernel_square(side, h):
    """Uniform square aperture of the given side, sampled on a lattice of step <= h."""
    d = _lattice(side / 2, h)
    w = np.full(d.shape[0], 1.0 / d.shape[0], dtype=np.complex128)
    return d, w


def kernel_gaussian(sigma, h, n_sigma=3.0):
    """Gaussian illumination, truncated at radius n_sigma * sigma."""
    rad = n_sigma * sigma
    d = _lattice(rad, h)
    r2 = (d ** 2).sum(1)
    keep = r2 <= rad * rad
    d, r2 = d[keep], r2[keep]
    w = np.exp(-0.5 * r2 / sigma ** 2)
    return d, (w / w.sum()).astype(np.complex128)


def kernel_disk(diameter, h):
    """Uniformly illuminated circular aperture (far field: Airy pattern)."""
    rad = diameter / 2
    d = _lattice(rad, h)
    keep = (d ** 2).sum(1) <= rad * rad
    if not keep.any():
        keep[np.argmin((d ** 2).sum(1))] = True
    d = d[keep]
    return d, np.full(d.shape[0], 1.0 / d.shape[0], dtype=np.complex128)


def kernel_point():
    return np.zeros((1, 2)), np.ones(1, dtype=np.complex128)


def pack_kernels(kernels):
    """List of (dxdy, w) per antenna -> CSR (kern_ptr [A+1] int32, dxdy [nt,2] f64, w [nt] c128)."""
    ptr = np.zeros(len(kernels) + 1, dtype=np.int32)
    ptr[1:] = np.cumsum([k[0].shape[0] for k in kernels])
    dxdy = np.concatenate([k[0] for k in kernels]).astype(np.float64)
    w = np.concatenate([k[1] for k in kernels]).astype(np.complex128)
    return ptr, dxdy, w


def centred_origin(pos, reach, dx, n_grid):
    """Grid origin (centre of cell (0,0), metres) putting the array's bounding box,
    widened by the kernel reach, in the middle of an n_grid x n_grid grid."""
    lo = pos.min(0) - reach
    hi = pos.max(0) + reach
    mid = 0.5 * (lo + hi)
    return mid - dx * (n_grid - 1) / 2.0


# ----------------------------------------------------------------------------------
# skies and voltages
# ----------------------------------------------------------------------------------
@dataclass
class Sky:
    l: np.ndarray
    m: np.ndarray
    flux: np.ndarray


def sky_box(rng, n_src, lmax, flux_lo, flux_hi):
    return Sky(rng.uniform(-lmax, lmax, n_src), rng.uniform(-lmax, lmax, n_src),
               rng.uniform(flux_lo, flux_hi, n_src))


def sky_powerlaw_hemisphere(rng, n_src, s_lo, s_hi, index=-1.5):
    """dN/dS ~ S^index on [s_lo, s_hi]; directions uniform over the visible hemisphere."""
    a = index + 1.0
    u = rng.uniform(0, 1, n_src)
    flux = (s_lo ** a + u * (s_hi ** a - s_lo ** a)) ** (1.0 / a)
    z = rng.uniform(0, 1, n_src)
    phi = rng.uniform(0, 2 * np.pi, n_src)
    rho = np.sqrt(1 - z * z)
    return Sky(rho * np.cos(phi), rho * np.sin(phi), flux)


def voltages(rng, pos, freqs_hz, n_time, n_pol, sky: Sky, noise_sigma, dtype=np.complex64, apertures=None):
    """V[t, c, p, a] = sum_s P_a(s_s) sqrt(S_s) e^{i phi_{t,p,s}} e^{-2 pi i r_a . s_s / lambda_c} + n.

    Source phases are drawn independently per (time, channel, pol, source): each sample is
    a fresh realisation of a stochastic sky.  Noise is circular complex Gaussian with
    per-sample variance noise_sigma**2.  The element response P_a is isotropic (1) unless
    `apertures` gives each antenna's aperture as a sample table (offsets [n, 2] m, weights
    [n]); then P_a(s) = sum_k w_k e^{-2 pi i delta_k . s / lambda}, the far-field voltage
    pattern of that aperture (the measurement equation of Sec. 2 with antenna beams).
    """
    n_ant = pos.shape[0]
    out = np.empty((n_time, len(freqs_hz), n_pol, n_ant), dtype=dtype)
    work = np.complex128 if np.dtype(dtype) == np.complex128 else np.complex64
    amp = np.sqrt(sky.flux)
    for c, f in enumerate(freqs_hz):
        lam = C_LIGHT / f
        geo = np.outer(sky.l, pos[:, 0]) + np.outer(sky.m, pos[:, 1])      # [S, A] metres
        steer = np.exp(-2j * np.pi * geo / lam)
        if apertures is not None:
            for a, (d, w) in enumerate(apertures):
                ph = np.outer(sky.l, d[:, 0]) + np.outer(sky.m, d[:, 1])   # [S, n] metres
                steer[:, a] *= np.exp(-2j * np.pi * ph / lam) @ w
        steer = steer.astype(work)
        for p in range(n_pol):
            ph = rng.uniform(0, 2 * np.pi, (n_time, sky.flux.size))
            src = (amp * np.exp(1j * ph)).astype(work)                       # [T, S]
            sig = src @ steer
            nz = (rng.standard_normal((n_time, n_ant)) + 1j * rng.standard_normal((n_time, n_ant)))
            nz *= noise_sigma / math.sqrt(2.0)
            out[:, c, p, :] = sig + nz.astype(work)
    return out


def random_gains(rng, shape, amp_spread=0.2):
    amp = 1.0 + rng.uniform(-amp_spread, amp_spread, shape)
    ph = rng.uniform(0, 2 * np.pi, shape)
    return (amp * np.exp(1j * ph)).astype(np.complex64)


# ----------------------------------------------------------------------------------
# encodings
# ----------------------------------------------------------------------------------
def quantize_ci4(v, rms_levels=2.0, scale=None):
    """Complex -> signed 4+4-bit byte: high nibble = real, low nibble = imag, both
    two's complement in [-7, 7] (-8 unused).  Scaled so the per-component rms is
    rms_levels, rounded half away from zero, clipped."""
    if scale is None:
        rms = math.sqrt(float(np.mean(np.abs(v.astype(np.complex128)) ** 2)) / 2.0)
        scale = rms_levels / rms
    re = np.clip(_round_half_away(v.real * scale), -7, 7).astype(np.int8)
    im = np.clip(_round_half_away(v.imag * scale), -7, 7).astype(np.int8)
    b = ((re.astype(np.uint8) & 0xF) << 4) | (im.astype(np.uint8) & 0xF)
    return b.astype(np.uint8), scale


def _round_half_away(x):
    return np.sign(x) * np.floor(np.abs(x) + 0.5)


def decode_ci4(b):
    """Signed 4+4-bit byte -> complex128 (exact)."""
    b = np.asarray(b, dtype=np.uint8)
    hi = (b >> 4).astype(np.int16)
    lo = (b & 0xF).astype(np.int16)
    hi = np.where(hi >= 8, hi - 16, hi)
    lo = np.where(lo >= 8, lo - 16, lo)
    return hi.astype(np.float64) + 1j * lo.astype(np.float64)


def to_f16_pairs(v):
    """Complex -> [..., 2] float16 (re, im)."""
    return np.stack([v.real, v.imag], axis=-1).astype(np.float16)


def from_f16_pairs(x):
    x = np.asarray(x, dtype=np.float64)
    return x[..., 0] + 1j * x[..., 1]


def to_c64_pairs(v):
    return np.stack([v.real, v.imag], axis=-1).astype(np.float32)


# ----------------------------------------------------------------------------------
# the workloads
# ----------------------------------------------------------------------------------
@dataclass
class Workload:
    name: str
    pos: np.ndarray                # [A, 2] f64, metres
    kern_ptr: np.ndarray           # [A+1] int32
    kern_dxdy: np.ndarray          # [nt, 2] f64, metres
    kern_w: np.ndarray             # [nt] complex128
    dx: float                      # grid spacing, metres
    origin: np.ndarray             # [2] f64, centre of cell (0, 0)
    n_grid: int                    # unpadded grid side N_g
    n_pad: int                     # padded side N_p (= image side)
    freqs: np.ndarray              # [C] Hz
    n_pol: int
    n_time: int
    vdtype: str                    # "c64" | "f16" | "ci4"
    volt_raw: np.ndarray = None    # encoded voltages as fed to the library
    volt: np.ndarray = None        # the same voltages as complex128 (exact decode)
    gains: np.ndarray = None       # [C, P, A] complex64 or None
    extra: dict = field(default_factory=dict)

    @property
    def n_ant(self):
        return self.pos.shape[0]

    @property
    def n_chan(self):
        return len(self.freqs)


def _finish(wl: Workload, v, vdtype, rng=None):
    wl.vdtype = vdtype
    if vdtype == "ci4":
        b, scale = quantize_ci4(v)
        wl.volt_raw = b
        wl.volt = decode_ci4(b)
        wl.extra["ci4_scale"] = scale
    elif vdtype == "f16":
        wl.volt_raw = to_f16_pairs(v)
        wl.volt = from_f16_pairs(wl.volt_raw)
    else:
        wl.volt_raw = to_c64_pairs(v)
        wl.volt = wl.volt_raw[..., 0].astype(np.float64) + 1j * wl.volt_raw[..., 1].astype(np.float64)
    return wl


def workload_tiny(seed=1, n_time=64):
    """16 antennas uniform in a 20 m x 20 m square, one pol, one channel at 60 MHz,
    3 point sources + unit complex Gaussian noise, 2 m square apertures, spacing lambda/2,
    N_p = 64 (N_g = 32), complex64 voltages."""
    rng = np.random.default_rng(seed)
    f = 60e6
    lam = C_LIGHT / f
    dx = lam / 2
    pos = layout_rect(rng, 16, 20.0, 20.0)
    kd, kw = kernel_square(2.0, dx / 4)
    ptr, dxdy, w = pack_kernels([(kd, kw)] * 16)
    n_grid, n_pad = 32, 64
    origin = centred_origin(pos, 1.0, dx, n_grid)
    sky = sky_box(rng, 3, 0.7, 1.0, 10.0)
    v = voltages(rng, pos, [f], n_time, 1, sky, 1.0)
    wl = Workload("tiny: 16 ant, 1 chan, 1 pol, T=%d, 64x64 image, c64" % n_time,
                  pos, ptr, dxdy, w, dx, origin, n_grid, n_pad, np.array([f]), 1, n_time, "c64")
    wl.extra["sky"] = sky
    return _finish(wl, v, "c64")


def workload_lwa(seed=2, n_chan=128, n_time=1024, n_pol=2, chan_index=None, n_ant=256):
    """LWA-like: 256 antennas uniform in a 100 m x 110 m ellipse, 2 pols, 128 channels over
    30-80 MHz, 1024 samples, 200 power-law sources (index -1.5) over the visible hemisphere
    at per-sample SNR 0.1, signed 4+4-bit voltages, Gaussian apertures (sigma 1.5 m, 3 sigma
    support), spacing lambda/2 at 80 MHz, N_p = 128 (N_g = 64).

    chan_index (optional) selects a subset of the 128 channel frequencies so reduced
    slices keep the full-size layout and frequency axis."""
    rng = np.random.default_rng(seed)
    freqs_all = np.linspace(30e6, 80e6, 128)
    freqs = freqs_all[:n_chan] if chan_index is None else freqs_all[np.asarray(chan_index)]
    dx = C_LIGHT / 80e6 / 2
    pos = layout_ellipse(rng, n_ant, 100.0, 110.0)
    sigma = 1.5
    kd, kw = kernel_gaussian(sigma, dx / 4)
    ptr, dxdy, w = pack_kernels([(kd, kw)] * n_ant)
    n_grid, n_pad = 64, 128
    origin = centred_origin(pos, 3 * sigma, dx, n_grid)
    sky = sky_powerlaw_hemisphere(rng, 200, 1.0, 100.0)
    noise = math.sqrt(sky.flux.sum() / 0.1)
    v = voltages(rng, pos, freqs, n_time, n_pol, sky, noise)
    wl = Workload("LWA-like: %d ant, %d chan, %d pol, T=%d, 128x128 image, ci4"
                  % (n_ant, len(freqs), n_pol, n_time),
                  pos, ptr, dxdy, w, dx, origin, n_grid, n_pad, freqs, n_pol, n_time, "ci4")
    wl.extra["sky"] = sky
    return _finish(wl, v, "ci4")


def workload_hera(seed=3, n_chan=1024, n_time=256):
    """Dense HERA-331-like hexagon (11 per side, 14 m spacing), 1 pol, channels over
    100-200 MHz, FP16 voltages (50 sources + unit noise), 14 m uniform disk apertures
    (far field: Airy disk) on a 2.5 m grid, N_p = 256 (N_g = 128)."""
    rng = np.random.default_rng(seed)
    freqs = np.linspace(100e6, 200e6, 1024)[:n_chan]
    dx = 2.5
    pos = layout_hex(11, 14.0)
    kd, kw = kernel_disk(14.0, dx / 4)
    ptr, dxdy, w = pack_kernels([(kd, kw)] * pos.shape[0])
    n_grid, n_pad = 128, 256
    origin = centred_origin(pos, 7.0, dx, n_grid)
    sky = sky_box(rng, 50, 0.7, 1.0, 10.0)
    v = voltages(rng, pos, freqs, n_time, 1, sky, 1.0)
    wl = Workload("HERA-like: 331 ant, %d chan, 1 pol, T=%d, 256x256 image, f16" % (len(freqs), n_time),
                  pos, ptr, dxdy, w, dx, origin, n_grid, n_pad, freqs, 1, n_time, "f16")
    wl.extra["sky"] = sky
    return _finish(wl, v, "f16")


def workload_calib(seed=5, n_chan=32, n_time=64, n_ant=1024):
    """Gain calibration: 1024 antennas uniform in a 300 m (diameter) disk, 32 channels over
    50-80 MHz, 64 samples, 1 pol, complex64; 50 sources; true gains amplitude 1 +- 0.2,
    uniform phase; Gaussian apertures sigma 1.5 m; N_p = 256 (N_g = 128)."""
    rng = np.random.default_rng(seed)
    freqs = np.linspace(50e6, 80e6, 32)[:n_chan]
    pos = layout_disk(rng, n_ant, 300.0)
    sigma = 1.5
    n_grid, n_pad = 128, 256
    dx = (300.0 + 2 * 3 * sigma) / n_grid
    kd, kw = kernel_gaussian(sigma, dx / 4)
    ptr, dxdy, w = pack_kernels([(kd, kw)] * n_ant)
    origin = centred_origin(pos, 3 * sigma, dx, n_grid)
    sky = sky_box(rng, 50, 0.7, 1.0, 10.0)
    v = voltages(rng, pos, freqs, n_time, 1, sky, 1.0)
    g_true = random_gains(rng, (n_ant,))
    v = v * g_true[None, None, None, :]
    wl = Workload("calibration: %d ant, %d chan, 1 pol, T=%d, 256x256 image, c64" % (n_ant, len(freqs), n_time),
                  pos, ptr, dxdy, w, dx, origin, n_grid, n_pad, freqs, 1, n_time, "c64")
    wl.extra["sky"] = sky
    wl.extra["g_true"] = g_true
    return _finish(wl, v, "c64")


def workload_twotype(seed=6, n_time=256, n_ant=51):
    """Heterogeneous array after Sec. 5: n_ant antennas uniform in a 100 m disk, alternately
    uniform squares of 1.1 m (type 1) and 6.6 m (type 2) sides; one channel at 150 MHz, one
    pol, T samples; 8 point sources of 10-30 Jy at pixel centres along the westward and
    south-westward directions within the type-2 main lobe; voltages carry each antenna's
    far-field pattern; no noise.  Grid 2 m (N_g = 64), N_p = 128, complex64."""
    rng = np.random.default_rng(seed)
    freqs = np.array([150e6])
    lam = C_LIGHT / freqs[0]
    dx = 2.0
    pos = layout_disk(rng, n_ant, 100.0)
    kern = [kernel_square(1.1 if a % 2 == 0 else 6.6, dx / 4) for a in range(n_ant)]
    ptr, dxdy, w = pack_kernels(kern)
    n_grid, n_pad = 64, 128
    origin = centred_origin(pos, 3.3, dx, n_grid)
    step = lam / (n_pad * dx)                       # direction cosine per image pixel
    k = np.array([6, 10, 14, 18])
    l = np.concatenate([-k * step, -k * step / 1.0])
    m = np.concatenate([np.zeros(4), -k * step])
    flux = rng.uniform(10.0, 30.0, 8)
    sky = Sky(l, m, flux)
    v = voltages(rng, pos, freqs, n_time, 1, sky, 0.0, dtype=np.complex128, apertures=kern)
    wl = Workload("two-type: %d ant (1.1 m / 6.6 m squares), 150 MHz, T=%d, 128x128 image, c64" % (n_ant, n_time),
                  pos, ptr, dxdy, w, dx, origin, n_grid, n_pad, freqs, 1, n_time, "c64")
    wl.extra["sky"] = sky
    wl.extra["src_pixel"] = [(int(round(mm / step)) + n_pad // 2, int(round(ll / step)) + n_pad // 2)
                             for ll, mm in zip(l, m)]
    wl.extra["types"] = np.array([a % 2 for a in range(n_ant)])
    return _finish(wl, v, "c64")


def workload_mwa_core(seed=7, dx=0.5):
    """The simulation of the paper's verification (Sec. 4.1) with a synthetic layout in place of
    the MWA's: 51 identical tiles uniform in a 150 m x 150 m box (at least 5 m apart, so that no
    two 4.4 m tiles overlap), uniform 4.4 m square apertures sampled on a lattice of step dx / 4,
    grid spacing dx (0.5 m by default, lambda / 4 at 150 MHz), N_g the least even side above
    (150 m + 4.4 m) / dx + 8 cells (318), N_p = 2 N_g, one channel at 150 MHz, one pol and one
    sample of unit voltages (the synthesised beam), complex64."""
    rng = np.random.default_rng(seed)
    freqs = np.array([150e6])
    side = 4.4
    pos = layout_rect_min_sep(rng, 51, 150.0, 150.0, 5.0)
    kd, kw = kernel_square(side, dx / 4)
    ptr, dxdy, w = pack_kernels([(kd, kw)] * 51)
    n_grid = int(math.ceil((150.0 + side) / dx)) + 8
    n_grid += n_grid % 2
    n_pad = 2 * n_grid
    origin = centred_origin(pos, side / 2, dx, n_grid)
    wl = Workload("MWA-core-like: 51 tiles of 4.4 m in 150 m, unit voltages, %gx%g m grid" % (dx, dx),
                  pos, ptr, dxdy, w, dx, origin, n_grid, n_pad, freqs, 1, 1, "c64")
    wl.extra["tile_side"] = side
    return _finish(wl, np.ones((1, 1, 1, 51), dtype=np.complex128), "c64")


def workload_batch(seed=4, n_sub=64, n_time=128, max_chan=None, max_ant=None, n_src=20):
    """Heterogeneous sub-arrays: antenna counts log-uniform in [32, 2048], positions uniform in
    disks of diameter U(30, 300) m, padded grids N_p uniform over {32, 64, 128, 256, 512}
    (N_g = N_p / 2, spacing (D_array + 21 m) / (N_g - 1) so the array plus the widest aperture
    reach, 10.5 m, fits the grid), channel counts log-uniform in [8, 256] over
    50-200 MHz, FP16 voltages (n_src sources + unit noise).  Every antenna draws its own
    aperture: a square, a Gaussian (sigma = D / 4, 3 sigma support) or a uniform disk, of size
    D ~ U(1, 14) m, sampled on a lattice of step max(dx / 2, D / 64).

    max_chan / max_ant (optional) cap the channel and antenna draws (the layouts keep their
    distributions otherwise) so reduced instances stay cheap to generate and check."""
    rng = np.random.default_rng(seed)
    subs = []
    for s in range(n_sub):
        n_ant = int(round(math.exp(rng.uniform(math.log(32), math.log(2048)))))
        if max_ant is not None:
            n_ant = min(n_ant, max_ant)
        diam = rng.uniform(30.0, 300.0)
        n_pad = int(rng.choice([32, 64, 128, 256, 512]))
        n_chan = int(round(math.exp(rng.uniform(math.log(8), math.log(256)))))
        if max_chan is not None:
            n_chan = min(n_chan, max_chan)
        n_grid = n_pad // 2
        dx = (diam + 21.0) / (n_grid - 1)
        pos = layout_disk(rng, n_ant, diam)
        kerns = []
        for _ in range(n_ant):
            size = rng.uniform(1.0, 14.0)
            kind = rng.integers(0, 3)
            if kind == 0:
                kerns.append(kernel_square(size, max(dx / 2, size / 64)))
            elif kind == 1:
                kerns.append(kernel_gaussian(size / 4, max(dx / 2, size / 64)))
            else:
                kerns.append(kernel_disk(size, max(dx / 2, size / 64)))
        ptr, dxdy, w = pack_kernels(kerns)
        reach = np.abs(dxdy).max() if dxdy.size else 0.0
        origin = centred_origin(pos, reach, dx, n_grid)
        freqs = np.linspace(50e6, 200e6, n_chan)
        sky = sky_box(rng, n_src, 0.7, 1.0, 10.0)
        v = voltages(rng, pos, freqs, n_time, 1, sky, 1.0)
        wl = Workload("sub-array %d: %d ant, %d chan, T=%d, %dx%d image, f16" % (s, n_ant, n_chan, n_time, n_pad, n_pad),
                      pos, ptr, dxdy, w, dx, origin, n_grid, n_pad, freqs, 1, n_time, "f16")
        subs.append(_finish(wl, v, "f16"))
    return subs
