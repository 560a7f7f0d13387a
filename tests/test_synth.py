"""The seeded input generators against the input recipe they implement (CPU only): layouts,
aperture tables, sky statistics, the measurement equation's sign and geometry, noise level,
encodings, and the shapes of every workload (reduced slices of the same layouts)."""
import math

import numpy as np
import pytest

from oracle import moff
from paper_1510_08318_gb300 import synth


def _inside_grid(wl):
    """Every footprint sample maps inside the N_g x N_g grid (the oracle's mapping rejects
    anything outside)."""
    moff.map_antennas(wl.pos, wl.kern_ptr, wl.kern_dxdy, wl.kern_w, wl.dx, wl.origin, wl.n_grid)


def test_layouts():
    rng = np.random.default_rng(0)
    p = synth.layout_ellipse(rng, 5000, 100.0, 110.0)
    assert p.shape == (5000, 2) and np.all((p[:, 0] / 50.0) ** 2 + (p[:, 1] / 55.0) ** 2 <= 1.0 + 1e-12)
    assert abs(p[:, 0].std() - 25.0) < 1.5 and abs(p[:, 1].std() - 27.5) < 1.5   # uniform fill: a/2
    h = synth.layout_hex(11, 14.0)
    assert h.shape == (331, 2)
    d = np.sqrt(((h[:, None, :] - h[None, :, :]) ** 2).sum(-1)) + np.eye(331) * 1e9
    assert abs(d.min() - 14.0) < 1e-9 and np.allclose(d.min(1), 14.0)
    assert np.all(np.sqrt((h ** 2).sum(1)) <= 10 * 14.0 + 1e-9)


@pytest.mark.parametrize("make, reach", [
    (lambda h: synth.kernel_square(2.0, h), math.sqrt(2.0)),
    (lambda h: synth.kernel_gaussian(1.5, h), 4.5),
    (lambda h: synth.kernel_disk(14.0, h), 7.0),
])
def test_aperture_tables(make, reach):
    h = 0.47
    d, w = make(h)
    assert abs(w.sum() - 1.0) < 1e-12 and np.all(w.real > 0) and np.all(w.imag == 0)
    assert np.sqrt((d ** 2).sum(1)).max() <= reach + 1e-12
    steps = np.diff(np.unique(np.round(d[:, 0], 12)))
    assert steps.max() <= h + 1e-12


def test_powerlaw_sky():
    rng = np.random.default_rng(1)
    sky = synth.sky_powerlaw_hemisphere(rng, 200000, 1.0, 100.0)
    assert sky.flux.min() >= 1.0 and sky.flux.max() <= 100.0
    assert np.all(sky.l ** 2 + sky.m ** 2 <= 1.0 + 1e-12)
    # dN/dS ~ S^-1.5: CDF(S) = (1 - S^-0.5) / (1 - 100^-0.5)
    for s in (2.0, 10.0, 50.0):
        want = (1 - s ** -0.5) / (1 - 0.1)
        assert abs(np.mean(sky.flux <= s) - want) < 0.005
    # uniform over the hemisphere: the projected radius has P(rho <= r) = 1 - sqrt(1 - r^2)
    rho = np.sqrt(sky.l ** 2 + sky.m ** 2)
    assert abs(np.mean(rho <= 0.6) - (1 - math.sqrt(1 - 0.36))) < 0.005


def test_measurement_equation_sign_and_noise():
    """One source, no noise: V_a / V_0 = exp(-2 pi i (r_a - r_0) . s / lambda) at every sample
    (Eq. "measured-E-field"); zero sky: per-sample noise variance sigma^2."""
    rng = np.random.default_rng(2)
    pos = np.array([[0.0, 0.0], [3.0, 1.0], [-2.0, 5.0]])
    f = 50e6
    lam = synth.C_LIGHT / f
    sky = synth.Sky(np.array([0.3]), np.array([-0.2]), np.array([4.0]))
    v = synth.voltages(rng, pos, [f], 16, 1, sky, 0.0, dtype=np.complex128)
    want = np.exp(-2j * np.pi * (pos[:, 0] * 0.3 + pos[:, 1] * -0.2) / lam)
    np.testing.assert_allclose(v[:, 0, 0, :] / v[:, 0, 0, :1], np.broadcast_to(want, (16, 3)), atol=1e-12)
    np.testing.assert_allclose(np.abs(v[:, 0, 0, 0]), 2.0, atol=1e-12)            # sqrt(S)
    nz = synth.voltages(rng, pos, [f], 20000, 1, synth.Sky(np.zeros(0), np.zeros(0), np.zeros(0)), 3.0,
                        dtype=np.complex128)
    assert abs(np.mean(np.abs(nz) ** 2) / 9.0 - 1.0) < 0.03


def test_lwa_like_workload():
    wl = synth.workload_lwa(n_chan=2, n_time=8, chan_index=[0, 127])
    assert wl.n_ant == 256 and wl.n_pol == 2 and wl.n_time == 8 and (wl.n_grid, wl.n_pad) == (64, 128)
    np.testing.assert_allclose(wl.freqs, [30e6, 80e6])
    assert abs(wl.dx - synth.C_LIGHT / 80e6 / 2) < 1e-12
    assert np.all((wl.pos[:, 0] / 50.0) ** 2 + (wl.pos[:, 1] / 55.0) ** 2 <= 1.0 + 1e-12)
    assert np.all(np.diff(wl.kern_ptr) == wl.kern_ptr[1])                          # one shared aperture
    assert np.sqrt((wl.kern_dxdy ** 2).sum(1)).max() <= 4.5 + 1e-12
    assert wl.volt_raw.shape == (8, 2, 2, 256) and wl.volt_raw.dtype == np.uint8
    np.testing.assert_array_equal(wl.volt, synth.decode_ci4(wl.volt_raw))
    sky = wl.extra["sky"]
    assert sky.flux.size == 200
    _inside_grid(wl)
    again = synth.workload_lwa(n_chan=2, n_time=8, chan_index=[0, 127])
    np.testing.assert_array_equal(wl.volt_raw, again.volt_raw)                     # seeded


def test_hera_calib_twotype_workloads():
    h = synth.workload_hera(n_chan=2, n_time=4)
    assert h.n_ant == 331 and h.vdtype == "f16" and h.volt_raw.dtype == np.float16
    assert (h.n_grid, h.n_pad, h.dx) == (128, 256, 2.5) and abs(h.freqs[0] - 100e6) < 1
    _inside_grid(h)
    c = synth.workload_calib(n_chan=1, n_time=2)
    assert c.n_ant == 1024 and (c.n_grid, c.n_pad) == (128, 256) and c.vdtype == "c64"
    assert np.all(np.sqrt((c.pos ** 2).sum(1)) <= 150.0 + 1e-9)
    g = c.extra["g_true"]
    assert np.all(np.abs(np.abs(g) - 1.0) <= 0.2 + 1e-6)
    _inside_grid(c)
    t = synth.workload_twotype(n_time=4)
    sides = [np.ptp(t.kern_dxdy[t.kern_ptr[a]:t.kern_ptr[a + 1], 0]) for a in range(t.n_ant)]
    assert all(s < 1.1 for s in sides[0::2]) and all(5.0 < s < 6.6 for s in sides[1::2])
    assert len(t.extra["src_pixel"]) == 8
    _inside_grid(t)


def test_batch_workload():
    subs = synth.workload_batch(n_sub=6, n_time=2, max_chan=2, max_ant=40)
    assert len(subs) == 6
    for wl in subs:
        assert wl.n_pad in (32, 64, 128, 256, 512) and wl.n_grid == wl.n_pad // 2
        assert 1 <= wl.n_chan <= 2 and 32 <= wl.n_ant <= 40 and wl.vdtype == "f16"
        assert 50e6 <= wl.freqs.min() and wl.freqs.max() <= 200e6
        _inside_grid(wl)


def test_mwa_core_like_workload():
    """The verification simulation's layout (Sec. 4.1): 51 tiles of 4.4 m in a 150 m box, no two
    tiles overlapping, unit voltages, every footprint sample on the grid with 2x padding."""
    wl = synth.workload_mwa_core()
    assert wl.n_ant == 51 and wl.n_pad == 2 * wl.n_grid and wl.dx == 0.5
    assert np.abs(wl.pos).max() <= 75.0
    d = np.hypot(*(wl.pos[:, None, :] - wl.pos[None, :, :]).transpose(2, 0, 1))
    assert d[~np.eye(51, dtype=bool)].min() >= 5.0
    assert np.all(wl.volt == 1.0) and wl.volt.shape == (1, 1, 1, 51)
    k = wl.kern_dxdy[wl.kern_ptr[0]:wl.kern_ptr[1]]
    assert np.abs(k).max() < 2.2 and abs(wl.kern_w[wl.kern_ptr[0]:wl.kern_ptr[1]].sum() - 1.0) < 1e-12
    x = (wl.pos[:, None, 0] + wl.kern_dxdy[None, :, 0] - wl.origin[0]) / wl.dx
    assert x.min() > 0 and x.max() < wl.n_grid - 1
