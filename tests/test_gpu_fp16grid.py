"""The FP16-gridding tensor-core form at N_p = 256 (EPIC_XFORM_DFTGEMM_FP16_GRID) against the
FP64 oracle through the C ABI (GPU only).

The form rounds two operands to FP16 before the gridding products: each aperture weight and each
calibrated voltage (4+4-bit and FP16 voltages with unit gains are exact).  Every product of two
FP16 numbers is exact in FP32 and the cells' sums are FP32; the transform then keeps FP16 hi + lo
operands (a few 1e-6 on its own).  Each rounding has a relative error of at most u = 2^-11 and
about u / sqrt(3) in the mean square, so the gridded field, and with it F, carries a relative
error of about sqrt(2) u / sqrt(3) ~ 4e-4 and |F|^2 twice that, ~1e-3 if every pixel's errors were
aligned.  The stated bound is that of the reduced-precision forms, 3e-3 relative L2 per image
cube and every pixel within 3e-3 of the cube's peak; the measured error is printed.

Real weights take the packed gather entries (FP16 weight and antenna in one word), complex
weights the FP32 tables rounded as they are read: both are covered, with gains, the three voltage
formats, ragged grids and a deep slice.
"""
import numpy as np
import pytest

from oracle import moff
from paper_1510_08318_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

BOUND = 3e-3


@pytest.fixture(scope="module")
def epic():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1510_08318_gb300 import build, epic as ep
    build.build()
    ep.load()
    return ep


def oracle_map(wl):
    return moff.map_antennas(wl.pos, wl.kern_ptr, wl.kern_dxdy, wl.kern_w, wl.dx, wl.origin, wl.n_grid)


def check(got, want, what, bound=BOUND):
    got = np.asarray(got, dtype=np.float64)
    rel = np.linalg.norm(got - want) / np.linalg.norm(want)
    worst = np.abs(got - want).max() / np.abs(want).max()
    print("%s: relative L2 %.2e, worst pixel %.2e of peak" % (what, rel, worst))
    assert rel < bound, "%s: relative L2 %.3e" % (what, rel)
    assert worst < bound, "%s: worst pixel %.3e of peak" % (what, worst)
    return rel


def gains_dev(g):
    return None if g is None else torch.from_numpy(np.ascontiguousarray(g.astype(np.complex64))).cuda()


def _image(epic, wl, gains=None, autocorr=False):
    plan = epic.Plan.from_workload(wl).set_transform("dftgemm_fp16grid")
    out = plan.image(torch.from_numpy(np.ascontiguousarray(wl.volt_raw)).cuda(), gains_dev(gains),
                     want_autocorr=autocorr)
    plan.sync()
    return {k: (x.cpu().numpy() if x is not None else None) for k, x in out.items()}


def _small_workload(n_grid, n_ant, n_time, n_chan, n_pol, seed, vdtype, complex_w, dx=1.0):
    rng = np.random.default_rng(seed)
    pos = rng.uniform(1.5 * dx, (n_grid - 2.5) * dx, (n_ant, 2))
    kerns = [synth.kernel_square(rng.uniform(0.5, 2.5) * dx, dx / 3) for _ in range(n_ant)]
    ptr, dxdy, w = synth.pack_kernels(kerns)
    if complex_w:
        w = w * np.exp(1j * rng.uniform(0, 2 * np.pi, w.shape))
    wl = synth.Workload("small", pos, ptr, dxdy, w, dx, np.zeros(2), n_grid, 256,
                        np.full(n_chan, 1e8), n_pol, n_time, vdtype)
    v = (rng.standard_normal((n_time, n_chan, n_pol, n_ant))
         + 1j * rng.standard_normal((n_time, n_chan, n_pol, n_ant)))
    return synth._finish(wl, v, vdtype)


def test_hera_slice(epic):
    """The dense HERA-331-like layout (real disk apertures: packed entries), FP16 voltages, two
    channels x 64 samples, with the auto-correlation term and the antenna power (which sums the
    calibrated voltages before their FP16 rounding)."""
    wl = synth.workload_hera(n_chan=2, n_time=64)
    M = oracle_map(wl)
    out = _image(epic, wl, autocorr=True)
    check(out["image"], moff.moff_image(M, wl.volt, None, wl.n_grid, wl.n_pad), "image")
    check(out["autocorr"], moff.autocorr_term(M, wl.volt, None, wl.n_grid, wl.n_pad), "autocorr", 1e-4)
    np.testing.assert_allclose(out["power"], (np.abs(wl.volt) ** 2).sum(0), rtol=1e-5)


def test_hera_slice_gains(epic):
    """Random complex gains: the calibrated voltages g V are no longer FP16 numbers and are
    rounded."""
    wl = synth.workload_hera(n_chan=1, n_time=48)
    rng = np.random.default_rng(3)
    g = synth.random_gains(rng, (1, 1, wl.n_ant))
    out = _image(epic, wl, g)
    check(out["image"], moff.moff_image(oracle_map(wl), wl.volt, g.astype(np.complex128), wl.n_grid, wl.n_pad),
          "image")


@pytest.mark.parametrize("n_grid, n_ant, n_time, n_chan, n_pol, vdtype, complex_w", [
    (128, 40, 1, 1, 1, "c64", True),      # one sample, complex weights (FP32 tables rounded on read)
    (100, 60, 5, 3, 2, "f16", True),      # ragged grid, several (channel, pol) blocks per range
    (128, 300, 9, 2, 1, "ci4", False),    # 4+4-bit voltages, real weights (packed entries)
    (77, 700, 3, 1, 2, "c64", False),     # 700 antennas, ragged grid, real weights
])
def test_small_cases(epic, n_grid, n_ant, n_time, n_chan, n_pol, vdtype, complex_w):
    wl = _small_workload(n_grid, n_ant, n_time, n_chan, n_pol, 57 + n_ant, vdtype, complex_w)
    rng = np.random.default_rng(n_ant + 1)
    g = synth.random_gains(rng, (n_chan, n_pol, n_ant))
    out = _image(epic, wl, g)
    want = moff.moff_image(oracle_map(wl), wl.volt, g.astype(np.complex128), wl.n_grid, wl.n_pad)
    check(out["image"], want, "image")


def test_calibration_layout(epic):
    """1024 antennas in a 300 m disk (Gaussian apertures, real weights), complex64, gains."""
    wl = synth.workload_calib(n_chan=1, n_time=12)
    rng = np.random.default_rng(29)
    g = synth.random_gains(rng, (1, 1, wl.n_ant))
    out = _image(epic, wl, g)
    check(out["image"], moff.moff_image(oracle_map(wl), wl.volt, g.astype(np.complex128), wl.n_grid, wl.n_pad),
          "image")


def test_deep_pipeline_against_fp32_forms(epic):
    """Eight HERA channels x 256 samples (every CTA runs about 27 samples through the pipeline):
    the cube against the FP32-gridding tensor-core form and the FFT form, and two channels
    against the oracle; continuation over two calls equals one call."""
    wl = synth.workload_hera(n_chan=8, n_time=256)
    v = torch.from_numpy(np.ascontiguousarray(wl.volt_raw)).cuda()
    plan = epic.Plan.from_workload(wl)
    fft = plan.image(v)["image"]
    dg = plan.set_transform("dftgemm")
    dg_img = dg.image(v)["image"]
    plan.set_transform("dftgemm_fp16grid")
    lp = plan.image(v)["image"]
    a = plan.image(v[:100])
    b = plan.image(v[100:], accum=a["accum"], t_prev=100)
    plan.sync()
    fft, dg_img, lp = fft.cpu().numpy(), dg_img.cpu().numpy(), lp.cpu().numpy()
    check(lp, fft.astype(np.float64), "FP16 gridding vs FFT form")
    check(lp, dg_img.astype(np.float64), "FP16 gridding vs FP32-gridding tensor-core form")
    np.testing.assert_allclose(b["image"].cpu().numpy(), lp, rtol=1e-5, atol=1e-6 * np.abs(lp).max())
    M = oracle_map(wl)
    want = moff.moff_image(M, wl.volt[:, [0, 7]], None, wl.n_grid, wl.n_pad)
    check(lp[[0, 7]], want, "FP16 gridding vs oracle")


def test_rejections(epic):
    """Only N_p = 256; no cross-polarisation variant."""
    wl128 = synth.workload_lwa(n_chan=1, n_time=2, chan_index=[0])
    with pytest.raises(epic.EpicError) as e:
        epic.Plan.from_workload(wl128).set_transform("dftgemm_fp16grid")
    assert e.value.status == epic.EPIC_EUNSUPPORTED
    two = _small_workload(64, 10, 2, 1, 2, 7, "c64", False)
    plan = epic.Plan.from_workload(two).set_transform("dftgemm_fp16grid")
    with pytest.raises(epic.EpicError) as e:
        plan.image_xpol(torch.from_numpy(np.ascontiguousarray(two.volt_raw)).cuda())
    assert e.value.status == epic.EPIC_EUNSUPPORTED
