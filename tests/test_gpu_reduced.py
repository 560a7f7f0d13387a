"""The reduced-precision tensor-core form (EPIC_XFORM_DFTGEMM_FP16, N_p = 128) against the FP64
oracle through the C ABI (GPU only).

The form rounds four operands to FP16 on the way to each transform value F: the gridding
weights, the calibrated voltages (exact for 4+4-bit voltages with unit gains), the gridded field
E and the stage-1 result X, and the DFT matrix W enters both stages in FP16; every product is
exact in FP32 and every sum is FP32.  Each rounding has a relative error of at most u = 2^-11
(FP16, round to nearest) and, summed over many terms, about u / sqrt(3) in the mean square, so
F carries a relative error of about sqrt(5) u / sqrt(3) ~ 6e-4 and |F|^2 twice that, ~1.3e-3
in the worst case of every pixel's errors aligned.  The stated bound is 3e-3 relative L2 per
image cube and every pixel within 3e-3 of the cube's peak; the measured error is printed.
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


def check(got, want, what):
    got = np.asarray(got, dtype=np.float64)
    rel = np.linalg.norm(got - want) / np.linalg.norm(want)
    worst = np.abs(got - want).max() / np.abs(want).max()
    print("%s: relative L2 %.2e, worst pixel %.2e of peak" % (what, rel, worst))
    assert rel < BOUND, "%s: relative L2 %.3e" % (what, rel)
    assert worst < BOUND, "%s: worst pixel %.3e of peak" % (what, worst)
    return rel


def _image(epic, wl, gains=None, accum=None, t_prev=0, volt=None):
    plan = epic.Plan.from_workload(wl).set_transform("dftgemm_fp16")
    v = torch.from_numpy(np.ascontiguousarray(wl.volt_raw)).cuda() if volt is None else volt
    g = None if gains is None else torch.from_numpy(np.ascontiguousarray(gains.astype(np.complex64))).cuda()
    out = plan.image(v, g, want_autocorr=True)
    plan.sync()
    return {k: (x.cpu().numpy() if x is not None else None) for k, x in out.items()}


def test_lwa_slice_gains(epic):
    """LWA-like layout, 4+4-bit voltages, two channels, two pols, 64 samples, random gains."""
    wl = synth.workload_lwa(n_chan=2, n_time=64, chan_index=[0, 127])
    g = synth.random_gains(np.random.default_rng(21), (wl.n_chan, wl.n_pol, wl.n_ant))
    out = _image(epic, wl, g)
    M = oracle_map(wl)
    gg = g.astype(np.complex128)
    check(out["image"], moff.moff_image(M, wl.volt, gg, wl.n_grid, wl.n_pad), "image")
    # the auto-correlation term and the power come from the FP32 voltages: the FP32 bound holds
    ac = moff.autocorr_term(M, wl.volt, gg, wl.n_grid, wl.n_pad)
    assert np.linalg.norm(out["autocorr"] - ac) / np.linalg.norm(ac) < 1e-4


def test_deep_slice_unit_gains(epic):
    """1024 samples of one channel (every CTA runs about 13 samples through the pipeline)."""
    wl = synth.workload_lwa(n_chan=1, n_time=1024, chan_index=[100])
    out = _image(epic, wl)
    check(out["image"], moff.moff_image(oracle_map(wl), wl.volt, None, wl.n_grid, wl.n_pad), "image")


@pytest.mark.parametrize("n_grid, n_ant, n_time, vdtype", [(64, 40, 9, "c64"), (45, 300, 7, "f16")])
def test_small_complex_weights(epic, n_grid, n_ant, n_time, vdtype):
    rng = np.random.default_rng(n_ant)
    pos = rng.uniform(1.5, n_grid - 2.5, (n_ant, 2))
    kerns = [synth.kernel_square(rng.uniform(0.5, 2.5), 1 / 3) for _ in range(n_ant)]
    ptr, dxdy, w = synth.pack_kernels(kerns)
    w = w * np.exp(1j * rng.uniform(0, 2 * np.pi, w.shape))
    wl = synth.Workload("small", pos, ptr, dxdy, w, 1.0, np.zeros(2), n_grid, 128, np.full(2, 1e8), 1, n_time,
                        vdtype)
    v = rng.standard_normal((n_time, 2, 1, n_ant)) + 1j * rng.standard_normal((n_time, 2, 1, n_ant))
    wl = synth._finish(wl, v, vdtype)
    out = _image(epic, wl)
    check(out["image"], moff.moff_image(oracle_map(wl), wl.volt, None, wl.n_grid, wl.n_pad), "image")


def test_rejections(epic):
    """The reduced-precision form exists for N_p = 128 and single-pol products only."""
    wl = synth.workload_hera(n_chan=1, n_time=2)
    plan = epic.Plan.from_workload(wl)
    with pytest.raises(epic.EpicError) as e:
        plan.set_transform("dftgemm_fp16")
    assert e.value.status == epic.EPIC_EUNSUPPORTED
    wl = synth.workload_lwa(n_chan=1, n_time=4, chan_index=[3])
    plan = epic.Plan.from_workload(wl).set_transform("dftgemm_fp16")
    with pytest.raises(epic.EpicError) as e:
        plan.image_xpol(torch.from_numpy(np.ascontiguousarray(wl.volt_raw)).cuda())
    assert e.value.status == epic.EPIC_EUNSUPPORTED
