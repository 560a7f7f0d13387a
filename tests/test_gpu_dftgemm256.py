"""The tensor-core DFT-GEMM form at N_p = 256 (FP16 hi + lo operands, FP32 accumulation) against
the FP64 oracle, element by element, through the C ABI (GPU only).

Tolerance: the FP32 path's bound, 1e-4 relative L2 per image cube and every pixel within 1e-4 of
the cube's peak.  The split operands carry about 22 bits each, the gridded field is scaled by a
power of two per image (|E| < 256, so |X| < 2^15 stays inside the FP16 range when X is split),
and the products accumulate in FP32 over K = 128: the error measured is a few 1e-6.

Two CTAs image each sample (one per half of the image rows) and each grids the whole image, so
the cases include one sample per CTA pair, several (channel, pol) blocks per CTA range, ragged
grids, complex weights, gains, the three voltage formats, continuation, a deep slice in which
every CTA runs tens of samples through the pipeline, and the antenna limit of the form's shared
memory.
"""
import numpy as np
import pytest

from oracle import moff
from paper_1510_08318_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

RTOL_L2 = 1e-4
PIX = 1e-4


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


def check_close(got, want, what):
    got = np.asarray(got, dtype=np.float64)
    rel = np.linalg.norm(got - want) / np.linalg.norm(want)
    worst = np.abs(got - want).max() / np.abs(want).max()
    assert rel < RTOL_L2, "%s: relative L2 %.3e" % (what, rel)
    assert worst < PIX, "%s: worst pixel %.3e of peak" % (what, worst)
    return rel


def gains_dev(g):
    return None if g is None else torch.from_numpy(np.ascontiguousarray(g.astype(np.complex64))).cuda()


def _small_workload(n_grid, n_ant, n_time, n_chan, n_pol, seed, vdtype, dx=1.0):
    rng = np.random.default_rng(seed)
    pos = rng.uniform(1.5 * dx, (n_grid - 2.5) * dx, (n_ant, 2))
    kerns = [synth.kernel_square(rng.uniform(0.5, 2.5) * dx, dx / 3) for _ in range(n_ant)]
    ptr, dxdy, w = synth.pack_kernels(kerns)
    w = w * np.exp(1j * rng.uniform(0, 2 * np.pi, w.shape))     # complex weights
    wl = synth.Workload("small", pos, ptr, dxdy, w, dx, np.zeros(2), n_grid, 256,
                        np.full(n_chan, 1e8), n_pol, n_time, vdtype)
    v = (rng.standard_normal((n_time, n_chan, n_pol, n_ant))
         + 1j * rng.standard_normal((n_time, n_chan, n_pol, n_ant)))
    return synth._finish(wl, v, vdtype)


def _run(epic, wl, gains=None, autocorr=False):
    plan = epic.Plan.from_workload(wl).set_transform("dftgemm")
    out = plan.image(torch.from_numpy(np.ascontiguousarray(wl.volt_raw)).cuda(), gains_dev(gains),
                     want_autocorr=autocorr)
    plan.sync()
    return plan, {k: (v.cpu().numpy() if v is not None else None) for k, v in out.items()}


@pytest.mark.parametrize("n_grid, n_ant, n_time, n_chan, n_pol, vdtype", [
    (128, 40, 1, 1, 1, "c64"),      # one sample: most CTA pairs idle, complex weights
    (100, 60, 5, 3, 2, "f16"),      # ragged grid, several (channel, pol) blocks per range
    (128, 300, 9, 2, 1, "ci4"),     # 4+4-bit, more antennas than decoding threads' first pass
    (77, 700, 3, 1, 2, "c64"),      # 700 antennas (beyond the prefetched two per thread)
])
def test_small_cases(epic, n_grid, n_ant, n_time, n_chan, n_pol, vdtype):
    wl = _small_workload(n_grid, n_ant, n_time, n_chan, n_pol, 31 + n_ant, vdtype)
    rng = np.random.default_rng(n_ant)
    g = synth.random_gains(rng, (n_chan, n_pol, n_ant))
    _, out = _run(epic, wl, g)
    want = moff.moff_image(oracle_map(wl), wl.volt, g.astype(np.complex128), wl.n_grid, wl.n_pad)
    check_close(out["image"], want, "image")


def test_hera_slice(epic):
    """The dense HERA-331-like layout (14 m disks, FP16 voltages): two channels x 64 samples, with
    the auto-correlation term and the antenna power (added by one CTA of each pair)."""
    wl = synth.workload_hera(n_chan=2, n_time=64)
    M = oracle_map(wl)
    plan, out = _run(epic, wl, autocorr=True)
    want = moff.moff_image(M, wl.volt, None, wl.n_grid, wl.n_pad)
    check_close(out["image"], want, "image")
    check_close(out["autocorr"], moff.autocorr_term(M, wl.volt, None, wl.n_grid, wl.n_pad), "autocorr")
    np.testing.assert_allclose(out["power"], (np.abs(wl.volt) ** 2).sum(0), rtol=1e-5)


def test_calibration_layout_gains(epic):
    """1024 antennas in a 300 m disk (Gaussian apertures), complex64, random gains."""
    wl = synth.workload_calib(n_chan=1, n_time=12)
    rng = np.random.default_rng(19)
    g = synth.random_gains(rng, (1, 1, wl.n_ant))
    _, out = _run(epic, wl, g)
    want = moff.moff_image(oracle_map(wl), wl.volt, g.astype(np.complex128), wl.n_grid, wl.n_pad)
    check_close(out["image"], want, "image")


def test_continuation(epic):
    """Two calls with t_prev equal one call over all samples."""
    wl = synth.workload_hera(n_chan=1, n_time=24)
    plan = epic.Plan.from_workload(wl).set_transform("dftgemm")
    v = torch.from_numpy(np.ascontiguousarray(wl.volt_raw)).cuda()
    a = plan.image(v[:10])
    b = plan.image(v[10:], accum=a["accum"], t_prev=10)
    plan.sync()
    want = moff.moff_image(oracle_map(wl), wl.volt, None, wl.n_grid, wl.n_pad)
    check_close(b["image"].cpu().numpy(), want, "continued image")


def test_deep_pipeline_matches_fft_form(epic):
    """Eight HERA channels x 256 samples (2,048 images: every CTA runs about 27 through the
    pipeline): the whole cube against the FP32 FFT form within the bound, and two channels
    against the oracle."""
    wl = synth.workload_hera(n_chan=8, n_time=256)
    v = torch.from_numpy(np.ascontiguousarray(wl.volt_raw)).cuda()
    plan = epic.Plan.from_workload(wl)
    fft = plan.image(v)["image"]
    dg = plan.set_transform("dftgemm").image(v)["image"]
    plan.sync()
    fft, dg = fft.cpu().numpy(), dg.cpu().numpy()
    check_close(dg, fft.astype(np.float64), "tensor-core vs FFT form")
    M = oracle_map(wl)
    sub = wl.volt[:, [0, 7]]
    want = moff.moff_image(M, sub, None, wl.n_grid, wl.n_pad)
    check_close(dg[[0, 7]], want, "tensor-core vs oracle")


def test_antenna_limit_and_rejections(epic):
    """The form keeps two voltage buffers, gains and power per antenna in shared memory beside
    its operand buffers: 1,800 antennas fit, 1,900 do not; cross-polarisation at 256 is refused."""
    ok = _small_workload(128, 1800, 2, 1, 1, 5, "c64")
    _, out = _run(epic, ok)
    want = moff.moff_image(oracle_map(ok), ok.volt, None, ok.n_grid, ok.n_pad)
    check_close(out["image"], want, "1800 antennas")
    big = _small_workload(128, 1900, 1, 1, 1, 6, "c64")
    plan = epic.Plan.from_workload(big)
    with pytest.raises(epic.EpicError) as e:
        plan.set_transform("dftgemm")
    assert e.value.status == epic.EPIC_EUNSUPPORTED
    two = _small_workload(64, 10, 2, 1, 2, 7, "c64")
    plan = epic.Plan.from_workload(two).set_transform("dftgemm")
    with pytest.raises(epic.EpicError) as e:
        plan.image_xpol(torch.from_numpy(np.ascontiguousarray(two.volt_raw)).cuda())
    assert e.value.status == epic.EPIC_EUNSUPPORTED


def test_timeout_reported_then_cleared(epic):
    wl = synth.workload_hera(n_chan=1, n_time=8)
    plan = epic.Plan.from_workload(wl).set_transform("dftgemm")
    v = torch.from_numpy(np.ascontiguousarray(wl.volt_raw)).cuda()
    plan.set_wait_limit(0)
    plan.image(v)
    with pytest.raises(epic.EpicError) as e:
        plan.sync()
    assert e.value.status == epic.EPIC_ETIMEOUT
    plan.set_wait_limit(1000)
    out = plan.image(v)
    plan.sync()
    want = moff.moff_image(oracle_map(wl), wl.volt, None, wl.n_grid, wl.n_pad)
    check_close(out["image"].cpu().numpy(), want, "image after a timeout")


@pytest.mark.parametrize("xform, bound", [("dftgemm", RTOL_L2), ("dftgemm_fp16grid", 3e-3)])
def test_grid_corner_cells(epic, xform, bound):
    """Antennas whose footprints fall on the grid's first cells, (x, y) = (0, 0), (0, 1) and (1, 0):
    the word of E^T that holds the cell pair (0, 0), (0, 1) is written by its own slot only (the
    slot table's positions that no slot took are marked and skipped, not stored as zeros)."""
    rng = np.random.default_rng(43)
    n_grid, n_ant, n_time = 128, 64, 6
    corner = np.array([[0.1, 0.1], [0.1, 1.1], [1.1, 0.1]])
    pos = np.vstack([corner, rng.uniform(2.5, n_grid - 3.5, (n_ant - 3, 2))])
    kerns = ([synth.kernel_square(0.3, 0.1) for _ in range(3)]
             + [synth.kernel_square(rng.uniform(0.5, 2.5), 1 / 3) for _ in range(n_ant - 3)])
    ptr, dxdy, w = synth.pack_kernels(kerns)
    wl = synth.Workload("corner", pos, ptr, dxdy, w, 1.0, np.zeros(2), n_grid, 256,
                        np.full(1, 1e8), 1, n_time, "c64")
    v = rng.standard_normal((n_time, 1, 1, n_ant)) + 1j * rng.standard_normal((n_time, 1, 1, n_ant))
    v[:, :, :, :3] *= 20.0      # the corner antennas dominate their cells
    wl = synth._finish(wl, v, "c64")
    M = oracle_map(wl)
    assert all(M[c].nnz > 0 for c in (0, 1, n_grid))   # cells (0, 0), (1, 0), (0, 1) are occupied
    plan = epic.Plan.from_workload(wl).set_transform(xform)
    out = plan.image(torch.from_numpy(np.ascontiguousarray(wl.volt_raw)).cuda())
    plan.sync()
    got = out["image"].cpu().numpy().astype(np.float64)
    want = moff.moff_image(M, wl.volt, None, wl.n_grid, wl.n_pad)
    rel = np.linalg.norm(got - want) / np.linalg.norm(want)
    worst = np.abs(got - want).max() / np.abs(want).max()
    assert rel < bound and worst < bound, (rel, worst)
