"""Cross-polarisation images (epic_image_xpol) vs the FP64 oracle's four products (GPU only).

XX and YY carry the FP32 bound of the single-pol path (1e-4 relative L2, every pixel within
1e-4 of the peak).  XY is formed from time sums of |F_v|^2 by the polarisation identity, so
its float32 error scales with the total power, not with |XY| itself: the bound is 1e-4 of
sqrt(|XX| |YY|) (relative L2 and per pixel); for strongly polarised fields (|XY| comparable
to XX) it is also checked against |XY| directly.
"""
import numpy as np
import pytest

from oracle import moff
from paper_1510_08318_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-4


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


def check(out, want, what, polarised=False):
    img, cross = out["image"].cpu().numpy(), out["cross"].cpu().numpy()
    for c in range(want.shape[0]):
        xx, yy, xy = want[c, 0, 0].real, want[c, 1, 1].real, want[c, 0, 1]
        for got, ref, name in ((img[c, 0], xx, "XX"), (img[c, 1], yy, "YY")):
            assert np.linalg.norm(got - ref) / np.linalg.norm(ref) < TOL, (what, c, name)
            assert np.abs(got - ref).max() < TOL * ref.max(), (what, c, name)
        scale = np.sqrt(np.linalg.norm(xx) * np.linalg.norm(yy))
        err = cross[c] - xy
        assert np.linalg.norm(err) < TOL * scale, (what, c, "XY", np.linalg.norm(err) / scale)
        assert np.abs(err).max() < TOL * np.sqrt(xx.max() * yy.max()), (what, c, "XY pixel")
        if polarised:
            assert np.linalg.norm(err) / np.linalg.norm(xy) < TOL, (what, c, "XY vs |XY|")


def _dual(n_pad, n_grid, n_ant, n_time, n_chan, vdtype, seed, alpha=0.6 - 0.5j):
    """Random complex-weight apertures; pol Y = alpha X + noise (a strongly polarised field)."""
    rng = np.random.default_rng(seed)
    pos = rng.uniform(1.5, n_grid - 2.5, (n_ant, 2))
    kerns = [synth.kernel_square(rng.uniform(0.5, 2.5), 1 / 3) for _ in range(n_ant)]
    ptr, dxdy, w = synth.pack_kernels(kerns)
    w = w * np.exp(1j * rng.uniform(0, 2 * np.pi, w.shape))
    wl = synth.Workload("dual", pos, ptr, dxdy, w, 1.0, np.zeros(2), n_grid, n_pad,
                        np.full(n_chan, 1e8), 2, n_time, vdtype)
    vx = rng.standard_normal((n_time, n_chan, n_ant)) + 1j * rng.standard_normal((n_time, n_chan, n_ant))
    nz = rng.standard_normal((n_time, n_chan, n_ant)) + 1j * rng.standard_normal((n_time, n_chan, n_ant))
    v = np.stack([vx, alpha * vx + 0.3 * nz], axis=2)
    return synth._finish(wl, v, vdtype)


def run(epic, wl, gains=None, t_split=None, xform="fft"):
    plan = epic.Plan.from_workload(wl).set_transform(xform)
    g = None if gains is None else torch.from_numpy(np.ascontiguousarray(gains.astype(np.complex64))).cuda()
    v = torch.from_numpy(np.ascontiguousarray(wl.volt_raw)).cuda()
    if t_split is None:
        out = plan.image_xpol(v, g)
    else:
        first = plan.image_xpol(v[:t_split].contiguous(), g)
        out = plan.image_xpol(v[t_split:].contiguous(), g, accum4=first["accum4"], t_prev=t_split)
    torch.cuda.synchronize()
    return out


def test_lwa_slice_ci4_gains(epic):
    """LWA-like layout, 4+4-bit voltages, two channels, 40 samples, random gains per pol."""
    wl = synth.workload_lwa(n_chan=2, n_time=40, chan_index=[0, 127])
    g = synth.random_gains(np.random.default_rng(5), (wl.n_chan, 2, wl.n_ant))
    out = run(epic, wl, g)
    check(out, moff.moff_cross_image(oracle_map(wl), wl.volt, g.astype(np.complex128), wl.n_grid, wl.n_pad), "lwa")


@pytest.mark.parametrize("n_pad, n_grid, n_ant, n_time, n_chan, vdtype", [
    (32, 16, 9, 7, 3, "c64"),
    (64, 20, 300, 11, 2, "ci4"),
    (128, 64, 700, 5, 1, "f16"),
    (256, 100, 64, 3, 2, "c64"),
    (512, 40, 30, 3, 1, "f16"),
])
def test_polarised_all_sizes(epic, n_pad, n_grid, n_ant, n_time, n_chan, vdtype):
    wl = _dual(n_pad, n_grid, n_ant, n_time, n_chan, vdtype, seed=n_pad + n_ant)
    g = synth.random_gains(np.random.default_rng(n_ant), (n_chan, 2, n_ant))
    out = run(epic, wl, g)
    want = moff.moff_cross_image(oracle_map(wl), wl.volt, g.astype(np.complex128), wl.n_grid, wl.n_pad)
    check(out, want, "N_p %d" % n_pad, polarised=vdtype != "ci4")


def test_continuation_and_single_pol_agreement(epic):
    """Two calls (t_prev) equal one; XX and YY equal epic_image's images of the same data."""
    wl = _dual(64, 30, 40, 12, 2, "c64", seed=3)
    one = run(epic, wl)
    two = run(epic, wl, t_split=5)
    for k in ("image", "cross"):
        a, b = one[k].cpu().numpy(), two[k].cpu().numpy()
        assert np.linalg.norm(a - b) / np.linalg.norm(a) < 1e-6
    plan = epic.Plan.from_workload(wl)
    img = plan.image(torch.from_numpy(np.ascontiguousarray(wl.volt_raw)).cuda())["image"].cpu().numpy()
    a = one["image"].cpu().numpy()
    assert np.linalg.norm(a - img) / np.linalg.norm(img) < 1e-6


# ---------------------------------------------------------------------------------------------
# the tensor-core DFT form (N_p = 128) runs the same virtual pols: same oracle, same bounds
# ---------------------------------------------------------------------------------------------
def test_dftgemm_lwa_slice_ci4_gains(epic):
    """400 samples: every CTA images about 21 consecutive virtual-pol samples."""
    wl = synth.workload_lwa(n_chan=2, n_time=400, chan_index=[0, 127])
    g = synth.random_gains(np.random.default_rng(6), (wl.n_chan, 2, wl.n_ant))
    out = run(epic, wl, g, xform="dftgemm")
    check(out, moff.moff_cross_image(oracle_map(wl), wl.volt, g.astype(np.complex128), wl.n_grid, wl.n_pad),
          "lwa tensor-core")


@pytest.mark.parametrize("n_grid, n_ant, n_time, n_chan, vdtype", [
    (64, 700, 5, 1, "f16"),      # A beyond the prefetched antennas' first slot
    (40, 60, 6, 2, "c64"),       # ragged grid, two channels
    (64, 1500, 3, 1, "c64"),     # A beyond the prefetched antennas (tail loop)
])
def test_dftgemm_polarised(epic, n_grid, n_ant, n_time, n_chan, vdtype):
    wl = _dual(128, n_grid, n_ant, n_time, n_chan, vdtype, seed=n_ant + 11)
    g = synth.random_gains(np.random.default_rng(n_ant + 1), (n_chan, 2, n_ant))
    out = run(epic, wl, g, xform="dftgemm")
    want = moff.moff_cross_image(oracle_map(wl), wl.volt, g.astype(np.complex128), wl.n_grid, wl.n_pad)
    check(out, want, "tensor-core %d antennas" % n_ant, polarised=True)


def test_dftgemm_continuation_matches_fft(epic):
    """Two tensor-core calls (t_prev) equal one, and agree with the FFT form's four products."""
    wl = _dual(128, 50, 80, 10, 2, "c64", seed=9)
    one = run(epic, wl, xform="dftgemm")
    two = run(epic, wl, t_split=4, xform="dftgemm")
    ref = run(epic, wl)
    for k in ("image", "cross"):
        a, b, f = one[k].cpu().numpy(), two[k].cpu().numpy(), ref[k].cpu().numpy()
        assert np.linalg.norm(a - b) / np.linalg.norm(a) < 1e-6
        assert np.linalg.norm(a - f) / np.linalg.norm(f) < 1e-4


def test_dftgemm_xpol_antenna_limit(epic):
    """The cross-polarisation form of the tensor-core kernel holds one more per-antenna array:
    2000 antennas fit the single-pol form but not this one, which is refused."""
    wl = _dual(128, 64, 2000, 1, 1, "ci4", seed=4)
    plan = epic.Plan.from_workload(wl).set_transform("dftgemm")
    with pytest.raises(epic.EpicError) as e:
        plan.image_xpol(torch.from_numpy(np.ascontiguousarray(wl.volt_raw)).cuda())
    assert e.value.status == epic.EPIC_EUNSUPPORTED


def test_rejects_single_pol_plan(epic):
    wl = synth.workload_tiny(n_time=2)
    plan = epic.Plan.from_workload(wl)
    with pytest.raises(epic.EpicError):
        plan.image_xpol(torch.from_numpy(np.ascontiguousarray(wl.volt_raw)).cuda())
