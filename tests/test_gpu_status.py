"""Device-side failure reporting and host-side argument checks on a real plan (GPU only).

A bounded wait on the tensor cores that runs out is made to happen without any fault: the
plan's wait limit is set to 0 tries, so every wait of the pipeline reports a timeout at its first
check while the products already issued still complete (the kernel drains them with its full
limit before it releases its tensor memory).  epic_sync must then return EPIC_ETIMEOUT, and the
next call with the default limit must return EPIC_OK and an image (or visibilities) that match
the FP64 oracle.  Misaligned device arrays are refused on the host before any launch.
"""
import numpy as np
import pytest

from oracle import fx, moff
from paper_1510_08318_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def epic():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1510_08318_gb300 import build, epic as ep
    build.build()
    ep.load()
    return ep


def _lwa_slice():
    return synth.workload_lwa(n_chan=1, n_time=40, chan_index=[64])


def _rel(got, want):
    return float(np.linalg.norm(got - want) / np.linalg.norm(want))


def test_imaging_timeout_is_reported_then_cleared(epic):
    wl = _lwa_slice()
    plan = epic.Plan.from_workload(wl).set_transform("dftgemm")
    volt = torch.from_numpy(np.ascontiguousarray(wl.volt_raw)).cuda()
    plan.set_wait_limit(0)
    plan.image(volt)                               # enqueued: the launch itself succeeds
    with pytest.raises(epic.EpicError) as e:
        plan.sync()
    assert e.value.status == epic.EPIC_ETIMEOUT
    assert "imaging" in str(e.value)
    plan.sync()                                    # the word was cleared
    plan.set_wait_limit(1000)
    out = plan.image(volt)
    plan.sync()
    M = moff.map_antennas(wl.pos, wl.kern_ptr, wl.kern_dxdy, wl.kern_w, wl.dx, wl.origin, wl.n_grid)
    want = moff.moff_image(M, wl.volt, None, wl.n_grid, wl.n_pad)
    assert _rel(out["image"].cpu().numpy(), want) < 1e-4


def test_cross_polarisation_timeout_is_reported(epic):
    wl = _lwa_slice()
    plan = epic.Plan.from_workload(wl).set_transform("dftgemm")
    volt = torch.from_numpy(np.ascontiguousarray(wl.volt_raw)).cuda()
    plan.set_wait_limit(0)
    plan.image_xpol(volt)
    with pytest.raises(epic.EpicError) as e:
        plan.sync()
    assert e.value.status == epic.EPIC_ETIMEOUT
    plan.set_wait_limit(1000)
    plan.image_xpol(volt)
    plan.sync()


def test_correlator_timeout_is_reported_then_cleared(epic):
    wl = synth.workload_lwa(n_chan=1, n_time=96, chan_index=[64])
    plan = epic.Plan.from_workload(wl)
    volt = torch.from_numpy(np.ascontiguousarray(wl.volt_raw)).cuda()
    plan.set_wait_limit(0)
    plan.correlate(volt)
    with pytest.raises(epic.EpicError) as e:
        plan.sync()
    assert e.value.status == epic.EPIC_ETIMEOUT
    assert "correlator" in str(e.value)
    plan.set_wait_limit(1000)
    vis = plan.correlate(volt)
    plan.sync()
    want = fx.visibilities(wl.volt[:, 0, 1, :], np.ones(wl.n_ant, dtype=np.complex128))
    got = vis.cpu().numpy()[0, 1]
    assert _rel(got, want) < 1e-6


def test_fft_form_reports_ok(epic):
    """The FFT form has no waits on the tensor cores: a wait limit of 0 changes nothing."""
    wl = synth.workload_tiny(n_time=8)
    plan = epic.Plan.from_workload(wl).set_wait_limit(0)
    out = plan.image(torch.from_numpy(wl.volt_raw).cuda())
    plan.sync()
    M = moff.map_antennas(wl.pos, wl.kern_ptr, wl.kern_dxdy, wl.kern_w, wl.dx, wl.origin, wl.n_grid)
    assert _rel(out["image"].cpu().numpy(), moff.moff_image(M, wl.volt, None, wl.n_grid, wl.n_pad)) < 1e-4


def test_wait_limit_range(epic):
    plan = epic.Plan.from_workload(synth.workload_tiny(n_time=4))
    for bad in (-1, 1000001):
        with pytest.raises(epic.EpicError) as e:
            plan.set_wait_limit(bad)
        assert e.value.status == epic.EPIC_EINVAL


def test_misaligned_arrays_refused_before_launch(epic):
    """Offset pointers into valid allocations: every call refuses them on the host (nothing is
    launched, so the offsets are never dereferenced)."""
    wl = synth.workload_tiny(n_time=4)                 # complex64 voltages: 8-byte samples
    plan = epic.Plan.from_workload(wl)
    C, P, A, NP = wl.n_chan, wl.n_pol, wl.n_ant, wl.n_pad
    volt = torch.from_numpy(wl.volt_raw).cuda()
    gains = torch.ones((C, P, A), dtype=torch.complex64, device="cuda")
    accum = torch.empty((C, P, NP, NP), dtype=torch.float64, device="cuda")
    power = torch.empty((C, P, A), dtype=torch.float64, device="cuda")
    img = torch.empty((C, P, NP, NP), dtype=torch.float32, device="cuda")
    st = torch.cuda.current_stream().cuda_stream
    v, g, ac, pw, im = volt.data_ptr(), gains.data_ptr(), accum.data_ptr(), power.data_ptr(), img.data_ptr()
    cases = [
        ("volt", (v + 4, 4, g, ac, pw, 0, im, None)),
        ("gains", (v, 4, g + 4, ac, pw, 0, im, None)),
        ("accum", (v, 4, g, ac + 4, pw, 0, im, None)),
        ("power", (v, 4, g, ac, pw + 4, 0, im, None)),
        ("image", (v, 4, g, ac, pw, 0, im + 2, None)),
    ]
    for name, args in cases:
        with pytest.raises(epic.EpicError) as e:
            epic.epic_image(plan._h, *args, st)
        assert e.value.status == epic.EPIC_EINVAL and name in str(e.value), name
    grid = torch.empty((4, C, P, wl.n_grid, wl.n_grid), dtype=torch.complex64, device="cuda")
    with pytest.raises(epic.EpicError) as e:
        epic.epic_grid(plan._h, v, 4, None, grid.data_ptr() + 4, st)
    assert e.value.status == epic.EPIC_EINVAL
    with pytest.raises(epic.EpicError) as e:
        epic.epic_image_backward(plan._h, v, 4, None, im + 2, g, st)
    assert e.value.status == epic.EPIC_EINVAL
    torch.cuda.synchronize()
    # the plan still works after the refusals
    out = plan.image(volt)
    plan.sync()
    assert torch.isfinite(out["image"]).all()
