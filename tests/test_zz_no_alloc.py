"""epic_image_noalloc through the C ABI (GPU only): the allocation-free imaging call for N_p = 512
plans, for callers that cannot allocate device memory while they image.  It stages each sample's
row-transformed grid in a device array built into the library instead of a buffer it allocates,
so it must give the images of the existing entry point, epic_image: checked on two calls in a
row (the second finds the first call's rows still in the shared array), with the FP32 path's
tolerance (1e-4 relative L2 per cube and per pixel of the peak).  Sizes beyond the array's
capacity are refused before anything is launched.

This file's name makes pytest collect it last."""
import numpy as np
import pytest

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


def _workload(seed, n_time, n_chan):
    rng = np.random.default_rng(seed)
    n_grid, n_ant = 200, 150
    pos = rng.uniform(1.5, n_grid - 2.5, (n_ant, 2))
    kerns = [synth.kernel_square(rng.uniform(0.5, 2.5), 1 / 3) for _ in range(n_ant)]
    ptr, dxdy, w = synth.pack_kernels(kerns)
    wl = synth.Workload("np512", pos, ptr, dxdy, w, 1.0, np.zeros(2), n_grid, 512, np.full(n_chan, 1e8), 1, n_time,
                        "f16")
    v = rng.standard_normal((n_time, n_chan, 1, n_ant)) + 1j * rng.standard_normal((n_time, n_chan, 1, n_ant))
    return synth._finish(wl, v, "f16")


def _close(got, want):
    got, want = np.asarray(got, np.float64), np.asarray(want, np.float64)
    assert np.linalg.norm(got - want) / np.linalg.norm(want) < TOL
    assert np.abs(got - want).max() < TOL * np.abs(want).max()


def test_noalloc_matches_epic_image_on_two_calls(epic):
    wl = _workload(61, 40, 3)
    plan = epic.Plan.from_workload(wl)
    C, NP, A = wl.n_chan, wl.n_pad, wl.n_ant
    st = torch.cuda.current_stream().cuda_stream
    v_all = torch.from_numpy(np.ascontiguousarray(wl.volt_raw)).cuda()
    gains = torch.from_numpy(synth.random_gains(np.random.default_rng(62), (C, 1, A)).astype(np.complex64)).cuda()
    for call, (v, g, chunk) in enumerate([(v_all[:25], None, 16), (v_all[25:], gains, 7)]):
        T = int(v.shape[0])
        ref = plan.image(v, g, want_autocorr=True)
        accum = torch.empty((C, 1, NP, NP), dtype=torch.float64, device="cuda")
        power = torch.empty((C, 1, A), dtype=torch.float64, device="cuda")
        image = torch.empty((C, 1, NP, NP), dtype=torch.float32, device="cuda")
        autoc = torch.empty((C, 1, NP, NP), dtype=torch.float32, device="cuda")
        epic.epic_image_noalloc(plan._h, v.data_ptr(), T, None if g is None else g.data_ptr(), accum.data_ptr(),
                                power.data_ptr(), 0, image.data_ptr(), autoc.data_ptr(), chunk, st)
        torch.cuda.synchronize()
        _close(image.cpu().numpy(), ref["image"].cpu().numpy())
        _close(autoc.cpu().numpy(), ref["autocorr"].cpu().numpy())
        _close(power.cpu().numpy(), ref["power"].cpu().numpy())   # FP32 partial sums, grouped differently


def test_noalloc_refuses_sizes_beyond_its_array(epic):
    wl = _workload(63, 4, 1)
    plan = epic.Plan.from_workload(wl)
    v = torch.from_numpy(np.ascontiguousarray(wl.volt_raw)).cuda()
    accum = torch.empty((1, 1, 512, 512), dtype=torch.float64, device="cuda")
    st = torch.cuda.current_stream().cuda_stream
    for chunk in (0, 65):
        with pytest.raises(epic.EpicError) as e:
            epic.epic_image_noalloc(plan._h, v.data_ptr(), 4, None, accum.data_ptr(), None, 0, None, None, chunk, st)
        assert e.value.status == epic.EPIC_EINVAL and "static scratch" in str(e.value)
    small = epic.Plan.from_workload(synth.workload_tiny(n_time=2))
    with pytest.raises(epic.EpicError) as e:
        epic.epic_image_noalloc(small._h, v.data_ptr(), 2, None, accum.data_ptr(), None, 0, None, None, 8, st)
    assert e.value.status == epic.EPIC_EUNSUPPORTED
