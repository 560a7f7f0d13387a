"""The two-pass form for N_p = 512 (EPIC_XFORM_FFT_TWOPASS): a row pass that writes each sample's
row-transformed grid to scratch and a column pass that transforms, squares and accumulates, in
chunks of 4 x SMs samples.  Against the FP64 oracle (FP32 bound: 1e-4 relative L2 per cube and
per pixel of the peak) and against the cluster form (the same FP32 arithmetic in another order:
1e-6), across chunk boundaries, with several (channel, pol) blocks per chunk, antenna power for
the auto-correlation term, continuation, and the batch executor's choice of form (GPU only)."""
import numpy as np
import pytest

from oracle import moff
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


def rel(a, b):
    a, b = np.asarray(a, np.float64), np.asarray(b, np.float64)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _workload(n_grid, n_ant, n_time, n_chan, n_pol, seed, vdtype, n_pad=512):
    rng = np.random.default_rng(seed)
    pos = rng.uniform(1.5, n_grid - 2.5, (n_ant, 2))
    kerns = [synth.kernel_square(rng.uniform(0.5, 2.5), 1 / 3) for _ in range(n_ant)]
    ptr, dxdy, w = synth.pack_kernels(kerns)
    w = w * np.exp(1j * rng.uniform(0, 2 * np.pi, w.shape))
    wl = synth.Workload("np%d" % n_pad, pos, ptr, dxdy, w, 1.0, np.zeros(2), n_grid, n_pad, np.full(n_chan, 1e8),
                        n_pol, n_time, vdtype)
    v = rng.standard_normal((n_time, n_chan, n_pol, n_ant)) + 1j * rng.standard_normal((n_time, n_chan, n_pol, n_ant))
    return synth._finish(wl, v, vdtype)


def _dev(wl):
    return torch.from_numpy(np.ascontiguousarray(wl.volt_raw)).cuda()


def test_against_oracle(epic):
    wl = _workload(256, 120, 4, 1, 2, 41, "c64")
    g = synth.random_gains(np.random.default_rng(42), (1, 2, wl.n_ant))
    plan = epic.Plan.from_workload(wl).set_transform("fft_twopass")
    out = plan.image(_dev(wl), torch.from_numpy(g.astype(np.complex64)).cuda(), want_autocorr=True)
    plan.sync()
    M = moff.map_antennas(wl.pos, wl.kern_ptr, wl.kern_dxdy, wl.kern_w, wl.dx, wl.origin, wl.n_grid)
    want = moff.moff_image(M, wl.volt, g.astype(np.complex128), wl.n_grid, wl.n_pad)
    got = out["image"].cpu().numpy()
    assert rel(got, want) < 1e-4
    assert np.abs(got - want).max() < 1e-4 * np.abs(want).max()
    ac = moff.autocorr_term(M, wl.volt, g.astype(np.complex128), wl.n_grid, wl.n_pad)
    assert rel(out["autocorr"].cpu().numpy(), ac) < 1e-4


def test_chunks_match_cluster_form(epic):
    """650 samples (more than one chunk of 608 on a 152-SM GPU) over 5 (channel, pol) blocks,
    4+4-bit voltages, power and auto-correlation term: equal to the cluster form."""
    wl = _workload(200, 300, 130, 5, 1, 43, "ci4")
    v = _dev(wl)
    plan = epic.Plan.from_workload(wl)
    ref = plan.image(v, want_autocorr=True)
    ref = {k: x.cpu().numpy() for k, x in ref.items()}
    out = plan.set_transform("fft_twopass").image(v, want_autocorr=True)
    plan.sync()
    assert rel(out["image"].cpu().numpy(), ref["image"]) < 1e-6
    assert rel(out["power"].cpu().numpy(), ref["power"]) < 1e-9
    assert rel(out["autocorr"].cpu().numpy(), ref["autocorr"]) < 1e-6


def test_continuation(epic):
    wl = _workload(256, 64, 9, 2, 1, 44, "f16")
    v = _dev(wl)
    plan = epic.Plan.from_workload(wl).set_transform("fft_twopass")
    a = plan.image(v[:4])
    b = plan.image(v[4:], accum=a["accum"], t_prev=4)
    plan.sync()
    M = moff.map_antennas(wl.pos, wl.kern_ptr, wl.kern_dxdy, wl.kern_w, wl.dx, wl.origin, wl.n_grid)
    want = moff.moff_image(M, wl.volt, None, wl.n_grid, wl.n_pad)
    assert rel(b["image"].cpu().numpy(), want) < 1e-4


def test_rejections(epic):
    small = synth.workload_tiny(n_time=2)
    plan = epic.Plan.from_workload(small)
    with pytest.raises(epic.EpicError) as e:
        plan.set_transform("fft_twopass")
    assert e.value.status == epic.EPIC_EUNSUPPORTED
    two = _workload(64, 10, 2, 1, 2, 45, "c64")
    plan = epic.Plan.from_workload(two).set_transform("fft_twopass")
    with pytest.raises(epic.EpicError) as e:
        plan.image_xpol(_dev(two))
    assert e.value.status == epic.EPIC_EUNSUPPORTED


def test_batch_autotune_chooses_a_form_per_class(epic):
    """A batch of N_p = 512 and 128 sub-arrays: the autotuner times the 512 class in both forms;
    whatever it keeps, the images equal per-plan calls, and epic_batch_class reports it."""
    subs = [_workload(256, 200, 40, 3, 1, 46, "f16"), _workload(180, 90, 40, 2, 1, 47, "f16"),
            _workload(64, 100, 40, 2, 1, 48, "f16", n_pad=128)]
    plans = [epic.Plan.from_workload(w) for w in subs]
    volts = [_dev(w) for w in subs]
    refs = [p.image(v)["image"].cpu().numpy() for p, v in zip(plans, volts)]
    batch = epic.Batch(plans)
    acc, img = batch.alloc()
    info = batch.autotune(volts, acc)
    assert {c["n_pad"] for c in info["classes"]} == {512, 128}
    forms = {c["n_pad"]: c["form"] for c in info["classes"]}
    assert forms[128] == "persistent" and forms[512] in ("persistent", "two-pass")
    batch.image(volts, acc, img)
    torch.cuda.synchronize()
    for got, ref in zip(img, refs):
        assert rel(got.cpu().numpy(), ref) < 1e-6
