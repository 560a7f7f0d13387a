"""Full-size workloads on the GPU (the launch configurations the benchmark times), checked
against the FP64 oracle on sampled (channel, pol) images it can compute one by one, and the
gain-calibration use of the adjoint (GPU only)."""
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


def rel_l2(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / np.linalg.norm(b))


@pytest.fixture(scope="module")
def lwa_full():
    return synth.workload_lwa()


@pytest.mark.parametrize("xform", ["fft", "dftgemm"])
def test_lwa_full_size_sampled(epic, lwa_full, xform):
    """256 antennas x 128 channels x 2 pols x 1024 samples, 4+4-bit, N_p = 128: the whole
    integration in one epic_image call, in both transform forms (the bench times both and
    reports the tensor-core one); three sampled (channel, pol) images and their
    auto-correlation terms against the oracle over all 1024 samples."""
    wl = lwa_full
    plan = epic.Plan.from_workload(wl).set_transform(xform)
    out = plan.image(torch.from_numpy(wl.volt_raw).cuda(), want_autocorr=True)
    torch.cuda.synchronize()
    img = out["image"].cpu().numpy()
    ac = out["autocorr"].cpu().numpy()
    M = moff.map_antennas(wl.pos, wl.kern_ptr, wl.kern_dxdy, wl.kern_w, wl.dx, wl.origin, wl.n_grid)
    assert plan.info["nnz"] == M.nnz
    for c, p in [(0, 0), (64, 1), (127, 1)]:
        v = wl.volt[:, c:c + 1, p:p + 1, :]
        want = moff.moff_image(M, v, None, wl.n_grid, wl.n_pad)[0, 0]
        assert rel_l2(img[c, p], want) < 1e-4
        assert np.abs(img[c, p] - want).max() < 1e-4 * want.max()
        want_ac = moff.autocorr_term(M, v, None, wl.n_grid, wl.n_pad)[0, 0]
        assert rel_l2(ac[c, p], want_ac) < 1e-4
    # properties that hold for every image of the cube
    assert np.isfinite(img).all() and img.min() >= 0.0
    assert (img.sum(axis=(2, 3)) > 0).all()


def test_lwa_full_size_forms_agree(epic, lwa_full):
    """Every one of the 256 (channel, pol) images of the full LWA-like integration: the
    tensor-core form within the FP32 bound (1e-4 relative L2, every pixel within 1e-4 of the
    peak) of the FFT form, whose own images the oracle checks on samples."""
    wl = lwa_full
    v = torch.from_numpy(wl.volt_raw).cuda()
    plan = epic.Plan.from_workload(wl)
    ref = plan.image(v)["image"].cpu().numpy().astype(np.float64)
    got = plan.set_transform("dftgemm").image(v)["image"].cpu().numpy().astype(np.float64)
    d = np.linalg.norm((got - ref).reshape(-1, wl.n_pad ** 2), axis=1) / np.linalg.norm(ref.reshape(-1, wl.n_pad ** 2), axis=1)
    assert d.max() < 1e-4, d.max()
    assert (np.abs(got - ref).max(axis=(2, 3)) < 1e-4 * ref.max(axis=(2, 3))).all()


def test_lwa_full_size_fx_route(epic, lwa_full):
    """The FX route on the full LWA-like integration, in the launches the bench times
    (epic_correlate of all 256 (channel, pol) planes, then epic_fx_image: 64 planes per warp
    with 16-byte visibility loads): every plane's FX image equals the MOFF image of the same
    data (Sec. 2: the two routes are equivalent with the autocorrelations included) within the
    FP32 bound, and two sampled planes equal the oracle's FX route."""
    from oracle import fx
    wl = lwa_full
    v = torch.from_numpy(wl.volt_raw).cuda()
    plan = epic.Plan.from_workload(wl)
    moff_img = plan.image(v)["image"].cpu().numpy().astype(np.float64)
    fx_img = plan.fx_image(plan.correlate(v)).cpu().numpy().astype(np.float64)
    n = wl.n_pad ** 2
    d = np.linalg.norm((fx_img - moff_img).reshape(-1, n), axis=1) / np.linalg.norm(moff_img.reshape(-1, n), axis=1)
    assert d.max() < 1e-4, d.max()
    assert (np.abs(fx_img - moff_img).max(axis=(2, 3)) < 1e-4 * moff_img.max(axis=(2, 3))).all()
    M = moff.map_antennas(wl.pos, wl.kern_ptr, wl.kern_dxdy, wl.kern_w, wl.dx, wl.origin, wl.n_grid)
    for c, p in [(5, 0), (127, 1)]:
        want = fx.fx_image(M, wl.volt[:, c:c + 1, p:p + 1, :], None, wl.n_grid, wl.n_pad).real[0, 0]
        assert rel_l2(fx_img[c, p], want) < 1e-4
        assert np.abs(fx_img[c, p] - want).max() < 1e-4 * np.abs(want).max()


def test_hera_full_size_both_forms(epic):
    """The dense layout at its full 1024 channels x 256 samples, FP16 voltages, N_p = 256, in the
    launches the bench times: the tensor-core split form's 1024 images within the FP32 bound of
    the FFT form's, and the first and last channel of both against the oracle."""
    wl = synth.workload_hera()
    v = torch.from_numpy(wl.volt_raw).cuda()
    plan = epic.Plan.from_workload(wl)
    ref = plan.image(v)["image"].cpu().numpy()
    got = plan.set_transform("dftgemm").image(v)["image"].cpu().numpy()
    plan.sync()
    n = wl.n_pad ** 2
    r64, g64 = ref.reshape(-1, n).astype(np.float64), got.reshape(-1, n).astype(np.float64)
    d = np.linalg.norm(g64 - r64, axis=1) / np.linalg.norm(r64, axis=1)
    assert d.max() < 1e-4, d.max()
    M = moff.map_antennas(wl.pos, wl.kern_ptr, wl.kern_dxdy, wl.kern_w, wl.dx, wl.origin, wl.n_grid)
    for c in (0, wl.n_chan - 1):
        want = moff.moff_image(M, wl.volt[:, c:c + 1], None, wl.n_grid, wl.n_pad)[0, 0]
        for img in (ref, got):
            assert rel_l2(img[c, 0], want) < 1e-4
            assert np.abs(img[c, 0] - want).max() < 1e-4 * want.max()


def test_hera_full_layout_channel_slice(epic):
    """331-antenna hexagon, FP16 voltages, N_p = 256 clusters, 16 channels x 256 samples;
    the first and last channel against the oracle over all samples."""
    wl = synth.workload_hera(n_chan=16, n_time=256)
    plan = epic.Plan.from_workload(wl)
    img = plan.image(torch.from_numpy(wl.volt_raw).cuda())["image"]
    torch.cuda.synchronize()
    img = img.cpu().numpy()
    M = moff.map_antennas(wl.pos, wl.kern_ptr, wl.kern_dxdy, wl.kern_w, wl.dx, wl.origin, wl.n_grid)
    want = moff.moff_image(M, wl.volt[:, 0:1], None, wl.n_grid, wl.n_pad)[0, 0]     # all 256 samples
    assert rel_l2(img[0, 0], want) < 1e-4
    want = moff.moff_image(M, wl.volt[:, 15:16], None, wl.n_grid, wl.n_pad)[0, 0]
    assert rel_l2(img[15, 0], want) < 1e-4
    assert np.isfinite(img).all() and img.min() >= 0.0


def test_gain_calibration_adam(epic):
    """Differentiation form (1024 antennas in a 300 m disk, 32 channels, 64 samples, N_p = 256):
    the loss is the squared L2 distance between the integrated image and the model image of
    the known sources; 100 Adam steps on the complex gains through the library's adjoint
    must reduce the loss and move the gains towards the true calibration (up to the global
    phase the image cannot see)."""
    wl = synth.workload_calib()
    rng = np.random.default_rng(51)
    g_true = wl.extra["g_true"]
    # model: the expectation over source phases of the noiseless image of the known sources
    # with unit gains, sum_s S_s |AF_s(k)|^2 -- one "sample" per source, each carrying a single
    # source with amplitude sqrt(n_src S_s), so the time average is the sum over sources
    sky = wl.extra["sky"]
    n_src = sky.flux.size
    model_v = np.zeros((n_src, wl.n_chan, 1, wl.n_ant), np.complex128)
    for s in range(n_src):
        one = synth.Sky(sky.l[s:s + 1], sky.m[s:s + 1], np.array([n_src * sky.flux[s]]))
        model_v[s:s + 1] = synth.voltages(np.random.default_rng(s), wl.pos, wl.freqs, 1, 1, one, 0.0,
                                          dtype=np.complex128)
    plan = epic.Plan.from_workload(wl)
    volt = torch.from_numpy(wl.volt_raw).cuda()
    mv = torch.from_numpy(synth.to_c64_pairs(model_v)).cuda()
    I_model = plan.image(mv)["image"].detach()
    # start inside the basin: the inverse true gains, perturbed in amplitude and phase
    ideal = (1.0 / g_true).astype(np.complex64)
    pert = (1 + 0.2 * rng.standard_normal(wl.n_ant)) * np.exp(0.4j * rng.standard_normal(wl.n_ant))
    g = torch.from_numpy((ideal * pert).astype(np.complex64)).cuda().requires_grad_(True)   # one gain per antenna
    opt = torch.optim.Adam([g], lr=0.01)

    def gain_error(gg):
        x = gg.detach().cpu().numpy() * g_true
        x = x * np.exp(-1j * np.angle(x.mean()))
        return float(np.linalg.norm(x - np.abs(x).mean()) / np.sqrt(x.size))

    losses = []
    err0 = gain_error(g)
    for _ in range(100):
        opt.zero_grad()
        gc = g.view(1, 1, -1).expand(wl.n_chan, 1, wl.n_ant).contiguous()   # shared by all channels
        img = epic.moff_image(gc, volt, plan)
        loss = ((img - I_model) ** 2).sum()
        loss.backward()
        opt.step()
        losses.append(float(loss.detach()))
    err1 = gain_error(g)
    assert all(np.isfinite(losses))
    assert losses[-1] < 0.5 * losses[0], (err0, err1, losses[0], losses[-1])
    assert err1 < 0.5 * err0, (err0, err1, losses[0], losses[-1])
