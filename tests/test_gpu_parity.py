"""CUDA path vs the FP64 oracle, element by element, through the C ABI (GPU only).

Tolerance: the FP32 path must match the FP64 oracle within 1e-4 relative L2 per image
cube, and every pixel within 1e-4 of the cube's peak (float32 gridding weights, float32
transforms of at most 2 x 8 radix stages and float32 partial sums over at most 1024
samples keep the error near 1e-6; the bound leaves two orders of margin).  Gradients:
1e-3 relative L2 against the oracle's FP64 gradient.
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


def to_dev(wl):
    if wl.vdtype == "ci4":
        return torch.from_numpy(np.ascontiguousarray(wl.volt_raw)).cuda()
    return torch.from_numpy(np.ascontiguousarray(wl.volt_raw)).cuda()


def gains_dev(g):
    return None if g is None else torch.from_numpy(np.ascontiguousarray(g.astype(np.complex64))).cuda()


def oracle_map(wl):
    return moff.map_antennas(wl.pos, wl.kern_ptr, wl.kern_dxdy, wl.kern_w, wl.dx, wl.origin, wl.n_grid)


def check_close(got, want, what):
    got = np.asarray(got, dtype=np.float64)
    rel = np.linalg.norm(got - want) / np.linalg.norm(want)
    worst = np.abs(got - want).max() / np.abs(want).max()
    assert rel < RTOL_L2, "%s: relative L2 %.3e" % (what, rel)
    assert worst < PIX, "%s: worst pixel %.3e of peak" % (what, worst)
    return rel


def run(epic, wl, gains=None, autocorr=True):
    plan = epic.Plan.from_workload(wl)
    out = plan.image(to_dev(wl), gains_dev(gains), want_autocorr=autocorr)
    torch.cuda.synchronize()
    return plan, {k: (v.cpu().numpy() if v is not None else None) for k, v in out.items()}


def test_tiny_image_and_autocorr(epic):
    """16 antennas, 2 m squares, N_p = 64, 64 samples, complex64."""
    wl = synth.workload_tiny(n_time=64)
    M = oracle_map(wl)
    plan, out = run(epic, wl)
    assert plan.info["nnz"] == M.nnz
    want = moff.moff_image(M, wl.volt, None, wl.n_grid, wl.n_pad)
    check_close(out["image"], want, "image")
    np.testing.assert_allclose(out["accum"], want * wl.n_time, rtol=1e-4, atol=1e-4 * want.max() * wl.n_time)
    ac = moff.autocorr_term(M, wl.volt, None, wl.n_grid, wl.n_pad)
    check_close(out["autocorr"], ac, "autocorr")
    pw = (np.abs(wl.volt) ** 2).sum(0)
    np.testing.assert_allclose(out["power"], pw, rtol=1e-5)


def test_lwa_slice_ci4_gains(epic):
    """LWA-like layout and 4+4-bit voltages, N_p = 128, two channels (lowest and highest),
    two pols, 48 samples, random gains."""
    wl = synth.workload_lwa(n_chan=2, n_time=48, chan_index=[0, 127])
    rng = np.random.default_rng(8)
    g = synth.random_gains(rng, (wl.n_chan, wl.n_pol, wl.n_ant))
    M = oracle_map(wl)
    _, out = run(epic, wl, g)
    want = moff.moff_image(M, wl.volt, g.astype(np.complex128), wl.n_grid, wl.n_pad)
    check_close(out["image"], want, "image")
    check_close(out["autocorr"], moff.autocorr_term(M, wl.volt, g.astype(np.complex128), wl.n_grid, wl.n_pad),
                "autocorr")


def test_hera_slice_f16_np256(epic):
    """Dense 331-antenna hexagon, 14 m disks, FP16 voltages, N_p = 256 (4-CTA clusters)."""
    wl = synth.workload_hera(n_chan=2, n_time=6)
    M = oracle_map(wl)
    _, out = run(epic, wl)
    want = moff.moff_image(M, wl.volt, None, wl.n_grid, wl.n_pad)
    check_close(out["image"], want, "image")
    check_close(out["autocorr"], moff.autocorr_term(M, wl.volt, None, wl.n_grid, wl.n_pad), "autocorr")


def test_calib_slice_np256_gains(epic):
    """1024 antennas (more than one voltage per thread), N_p = 256, complex64, gains."""
    wl = synth.workload_calib(n_chan=1, n_time=5)
    rng = np.random.default_rng(9)
    g = synth.random_gains(rng, (1, 1, wl.n_ant))
    M = oracle_map(wl)
    _, out = run(epic, wl, g, autocorr=False)
    want = moff.moff_image(M, wl.volt, g.astype(np.complex128), wl.n_grid, wl.n_pad)
    check_close(out["image"], want, "image")


def _small_workload(n_pad, n_grid, n_ant, n_time, n_chan, n_pol, seed, vdtype="c64", dx=1.0):
    rng = np.random.default_rng(seed)
    origin = np.zeros(2)
    pos = rng.uniform(1.5 * dx, (n_grid - 2.5) * dx, (n_ant, 2))
    kerns = [synth.kernel_square(rng.uniform(0.5, 2.5) * dx, dx / 3) for _ in range(n_ant)]
    ptr, dxdy, w = synth.pack_kernels(kerns)
    w = w * np.exp(1j * rng.uniform(0, 2 * np.pi, w.shape))     # complex weights
    wl = synth.Workload("small", pos, ptr, dxdy, w, dx, origin, n_grid, n_pad,
                        np.full(n_chan, 1e8), n_pol, n_time, vdtype)
    v = (rng.standard_normal((n_time, n_chan, n_pol, n_ant))
         + 1j * rng.standard_normal((n_time, n_chan, n_pol, n_ant)))
    return synth._finish(wl, v, vdtype)


@pytest.mark.parametrize("n_pad, n_grid, n_ant, n_time, n_chan, n_pol, vdtype", [
    (32, 16, 5, 7, 3, 2, "c64"),       # smallest size, several (c, p) per CTA range
    (32, 11, 40, 33, 1, 1, "f16"),     # unpadded grid smaller than N_p / 2
    (64, 32, 1, 3, 1, 1, "c64"),       # a single antenna
    (64, 20, 300, 17, 2, 1, "ci4"),    # ragged grid, A > threads per CTA
    (128, 64, 700, 9, 1, 2, "c64"),    # A beyond the register prefetch (4 per thread)
    (256, 100, 64, 3, 2, 1, "f16"),
    (256, 90, 80, 150, 1, 1, "c64"),   # two row-pass buffers, several items (both parities) per cluster
    (256, 60, 1600, 150, 1, 1, "ci4"), # one row-pass buffer (two do not fit beside 1600 antennas)
    (512, 40, 30, 3, 1, 1, "c64"),     # 16-CTA clusters
    (512, 40, 30, 40, 1, 1, "c64"),    # several items per 16-CTA cluster
    (512, 256, 12, 2, 1, 1, "f16"),    # full 256 x 256 unpadded grid
])
def test_small_sizes(epic, n_pad, n_grid, n_ant, n_time, n_chan, n_pol, vdtype):
    wl = _small_workload(n_pad, n_grid, n_ant, n_time, n_chan, n_pol, seed=n_pad + n_ant, vdtype=vdtype)
    rng = np.random.default_rng(n_ant)
    g = synth.random_gains(rng, (n_chan, n_pol, n_ant))
    M = oracle_map(wl)
    _, out = run(epic, wl, g)
    gg = g.astype(np.complex128)
    check_close(out["image"], moff.moff_image(M, wl.volt, gg, wl.n_grid, wl.n_pad), "image")
    check_close(out["autocorr"], moff.autocorr_term(M, wl.volt, gg, wl.n_grid, wl.n_pad), "autocorr")


def test_dense_footprints(epic):
    """Apertures much wider than the grid spacing (more than 24 mapping entries per occupied
    cell on average, long CSR rows in the gridding gather); same bound against the oracle, at
    N_p = 64 and at N_p = 256 (clusters, round-robin gather), forward and gradient."""
    for n_pad, n_grid, n_ant in ((64, 32, 300), (256, 40, 450)):
        rng = np.random.default_rng(n_pad)
        dx = 1.0
        pos = rng.uniform(7.0, n_grid - 8.0, (n_ant, 2))
        kerns = [synth.kernel_square(rng.uniform(8.0, 11.0), 0.5) for _ in range(n_ant)]
        ptr, dxdy, w = synth.pack_kernels(kerns)
        wl = synth.Workload("dense", pos, ptr, dxdy, w, dx, np.zeros(2), n_grid, n_pad, np.full(2, 1e8), 1, 5, "c64")
        v = rng.standard_normal((5, 2, 1, n_ant)) + 1j * rng.standard_normal((5, 2, 1, n_ant))
        wl = synth._finish(wl, v, "c64")
        M = oracle_map(wl)
        plan, out = run(epic, wl)
        assert plan.info["nnz"] / plan.info["n_cells"] >= 24.0
        check_close(out["image"], moff.moff_image(M, wl.volt, None, wl.n_grid, wl.n_pad), "image")
        G = rng.standard_normal((2, 1, n_pad, n_pad)).astype(np.float32)
        want = moff.grad_gains(M, wl.volt, np.ones((2, 1, n_ant)), wl.n_grid, wl.n_pad, G.astype(np.float64))
        got = plan.image_backward(to_dev(wl), None, torch.from_numpy(G).cuda()).cpu().numpy()
        assert np.linalg.norm(got - want) / np.linalg.norm(want) < 1e-3


def test_continuation_matches_single_call(epic):
    """Resuming an integration (t_prev > 0) equals integrating all samples at once."""
    wl = synth.workload_tiny(n_time=40)
    plan = epic.Plan.from_workload(wl)
    v = to_dev(wl)
    full = plan.image(v, want_autocorr=True)
    part = plan.image(v[:15].contiguous(), want_autocorr=True)
    rest = plan.image(v[15:].contiguous(), accum=part["accum"], power=part["power"], t_prev=15, want_autocorr=True)
    torch.cuda.synchronize()
    for k in ("image", "autocorr", "accum", "power"):
        a, b = full[k].cpu().numpy(), rest[k].cpu().numpy()
        assert np.abs(a - b).max() <= 1e-6 * np.abs(a).max(), k


def test_zero_gains_and_empty_antennas(epic):
    wl = _small_workload(64, 32, 6, 4, 1, 1, seed=3)
    # antennas 2 and 4 have no footprint samples
    ptr = wl.kern_ptr.copy()
    keep = np.ones(wl.kern_dxdy.shape[0], bool)
    for a in (2, 4):
        keep[ptr[a]:ptr[a + 1]] = False
    counts = np.diff(ptr)
    counts[[2, 4]] = 0
    wl.kern_ptr = np.concatenate([[0], np.cumsum(counts)]).astype(np.int32)
    wl.kern_dxdy, wl.kern_w = wl.kern_dxdy[keep], wl.kern_w[keep]
    M = oracle_map(wl)
    _, out = run(epic, wl)
    check_close(out["image"], moff.moff_image(M, wl.volt, None, wl.n_grid, wl.n_pad), "image")
    _, out0 = run(epic, wl, np.zeros((1, 1, wl.n_ant), np.complex64))
    assert np.abs(out0["image"]).max() == 0.0


def test_determinism_of_mapping_counts(epic):
    wl = synth.workload_lwa(n_chan=1, n_time=2, chan_index=[5])
    plan = epic.Plan.from_workload(wl)
    M = oracle_map(wl)
    assert plan.info["nnz"] == M.nnz
    assert plan.info["n_cells"] == len(np.unique(M.tocoo().row))


@pytest.mark.parametrize("n_pad, n_grid, n_ant, n_time, n_chan, vdtype", [
    (32, 16, 7, 5, 2, "c64"),
    (64, 30, 40, 6, 1, "ci4"),
    (128, 64, 90, 4, 1, "f16"),
    (256, 128, 50, 3, 1, "c64"),
    (512, 60, 20, 2, 1, "f16"),
])
def test_gradient_matches_oracle(epic, n_pad, n_grid, n_ant, n_time, n_chan, vdtype):
    wl = _small_workload(n_pad, n_grid, n_ant, n_time, n_chan, 1, seed=n_ant, vdtype=vdtype)
    rng = np.random.default_rng(n_pad)
    g = synth.random_gains(rng, (n_chan, 1, n_ant))
    G = rng.standard_normal((n_chan, 1, n_pad, n_pad)).astype(np.float32)
    M = oracle_map(wl)
    want = moff.grad_gains(M, wl.volt, g.astype(np.complex128), wl.n_grid, wl.n_pad, G.astype(np.float64))
    plan = epic.Plan.from_workload(wl)
    got = plan.image_backward(to_dev(wl), gains_dev(g), torch.from_numpy(G).cuda()).cpu().numpy()
    rel = np.linalg.norm(got - want) / np.linalg.norm(want)
    assert rel < 1e-3, rel
    # element by element: no antenna's gradient is off by more than 1e-4 of the largest one
    # (FP32 sums over every pixel and sample), and every antenna whose gradient is at least 1 %
    # of the largest is within 1e-3 of its own value
    err, scale = np.abs(got - want), np.abs(want).max()
    assert err.max() <= 1e-4 * scale, (err.max(), scale)
    big = np.abs(want) >= 1e-2 * scale
    assert big.any() and (err[big] <= 1e-3 * np.abs(want[big])).all(), (err[big] / np.abs(want[big])).max()


def test_autograd_function(epic):
    """torch.autograd through the library's adjoint equals the oracle gradient of
    L = sum (I - I_model)^2."""
    wl = _small_workload(64, 32, 12, 6, 1, 1, seed=21)
    rng = np.random.default_rng(22)
    g0 = synth.random_gains(rng, (1, 1, wl.n_ant))
    I_model = rng.uniform(0, 1, (1, 1, 64, 64))
    plan = epic.Plan.from_workload(wl)
    g = gains_dev(g0).requires_grad_(True)
    img = epic.moff_image(g, to_dev(wl), plan)
    loss = ((img.double() - torch.from_numpy(I_model).cuda()) ** 2).sum()
    loss.backward()
    M = oracle_map(wl)
    I = moff.moff_image(M, wl.volt, g0.astype(np.complex128), 32, 64)
    want = moff.grad_gains(M, wl.volt, g0.astype(np.complex128), 32, 64, 2 * (I - I_model))
    got = g.grad.cpu().numpy()
    assert np.linalg.norm(got - want) / np.linalg.norm(want) < 1e-3


def test_python_layer_rejects_bad_shapes(epic):
    wl = synth.workload_tiny(n_time=4)
    plan = epic.Plan.from_workload(wl)
    with pytest.raises(ValueError):
        plan.image(torch.zeros((4, 1, 1, wl.n_ant + 1), dtype=torch.complex64, device="cuda"))
    with pytest.raises(ValueError):
        plan.image(to_dev(wl), torch.ones((1, 1, 3), dtype=torch.complex64, device="cuda"))
    with pytest.raises(epic.EpicError):
        epic.epic_image(plan._h, to_dev(wl).data_ptr(), 0, None, None, None, 0, None, None, None)


# ---------------------------------------------------------------------------------------------
# the tensor-core DFT form (N_p = 128), same oracle and same tolerance as the FP32 FFT form
# ---------------------------------------------------------------------------------------------
@pytest.mark.parametrize("n_grid, n_ant, n_time, n_chan, n_pol, vdtype", [
    (64, 40, 5, 2, 1, "c64"),       # complex weights, two channels
    (37, 300, 9, 1, 2, "f16"),      # ragged grid, A above the threads per CTA
    (64, 700, 4, 1, 1, "ci4"),      # many antennas
])
def test_dftgemm_small(epic, n_grid, n_ant, n_time, n_chan, n_pol, vdtype):
    wl = _small_workload(128, n_grid, n_ant, n_time, n_chan, n_pol, seed=n_ant + 7, vdtype=vdtype)
    rng = np.random.default_rng(n_ant + 1)
    g = synth.random_gains(rng, (n_chan, n_pol, n_ant))
    M = oracle_map(wl)
    plan = epic.Plan.from_workload(wl).set_transform("dftgemm")
    out = plan.image(to_dev(wl), gains_dev(g), want_autocorr=True)
    torch.cuda.synchronize()
    gg = g.astype(np.complex128)
    check_close(out["image"].cpu().numpy(), moff.moff_image(M, wl.volt, gg, wl.n_grid, wl.n_pad), "image")
    check_close(out["autocorr"].cpu().numpy(), moff.autocorr_term(M, wl.volt, gg, wl.n_grid, wl.n_pad), "autocorr")
    np.testing.assert_allclose(out["power"].cpu().numpy(), (np.abs(wl.volt * gg[None]) ** 2).sum(0), rtol=1e-5)


def test_dftgemm_deep_pipeline_gains(epic):
    """LWA-like slice, 2 channels x 2 pols x 1024 samples: every CTA images about 27
    consecutive samples, so the double-buffered pipeline runs in its steady state (gridding of
    sample i+1 under both DFT stages of sample i) and across (channel, pol) boundaries; random
    gains, power and auto-correlation term against the oracle."""
    wl = synth.workload_lwa(n_chan=2, n_time=1024, chan_index=[5, 100])
    rng = np.random.default_rng(17)
    g = synth.random_gains(rng, (wl.n_chan, wl.n_pol, wl.n_ant))
    M = oracle_map(wl)
    plan = epic.Plan.from_workload(wl).set_transform("dftgemm")
    out = plan.image(to_dev(wl), gains_dev(g), want_autocorr=True)
    torch.cuda.synchronize()
    gg = g.astype(np.complex128)
    check_close(out["image"].cpu().numpy(), moff.moff_image(M, wl.volt, gg, wl.n_grid, wl.n_pad), "image")
    check_close(out["autocorr"].cpu().numpy(), moff.autocorr_term(M, wl.volt, gg, wl.n_grid, wl.n_pad), "autocorr")
    np.testing.assert_allclose(out["power"].cpu().numpy(), (np.abs(wl.volt * gg[None]) ** 2).sum(0), rtol=1e-5)


def test_dftgemm_tables_beyond_shared_memory(epic):
    """2000 antennas with complex weights: the gridding's slot tables (over 10,000 entries of
    12 bytes) do not fit in shared memory beside the DFT operand tables, so the kernel reads
    them through L1 instead of copying them; same oracle, same tolerance."""
    wl = _small_workload(128, 64, 2000, 3, 1, 1, seed=2021, vdtype="c64")
    M = oracle_map(wl)
    assert M.nnz * 12 > 96 * 1024      # more than shared memory has left for the tables
    rng = np.random.default_rng(5)
    g = synth.random_gains(rng, (1, 1, wl.n_ant))
    plan = epic.Plan.from_workload(wl).set_transform("dftgemm")
    out = plan.image(to_dev(wl), gains_dev(g))
    torch.cuda.synchronize()
    check_close(out["image"].cpu().numpy(), moff.moff_image(M, wl.volt, g.astype(np.complex128), wl.n_grid, wl.n_pad),
                "image")


def test_dftgemm_antenna_limit(epic):
    """The tensor-core form keeps four per-antenna arrays beside its operand tables in shared
    memory: 2400 antennas fit (imaged against the oracle, gather tables read through L1),
    2500 do not and the transform is refused with EPIC_EUNSUPPORTED."""
    wl = _small_workload(128, 64, 2400, 2, 1, 1, seed=24, vdtype="ci4")
    M = oracle_map(wl)
    plan = epic.Plan.from_workload(wl).set_transform("dftgemm")
    out = plan.image(to_dev(wl))
    torch.cuda.synchronize()
    check_close(out["image"].cpu().numpy(), moff.moff_image(M, wl.volt, None, wl.n_grid, wl.n_pad), "image")
    big = _small_workload(128, 64, 2500, 1, 1, 1, seed=25, vdtype="ci4")
    plan = epic.Plan.from_workload(big)
    with pytest.raises(epic.EpicError) as e:
        plan.set_transform("dftgemm")
    assert e.value.status == epic.EPIC_EUNSUPPORTED


def test_dftgemm_lwa_slice_matches_fft(epic):
    """LWA-like slice (4+4-bit, 2 channels, 2 pols, 48 samples): tensor-core form vs the oracle
    and vs the FP32 FFT form; the continuation rule holds for it too."""
    wl = synth.workload_lwa(n_chan=2, n_time=48, chan_index=[3, 120])
    M = oracle_map(wl)
    v = to_dev(wl)
    plan = epic.Plan.from_workload(wl)
    ref = plan.image(v)["image"].cpu().numpy()
    plan.set_transform("dftgemm")
    got = plan.image(v)["image"].cpu().numpy()
    want = moff.moff_image(M, wl.volt, None, wl.n_grid, wl.n_pad)
    check_close(got, want, "tensor-core image")
    check_close(ref, want, "fft image")
    part = plan.image(v[:20].contiguous())
    rest = plan.image(v[20:].contiguous(), accum=part["accum"], t_prev=20)["image"].cpu().numpy()
    assert np.abs(rest - got).max() <= 1e-6 * np.abs(got).max()


def test_dftgemm_rejects_other_sizes(epic):
    wl = synth.workload_tiny(n_time=2)
    plan = epic.Plan.from_workload(wl)
    with pytest.raises(epic.EpicError) as e:
        plan.set_transform("dftgemm")
    assert e.value.status == epic.EPIC_EUNSUPPORTED


def test_forward_only_plan_beyond_adjoint_limit(epic):
    """3000 antennas at N_p = 128 fit the forward kernel but not the adjoint's four per-antenna
    arrays: the plan is created and images against the oracle, and the adjoint call is refused
    on the host (EPIC_EUNSUPPORTED) before any launch."""
    wl = _small_workload(128, 40, 3000, 3, 1, 1, seed=30, vdtype="ci4")
    M = oracle_map(wl)
    plan, out = run(epic, wl, autocorr=False)
    check_close(out["image"], moff.moff_image(M, wl.volt, None, wl.n_grid, wl.n_pad), "image")
    G = torch.ones((1, 1, wl.n_pad, wl.n_pad), dtype=torch.float32, device="cuda")
    with pytest.raises(epic.EpicError) as e:
        plan.image_backward(to_dev(wl), None, G)
    assert e.value.status == epic.EPIC_EUNSUPPORTED
