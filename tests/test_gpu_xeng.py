"""X-engine of the FX route (epic_correlate) vs the FP64 oracle's visibilities (GPU only).

Tolerance: for 4+4-bit voltages the tensor-core sums are exact integers (FP16 operands, FP32
accumulation below 2^24), so the only rounding is the FP32 scaling by 1/T and the gains:
relative L2 < 1e-6 per (channel, pol) matrix and every element within 1e-6 of the largest.
FP16 voltages: products are exact in FP32, their sums round; the same bound holds with
margin for the sample counts used here.
"""
import numpy as np
import pytest

from oracle import fx, moff
from paper_1510_08318_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-6


@pytest.fixture(scope="module")
def epic():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1510_08318_gb300 import build, epic as ep
    build.build()
    ep.load()
    return ep


def run(epic, wl, gains=None):
    plan = epic.Plan.from_workload(wl)
    g = None if gains is None else torch.from_numpy(np.ascontiguousarray(gains.astype(np.complex64))).cuda()
    vis = plan.correlate(torch.from_numpy(np.ascontiguousarray(wl.volt_raw)).cuda(), g)
    torch.cuda.synchronize()
    return plan, vis.cpu().numpy()


def check(got, wl, gains, what):
    T, C, P, A = wl.volt.shape
    for c in range(C):
        for p in range(P):
            g = np.ones(A, dtype=np.complex128) if gains is None else gains[c, p].astype(np.complex128)
            want = fx.visibilities(wl.volt[:, c, p, :], g)
            err = got[c, p] - want
            assert np.linalg.norm(err) / np.linalg.norm(want) < TOL, (what, c, p)
            assert np.abs(err).max() < TOL * np.abs(want).max(), (what, c, p)
            # Hermitian (mirrored blocks are written as exact conjugates)
            assert np.abs(got[c, p] - np.conj(got[c, p].T)).max() <= 1e-6 * np.abs(want).max(), (what, "hermitian")


def _small(n_ant, n_time, n_chan, n_pol, vdtype, seed, n_grid=24, n_pad=64):
    rng = np.random.default_rng(seed)
    pos = rng.uniform(2.0, n_grid - 3.0, (n_ant, 2))
    kerns = [synth.kernel_square(rng.uniform(0.5, 2.5), 1 / 3) for _ in range(n_ant)]
    ptr, dxdy, w = synth.pack_kernels(kerns)
    wl = synth.Workload("xeng", pos, ptr, dxdy, w, 1.0, np.zeros(2), n_grid, n_pad,
                        np.full(n_chan, 1e8), n_pol, n_time, vdtype)
    v = (rng.standard_normal((n_time, n_chan, n_pol, n_ant))
         + 1j * rng.standard_normal((n_time, n_chan, n_pol, n_ant)))
    return synth._finish(wl, v, vdtype)


def test_lwa_slice_ci4_gains(epic):
    """LWA-like 4+4-bit voltages, 256 antennas (2 x 2 blocks), two channels x two pols, 70
    samples (a ragged 32-sample chunk), random gains."""
    wl = synth.workload_lwa(n_chan=2, n_time=70, chan_index=[0, 127])
    g = synth.random_gains(np.random.default_rng(8), (wl.n_chan, wl.n_pol, wl.n_ant))
    _, vis = run(epic, wl, g)
    check(vis, wl, g, "lwa")


def test_lwa_units_beyond_one_per_cta(epic):
    """384 units (64 channels x 2 pols x 3 blocks) on at most one CTA per SM: CTAs that own
    several units load the next unit's first chunks while finishing the current one and drain
    one accumulator buffer while filling the other (4+4-bit voltages on 4-byte loads; 40
    samples, a ragged second chunk)."""
    wl = synth.workload_lwa(n_chan=64, n_time=40, chan_index=list(range(0, 128, 2)))
    g = synth.random_gains(np.random.default_rng(9), (wl.n_chan, wl.n_pol, wl.n_ant))
    _, vis = run(epic, wl, g)
    check(vis, wl, g, "lwa 384 units")


def test_hera_slice_f16(epic):
    """331 antennas (3 x 3 blocks with a 75-antenna tail), FP16 voltages, 40 samples."""
    wl = synth.workload_hera(n_chan=2, n_time=40)
    _, vis = run(epic, wl)
    check(vis, wl, None, "hera")


@pytest.mark.parametrize("n_ant, n_time, n_chan, n_pol, vdtype", [
    (1, 1, 1, 1, "ci4"),        # one antenna, one sample
    (129, 31, 1, 2, "f16"),     # a one-antenna tail block, less than one chunk
    (300, 33, 2, 1, "ci4"),     # three blocks, one sample past a chunk
    (640, 64, 1, 1, "ci4"),     # five full blocks, two full chunks
    (336, 45, 1, 2, "ci4"),     # 4-byte loads with an 80-antenna tail block, a ragged chunk
    (130, 70, 1, 1, "ci4"),     # A not a multiple of 4: byte loads, a two-antenna tail block
    (4, 3, 3, 2, "ci4"),        # the smallest 4-byte-load case: one lane's antennas, 3 samples
])
def test_small_shapes(epic, n_ant, n_time, n_chan, n_pol, vdtype):
    wl = _small(n_ant, n_time, n_chan, n_pol, vdtype, seed=n_ant + n_time)
    g = synth.random_gains(np.random.default_rng(n_ant), (n_chan, n_pol, n_ant))
    _, vis = run(epic, wl, g)
    check(vis, wl, g, "A=%d T=%d" % (n_ant, n_time))


def test_fx_image_from_gpu_visibilities_equals_moff(epic):
    """The two routes of Sec. 2 on the same data: the FX image formed (by the oracle's lag-plane
    gridding and transform) from the GPU's visibilities equals the GPU's MOFF image."""
    wl = _small(48, 40, 1, 1, "f16", seed=5, n_grid=24, n_pad=64)
    plan, vis = run(epic, wl)
    M = moff.map_antennas(wl.pos, wl.kern_ptr, wl.kern_dxdy, wl.kern_w, wl.dx, wl.origin, wl.n_grid)
    img_fx = fx.image_from_uv(fx.uv_plane(M, vis[0, 0].astype(np.complex128), wl.n_grid), wl.n_grid, wl.n_pad)
    img = plan.image(torch.from_numpy(np.ascontiguousarray(wl.volt_raw)).cuda())["image"].cpu().numpy()[0, 0]
    assert np.abs(img_fx.imag).max() < 1e-5 * img.max()
    assert np.linalg.norm(img_fx.real - img) / np.linalg.norm(img) < 1e-5


def test_full_lwa_workload_sampled(epic):
    """The full LWA-like call (128 channels x 2 pols x 1024 samples) in the bench's launch;
    three (channel, pol) matrices against the oracle."""
    wl = synth.workload_lwa()
    plan = epic.Plan.from_workload(wl)
    vis = plan.correlate(torch.from_numpy(np.ascontiguousarray(wl.volt_raw)).cuda())
    torch.cuda.synchronize()
    one = np.ones(wl.n_ant, dtype=np.complex128)
    for c, p in ((0, 0), (64, 1), (127, 1)):
        want = fx.visibilities(wl.volt[:, c, p, :], one)
        got = vis[c, p].cpu().numpy()
        assert np.linalg.norm(got - want) / np.linalg.norm(want) < TOL, (c, p)


def test_rejects_complex64(epic):
    wl = synth.workload_tiny(n_time=2)
    plan = epic.Plan.from_workload(wl)
    with pytest.raises(epic.EpicError):
        plan.correlate(torch.from_numpy(np.ascontiguousarray(wl.volt_raw)).cuda())


def test_gpu_fx_route_equals_moff(epic):
    """Both routes of Sec. 2 entirely on the GPU: epic_correlate then epic_fx_image gives the
    image epic_image gives (LWA slice, 4+4-bit, gains; N_p = 128), and matches the FP64 oracle."""
    wl = synth.workload_lwa(n_chan=2, n_time=64, chan_index=[0, 127])
    g = synth.random_gains(np.random.default_rng(4), (wl.n_chan, wl.n_pol, wl.n_ant))
    gd = torch.from_numpy(np.ascontiguousarray(g.astype(np.complex64))).cuda()
    plan = epic.Plan.from_workload(wl)
    v = torch.from_numpy(np.ascontiguousarray(wl.volt_raw)).cuda()
    fx_img = plan.fx_image(plan.correlate(v, gd)).cpu().numpy()
    moff_img = plan.image(v, gd)["image"].cpu().numpy()
    M = moff.map_antennas(wl.pos, wl.kern_ptr, wl.kern_dxdy, wl.kern_w, wl.dx, wl.origin, wl.n_grid)
    want = moff.moff_image(M, wl.volt, g.astype(np.complex128), wl.n_grid, wl.n_pad)
    for got in (fx_img, moff_img):
        assert np.linalg.norm(got - want) / np.linalg.norm(want) < 1e-4
        assert np.abs(got - want).max() < 1e-4 * want.max()


@pytest.mark.parametrize("n_pad, n_grid, n_ant", [(32, 14, 20), (64, 30, 60)])
def test_gpu_fx_image_small_sizes_complex_weights(epic, n_pad, n_grid, n_ant):
    """FX imaging at N_p = 32 and 64 with complex footprint weights, against the oracle's FX route."""
    rng = np.random.default_rng(n_pad)
    pos = rng.uniform(2.0, n_grid - 3.0, (n_ant, 2))
    kerns = [synth.kernel_square(rng.uniform(0.5, 2.5), 1 / 3) for _ in range(n_ant)]
    ptr, dxdy, w = synth.pack_kernels(kerns)
    w = w * np.exp(1j * rng.uniform(0, 2 * np.pi, w.shape))
    wl = synth.Workload("fxs", pos, ptr, dxdy, w, 1.0, np.zeros(2), n_grid, n_pad, np.full(1, 1e8), 1, 24, "f16")
    v = rng.standard_normal((24, 1, 1, n_ant)) + 1j * rng.standard_normal((24, 1, 1, n_ant))
    wl = synth._finish(wl, v, "f16")
    plan = epic.Plan.from_workload(wl)
    img = plan.fx_image(plan.correlate(torch.from_numpy(np.ascontiguousarray(wl.volt_raw)).cuda())).cpu().numpy()
    M = moff.map_antennas(wl.pos, wl.kern_ptr, wl.kern_dxdy, wl.kern_w, wl.dx, wl.origin, wl.n_grid)
    want = fx.fx_image(M, wl.volt, None, wl.n_grid, wl.n_pad).real
    assert np.linalg.norm(img - want) / np.linalg.norm(want) < 1e-4


@pytest.mark.parametrize("n_chan, n_pol", [(1, 1), (2, 1), (3, 1), (20, 2), (33, 2), (65, 1)])
def test_gpu_fx_image_plane_groupings(epic, n_chan, n_pol):
    """The lag-plane gather's groupings of (channel, pol) planes: 1 and 2 planes (32 and 16
    entries side by side per warp), 3 planes (one group of 4),
    40 (two groups of 32, the second ragged), 66 (two groups of 64 read 16 bytes per lane, the
    second ragged) and 65 (odd: three groups of 32).  Every plane against the oracle's FX route
    (complex footprint weights, N_p = 32)."""
    rng = np.random.default_rng(100 + n_chan * n_pol)
    n_grid, n_pad, n_ant, n_time = 14, 32, 20, 16
    pos = rng.uniform(2.0, n_grid - 3.0, (n_ant, 2))
    kerns = [synth.kernel_square(rng.uniform(0.5, 2.5), 1 / 3) for _ in range(n_ant)]
    ptr, dxdy, w = synth.pack_kernels(kerns)
    w = w * np.exp(1j * rng.uniform(0, 2 * np.pi, w.shape))
    wl = synth.Workload("fxg", pos, ptr, dxdy, w, 1.0, np.zeros(2), n_grid, n_pad, np.full(n_chan, 1e8), n_pol,
                        n_time, "f16")
    v = rng.standard_normal((n_time, n_chan, n_pol, n_ant)) + 1j * rng.standard_normal((n_time, n_chan, n_pol, n_ant))
    wl = synth._finish(wl, v, "f16")
    plan = epic.Plan.from_workload(wl)
    img = plan.fx_image(plan.correlate(torch.from_numpy(np.ascontiguousarray(wl.volt_raw)).cuda())).cpu().numpy()
    M = moff.map_antennas(wl.pos, wl.kern_ptr, wl.kern_dxdy, wl.kern_w, wl.dx, wl.origin, wl.n_grid)
    want = fx.fx_image(M, wl.volt, None, wl.n_grid, wl.n_pad).real
    assert img.shape == want.shape == (n_chan, n_pol, n_pad, n_pad)
    for c in range(n_chan):
        for p in range(n_pol):
            assert np.linalg.norm(img[c, p] - want[c, p]) / np.linalg.norm(want[c, p]) < 1e-4, (c, p)
            assert np.abs(img[c, p] - want[c, p]).max() < 1e-4 * np.abs(want[c, p]).max(), (c, p)


@pytest.mark.parametrize("n_ant, n_time, n_chan, n_pol", [
    (256, 40, 52, 2),     # 312 units: two per SM and 8 left over (two chunks)
    (200, 70, 51, 1),     # 153 units: one left over, a ragged 70-sample K, a 72-antenna tail block
])
def test_units_not_dividing_over_the_sms(epic, n_ant, n_time, n_chan, n_pol):
    """Unit counts that leave some SMs one unit more than others, 4+4-bit voltages with gains:
    every matrix against the oracle, and a second call on the same plan gives the same bits."""
    wl = _small(n_ant, n_time, n_chan, n_pol, "ci4", seed=n_ant + n_chan)
    g = synth.random_gains(np.random.default_rng(n_time), (n_chan, n_pol, n_ant))
    plan, vis = run(epic, wl, g)
    check(vis, wl, g, "A=%d C=%d" % (n_ant, n_chan))
    g2 = torch.from_numpy(np.ascontiguousarray(g.astype(np.complex64))).cuda()
    vis2 = plan.correlate(torch.from_numpy(np.ascontiguousarray(wl.volt_raw)).cuda(), g2)
    torch.cuda.synchronize()
    assert np.array_equal(vis2.cpu().numpy(), vis)


def test_longest_integration_reaches_2_to_24(epic):
    """n_time = 131072, the most a call accepts: with every 4+4-bit voltage at -8 - 8i each
    sample adds (-8 - 8i)(-8 + 8i) = 128 to every pair's sum, which reaches 128 x 131072 = 2^24,
    the top of the exact FP32 integer range; every visibility must be exactly 128 + 0i (2^24
    scaled by 1/T = 2^-17 is exact).  One sample more is refused before any launch."""
    wl = _small(16, 4, 1, 1, "ci4", seed=3)
    plan = epic.Plan.from_workload(wl)
    T = 131072
    raw = torch.full((T, 1, 1, 16), 0x88, dtype=torch.uint8, device="cuda")
    vis = plan.correlate(raw).cpu().numpy()
    assert np.array_equal(vis, np.full((1, 1, 16, 16), 128 + 0j, dtype=np.complex64))
    with pytest.raises(epic.EpicError) as e:
        plan.correlate(torch.full((T + 1, 1, 1, 16), 0x88, dtype=torch.uint8, device="cuda"))
    assert e.value.status == epic.EPIC_EUNSUPPORTED
