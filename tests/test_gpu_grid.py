"""Standalone gridder (epic_grid) vs the FP64 oracle's gridding step, element by element
(GPU only).

Tolerance: every gridded value is a float32 sum of at most a few hundred products of
float32-rounded weights and decoded voltages, so its error is a few float32 ulps of the
magnitudes summed; the bound is 1e-5 of each grid's peak per element and 1e-5 relative L2
per call.
"""
import numpy as np
import pytest

from oracle import moff
from paper_1510_08318_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-5


@pytest.fixture(scope="module")
def epic():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1510_08318_gb300 import build, epic as ep
    build.build()
    ep.load()
    return ep


def oracle_grid(wl, gains=None, t_index=None, cp_index=None):
    """E_t(g) of the oracle, [T, C, P, N_g, N_g] (optionally a subset of samples / (c, p))."""
    M = moff.map_antennas(wl.pos, wl.kern_ptr, wl.kern_dxdy, wl.kern_w, wl.dx, wl.origin, wl.n_grid)
    T, C, P = wl.volt.shape[:3]
    ts = range(T) if t_index is None else t_index
    cps = [(c, p) for c in range(C) for p in range(P)] if cp_index is None else cp_index
    out = {}
    for c, p in cps:
        g = np.ones(wl.n_ant) if gains is None else gains[c, p].astype(np.complex128)
        out[(c, p)] = moff.grid_efields(M, wl.volt[list(ts), c, p, :], g, wl.n_grid)
    return M, out


def check(got, want, what):
    got = np.asarray(got, np.complex128)
    peak = np.abs(want).max()
    assert peak > 0, what
    worst = np.abs(got - want).max() / peak
    rel = np.linalg.norm(got - want) / np.linalg.norm(want)
    assert worst < TOL, "%s: worst element %.3e of peak" % (what, worst)
    assert rel < TOL, "%s: relative L2 %.3e" % (what, rel)


def run(epic, wl, gains=None):
    plan = epic.Plan.from_workload(wl)
    g = None if gains is None else torch.from_numpy(np.ascontiguousarray(gains.astype(np.complex64))).cuda()
    E = plan.grid(torch.from_numpy(np.ascontiguousarray(wl.volt_raw)).cuda(), g)
    torch.cuda.synchronize()
    return plan, E.cpu().numpy()


def test_tiny_ragged_time_blocks(epic):
    """16 antennas, complex64, 21 samples: one full block of 16 samples and a ragged one."""
    wl = synth.workload_tiny(n_time=21)
    plan, E = run(epic, wl)
    M, want = oracle_grid(wl)
    assert plan.info["nnz"] == M.nnz
    assert E.shape == (21, 1, 1, wl.n_grid, wl.n_grid)
    check(E[:, 0, 0], want[(0, 0)], "tiny")


def test_lwa_slice_ci4_gains(epic):
    """LWA-like layout, 4+4-bit voltages, two channels, two pols, 21 samples, random gains."""
    wl = synth.workload_lwa(n_chan=2, n_time=21, chan_index=[0, 127])
    g = synth.random_gains(np.random.default_rng(8), (wl.n_chan, wl.n_pol, wl.n_ant))
    _, E = run(epic, wl, g)
    _, want = oracle_grid(wl, g)
    for (c, p), w in want.items():
        check(E[:, c, p], w, "lwa c=%d p=%d" % (c, p))


def test_hera_slice_f16(epic):
    """331-antenna hexagon with 14 m disks (49-cell footprints), FP16, 5 samples (< one block)."""
    wl = synth.workload_hera(n_chan=2, n_time=5)
    _, E = run(epic, wl)
    _, want = oracle_grid(wl)
    for (c, p), w in want.items():
        check(E[:, c, p], w, "hera c=%d" % c)


def _small(n_pad, n_grid, n_ant, n_time, n_chan, n_pol, vdtype, seed):
    rng = np.random.default_rng(seed)
    dx = 1.0
    pos = rng.uniform(1.5 * dx, (n_grid - 2.5) * dx, (n_ant, 2))
    kerns = [synth.kernel_square(rng.uniform(0.5, 2.5) * dx, dx / 3) for _ in range(n_ant)]
    ptr, dxdy, w = synth.pack_kernels(kerns)
    w = w * np.exp(1j * rng.uniform(0, 2 * np.pi, w.shape))     # complex weights
    wl = synth.Workload("small", pos, ptr, dxdy, w, dx, np.zeros(2), n_grid, n_pad,
                        np.full(n_chan, 1e8), n_pol, n_time, vdtype)
    v = (rng.standard_normal((n_time, n_chan, n_pol, n_ant))
         + 1j * rng.standard_normal((n_time, n_chan, n_pol, n_ant)))
    return synth._finish(wl, v, vdtype)


@pytest.mark.parametrize("n_pad, n_grid, n_ant, n_time, n_chan, n_pol, vdtype", [
    (32, 11, 40, 33, 1, 1, "f16"),      # unpadded grid smaller than N_p / 2
    (64, 20, 300, 17, 2, 1, "ci4"),     # ragged grid and time blocks
    (128, 64, 700, 9, 1, 2, "c64"),     # A > threads per CTA
    (512, 256, 12, 2, 1, 1, "f16"),     # full 256 x 256 grid
    (64, 32, 1000, 11, 1, 1, "ci4"),    # 8-sample blocks
    (64, 32, 4096, 9, 1, 1, "c64"),     # largest antenna count: 4-sample blocks
])
def test_small_sizes_complex_weights(epic, n_pad, n_grid, n_ant, n_time, n_chan, n_pol, vdtype):
    wl = _small(n_pad, n_grid, n_ant, n_time, n_chan, n_pol, vdtype, seed=n_pad + n_ant)
    g = synth.random_gains(np.random.default_rng(n_ant), (n_chan, n_pol, n_ant))
    _, E = run(epic, wl, g)
    _, want = oracle_grid(wl, g)
    for (c, p), w in want.items():
        check(E[:, c, p], w, "c=%d p=%d" % (c, p))


def test_one_cell_grid(epic):
    """N_g = 1: every footprint sample of three antennas lands in the single cell, so the
    grid is sum_a (sum_k w_ak) g_a V_a(t)."""
    rng = np.random.default_rng(3)
    kerns = [synth.kernel_square(0.4, 0.2) for _ in range(3)]
    ptr, dxdy, w = synth.pack_kernels(kerns)
    wl = synth.Workload("one-cell", np.zeros((3, 2)), ptr, dxdy, w, 1.0, np.zeros(2), 1, 64,
                        np.full(1, 1e8), 1, 2, "c64")
    v = rng.standard_normal((2, 1, 1, 3)) + 1j * rng.standard_normal((2, 1, 1, 3))
    wl = synth._finish(wl, v, "c64")
    _, E = run(epic, wl)
    wsum = np.array([w[ptr[a]:ptr[a + 1]].sum() for a in range(3)])
    check(E[:, 0, 0, 0, 0], wl.volt[:, 0, 0, :] @ wsum, "one cell")


def test_zero_gains_give_zero_grid(epic):
    wl = synth.workload_tiny(n_time=3)
    _, E = run(epic, wl, np.zeros((1, 1, wl.n_ant), np.complex64))
    assert not np.any(E)


def test_matches_the_imaging_step(epic):
    """Property at any size: the time average of |FFT(zero-padded E_t)|^2 of the gridded
    fields equals epic_image's image (shifted), tying the two entry points together."""
    wl = synth.workload_lwa(n_chan=1, n_time=16, chan_index=[64])
    plan, E = run(epic, wl)
    img = plan.image(torch.from_numpy(np.ascontiguousarray(wl.volt_raw)).cuda())["image"].cpu().numpy()
    Ep = np.zeros(E.shape[:3] + (wl.n_pad, wl.n_pad), np.complex128)
    Ep[..., :wl.n_grid, :wl.n_grid] = E
    F = np.fft.ifft2(Ep) * wl.n_pad ** 2          # unnormalised exp(+2 pi i g.k / N_p)
    want = moff.fftshift2((np.abs(F) ** 2).mean(0))
    rel = np.linalg.norm(img - want) / np.linalg.norm(want)
    assert rel < 1e-4, rel


def test_rejects_misaligned_and_null(epic):
    wl = synth.workload_tiny(n_time=2)
    plan = epic.Plan.from_workload(wl)
    v = torch.from_numpy(np.ascontiguousarray(wl.volt_raw)).cuda()
    out = torch.empty(4 * wl.n_grid * wl.n_grid + 4, dtype=torch.float32, device="cuda")
    st = torch.cuda.current_stream().cuda_stream
    with pytest.raises(epic.EpicError):
        epic.epic_grid(plan._h, v.data_ptr(), 2, None, out.data_ptr() + 4, st)
    with pytest.raises(epic.EpicError):
        epic.epic_grid(plan._h, v.data_ptr(), 2, None, None, st)
    with pytest.raises(epic.EpicError):
        epic.epic_grid(plan._h, v.data_ptr(), 0, None, out.data_ptr(), st)


def test_full_lwa_workload_sampled(epic):
    """The full LWA-like call (128 channels x 2 pols x 1024 samples, 8.6 GB of grids) in the
    launch the bench times; sampled (t, c, p) grids against the oracle."""
    wl = synth.workload_lwa()
    cps, ts = [(0, 0), (63, 1), (127, 0)], [0, 517, 1023]
    plan = epic.Plan.from_workload(wl)
    E = plan.grid(torch.from_numpy(np.ascontiguousarray(wl.volt_raw)).cuda())
    torch.cuda.synchronize()
    _, want = oracle_grid(wl, t_index=ts, cp_index=cps)
    for (c, p), w in want.items():
        got = E[ts, c, p].cpu().numpy()
        check(got, w, "full c=%d p=%d" % (c, p))
    del E
    torch.cuda.empty_cache()
