"""F-engine (epic_fengine) vs the FP64 oracle's spectra, and the F-engine -> imaging chain
(GPU only).

Tolerances: complex64 spectra are float32 FFTs of at most log2(512) = 9 stages: 1e-6
relative L2 per block set; FP16 spectra are additionally rounded to 11 bits: 1e-3.  The
chained image carries the imaging path's 1e-4 bound.
"""
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


def raw_samples(rng, n, P, A, dtype):
    """Seeded random time samples in the given format: (device tensor, decoded complex128)."""
    v = rng.standard_normal((n, P, A)) + 1j * rng.standard_normal((n, P, A))
    if dtype == "ci4":
        b, _ = synth.quantize_ci4(v)
        return torch.from_numpy(b).cuda(), synth.decode_ci4(b)
    if dtype == "f16":
        x = synth.to_f16_pairs(v)
        return torch.from_numpy(x).cuda(), synth.from_f16_pairs(x)
    x = v.astype(np.complex64)
    return torch.from_numpy(x).cuda(), x.astype(np.complex128)


@pytest.mark.parametrize("C", [32, 64, 128, 256, 512])
@pytest.mark.parametrize("dtype", ["c64", "f16", "ci4"])
@pytest.mark.parametrize("A", [33, 66])
def test_spectra_match_oracle(epic, C, dtype, A):
    """A = 33: one antenna per thread, a ragged 32-antenna tile; A = 66 (C <= 128): two antennas
    per thread in packed pairs, a ragged 64-antenna tile."""
    rng = np.random.default_rng(C + A)
    T, P = 3, 2
    raw, dec = raw_samples(rng, T * C, P, A, dtype)
    want = moff.fengine(dec, C)
    got = epic.fengine(raw, C, dtype, "c64").cpu().numpy()
    assert np.linalg.norm(got - want) / np.linalg.norm(want) < 1e-6, (C, dtype)
    g16 = epic.fengine(raw, C, dtype, "f16").cpu().numpy().astype(np.float64)
    g16 = g16[..., 0] + 1j * g16[..., 1]
    assert np.linalg.norm(g16 - want) / np.linalg.norm(want) < 1e-3, (C, dtype)


def test_pure_tone(epic):
    """x_j = exp(+2 pi i 7 j / 128) in every antenna: bin 7 holds 128, the others ~0."""
    C, T, A = 128, 2, 40
    j = np.arange(T * C)
    tone = np.exp(2j * np.pi * 7 * j / C)[:, None, None] * np.ones((1, 1, A))
    V = epic.fengine(torch.from_numpy(tone.astype(np.complex64)).cuda(), C, "c64", "c64").cpu().numpy()
    assert np.allclose(V[:, 7], 128, atol=1e-3)
    assert np.abs(np.delete(V, 7, axis=1)).max() < 1e-3


def test_fengine_then_image(epic):
    """Raw 4+4-bit time samples -> F-engine (complex64) -> epic_image: the image equals the
    oracle's image of the oracle's spectra of the same samples."""
    rng = np.random.default_rng(9)
    C, T, P = 64, 12, 1
    wl0 = synth.workload_tiny(n_time=2)
    A = wl0.n_ant
    raw, dec = raw_samples(rng, T * C, P, A, "ci4")
    V = epic.fengine(raw, C, "ci4", "c64")
    plan = epic.Plan(wl0.pos, wl0.kern_ptr, wl0.kern_dxdy, wl0.kern_w, wl0.dx, wl0.origin, wl0.n_grid, wl0.n_pad,
                     C, P, "c64")
    img = plan.image(V)["image"].cpu().numpy()
    M = moff.map_antennas(wl0.pos, wl0.kern_ptr, wl0.kern_dxdy, wl0.kern_w, wl0.dx, wl0.origin, wl0.n_grid)
    want = moff.moff_image(M, moff.fengine(dec, C), None, wl0.n_grid, wl0.n_pad)
    assert np.linalg.norm(img - want) / np.linalg.norm(want) < 1e-4
    assert np.abs(img - want).max() < 1e-4 * want.max()


def test_rejects_unsupported(epic):
    raw = torch.zeros((100, 1, 4), dtype=torch.complex64, device="cuda")
    with pytest.raises(epic.EpicError):
        epic.epic_fengine(4, 1, 100, 1, 0, raw.data_ptr(), 0, raw.data_ptr(), 0, None)
    with pytest.raises(epic.EpicError):
        epic.epic_fengine(4, 1, 64, 1, 0, raw.data_ptr(), 2, raw.data_ptr(), 0, None)
