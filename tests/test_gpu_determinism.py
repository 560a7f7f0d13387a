"""Bitwise determinism of the paths that sum without atomics (GPU only): the same call twice on
the same inputs gives the same bits.  The gridder (one cell's entries summed in a fixed order by
one thread), the F-engine (register and shared-memory FFTs), the X-engine (tensor-core sums of
each block by one CTA) and the FX imaging (each lag cell summed by one warp in table order, one
CTA per transform).  The imaging accumulators are not in this list: their FP64 atomic flushes
from several CTAs may land in any order (differences at the FP64 rounding level)."""
import numpy as np
import pytest

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


@pytest.fixture(scope="module")
def lwa(epic):
    wl = synth.workload_lwa(n_chan=4, n_time=96, chan_index=[0, 40, 80, 127])
    plan = epic.Plan.from_workload(wl)
    volt = torch.from_numpy(np.ascontiguousarray(wl.volt_raw)).cuda()
    gains = torch.from_numpy(np.ascontiguousarray(
        synth.random_gains(np.random.default_rng(5), (wl.n_chan, wl.n_pol, wl.n_ant)).astype(np.complex64))).cuda()
    return wl, plan, volt, gains


def _same_bits(a, b):
    a, b = a.contiguous().view(torch.uint8), b.contiguous().view(torch.uint8)
    return bool(torch.equal(a, b))


def test_gridder_bits(epic, lwa):
    wl, plan, volt, gains = lwa
    g1 = plan.grid(volt, gains).clone()
    g2 = plan.grid(volt, gains)
    torch.cuda.synchronize()
    assert _same_bits(g1, g2)


def test_correlator_and_fx_imaging_bits(epic, lwa):
    wl, plan, volt, gains = lwa
    v1 = plan.correlate(volt, gains).clone()
    v2 = plan.correlate(volt, gains)
    torch.cuda.synchronize()
    assert _same_bits(v1, v2)
    i1 = plan.fx_image(v1).clone()
    i2 = plan.fx_image(v2)
    torch.cuda.synchronize()
    assert _same_bits(i1, i2)


def test_fengine_bits(epic):
    rng = np.random.default_rng(7)
    raw = torch.from_numpy(rng.integers(0, 256, (128 * 24, 2, 256), dtype=np.uint8)).cuda()
    s1 = epic.fengine(raw, 128, "ci4", "f16").clone()
    s2 = epic.fengine(raw, 128, "ci4", "f16")
    torch.cuda.synchronize()
    assert _same_bits(s1, s2)
