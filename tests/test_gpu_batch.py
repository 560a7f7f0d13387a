"""Batching form (GPU only): 64 heterogeneous sub-arrays (N_p from 32 to 512, mixed square,
Gaussian and disk apertures per antenna, uneven antenna and channel counts) imaged by one
launch per size class, checked against per-plan calls and, on the smallest sub-array of each
size class, against the FP64 oracle; then captured and replayed as one CUDA graph, and
autotuned."""
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


@pytest.fixture(scope="module")
def setup(epic):
    # the batching configuration's 128 samples per sub-array (channels capped at 3 to keep the
    # oracle checks short)
    subs = synth.workload_batch(n_time=128, max_chan=3)
    plans = [epic.Plan.from_workload(w) for w in subs]
    volts = [torch.from_numpy(np.ascontiguousarray(w.volt_raw)).cuda() for w in subs]
    batch = epic.Batch(plans)
    return subs, plans, volts, batch


def rel(a, b):
    a, b = np.asarray(a, np.float64), np.asarray(b, np.float64)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def test_batch_matches_single_plans(epic, setup):
    subs, plans, volts, batch = setup
    acc, img = batch.alloc()
    batch.image(volts, acc, img)
    torch.cuda.synchronize()
    assert batch.info()["n_classes"] == len({w.n_pad for w in subs})
    for p, v, got in zip(plans, volts, img):
        ref = p.image(v)["image"]
        torch.cuda.synchronize()
        assert rel(got.cpu().numpy(), ref.cpu().numpy()) < 1e-6


def test_batch_against_oracle(epic, setup):
    subs, plans, volts, batch = setup
    acc, img = batch.alloc()
    batch.image(volts, acc, img)
    torch.cuda.synchronize()
    checked = set()
    for i in np.argsort([w.n_ant * w.kern_dxdy.shape[0] for w in subs]):
        w = subs[i]
        if w.n_pad in checked:
            continue
        checked.add(w.n_pad)
        M = moff.map_antennas(w.pos, w.kern_ptr, w.kern_dxdy, w.kern_w, w.dx, w.origin, w.n_grid)
        assert plans[i].info["nnz"] == M.nnz
        want = moff.moff_image(M, w.volt[:, :1], None, w.n_grid, w.n_pad)[0, 0]
        got = img[i].cpu().numpy()[0, 0]
        assert rel(got, want) < 1e-4, (w.name, rel(got, want))
        assert np.abs(got - want).max() < 1e-4 * want.max()
    assert checked == {32, 64, 128, 256, 512}


def test_batch_graph_capture_and_autotune(epic, setup):
    subs, plans, volts, batch = setup
    acc, img = batch.alloc()
    batch.image(volts, acc, img)          # eager reference (also warms every launch path)
    torch.cuda.synchronize()
    ref = [x.cpu().numpy() for x in img]
    acc2, img2 = batch.alloc()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    g = torch.cuda.CUDAGraph()
    with torch.cuda.stream(s):
        with torch.cuda.graph(g, stream=s):
            batch.image(volts, acc2, img2)
    for _ in range(2):
        g.replay()
    torch.cuda.synchronize()
    for a, b in zip(ref, img2):
        assert rel(b.cpu().numpy(), a) < 1e-6
    info = batch.autotune(volts, acc)
    assert info["n_classes"] == len(info["workers"]) == len(info["classes"])
    for c in info["classes"]:
        assert (c["form"] == "persistent" or (c["form"] == "two-pass" and c["n_pad"] == 512)
                or (c["form"] == "persistent, one buffer" and c["n_pad"] == 256))
    batch.image(volts, acc, img)
    torch.cuda.synchronize()
    for a, b in zip(ref, img):
        assert rel(b.cpu().numpy(), a) < 1e-6


def test_batch_rejects_mixed_formats(epic):
    a = synth.workload_tiny(n_time=2)
    b = synth.workload_lwa(n_chan=1, n_time=2, chan_index=[0])
    pa, pb = epic.Plan.from_workload(a), epic.Plan.from_workload(b)
    with pytest.raises(epic.EpicError):
        epic.Batch([pa, pb])


def test_batch_full_configuration(epic):
    """The batching configuration at full size, as the bench runs it (64 sub-arrays with their
    full channel counts, 8 to 256, T = 128): autotuned and replayed as one CUDA graph, every
    sub-array's images equal its per-plan call (1e-6), and one channel of the smallest sub-array
    of each size class against the oracle."""
    subs = synth.workload_batch(n_time=128)
    plans = [epic.Plan.from_workload(w) for w in subs]
    volts = [torch.from_numpy(np.ascontiguousarray(w.volt_raw)).cuda() for w in subs]
    batch = epic.Batch(plans)
    acc, img = batch.alloc()
    batch.autotune(volts, acc)
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    g = torch.cuda.CUDAGraph()
    with torch.cuda.stream(s):
        with torch.cuda.graph(g, stream=s):
            batch.image(volts, acc, img)
    g.replay()
    torch.cuda.synchronize()
    for p, v, got in zip(plans, volts, img):
        ref = p.image(v)["image"]
        torch.cuda.synchronize()
        assert rel(got.cpu().numpy(), ref.cpu().numpy()) < 1e-6
    checked = set()
    for i in np.argsort([w.n_ant * w.kern_dxdy.shape[0] for w in subs]):
        w = subs[i]
        if w.n_pad in checked:
            continue
        checked.add(w.n_pad)
        c = w.n_chan - 1
        M = moff.map_antennas(w.pos, w.kern_ptr, w.kern_dxdy, w.kern_w, w.dx, w.origin, w.n_grid)
        want = moff.moff_image(M, w.volt[:, c:c + 1, :1], None, w.n_grid, w.n_pad)[0, 0]
        got = img[i][c, 0].cpu().numpy()
        assert rel(got, want) < 1e-4, (w.name, rel(got, want))
        assert np.abs(got - want).max() < 1e-4 * want.max()
    assert checked == {32, 64, 128, 256, 512}
