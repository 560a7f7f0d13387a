"""Host logic of the tensor-core kernel's gridding (no GPU): the slot tables built by the
library's own builder, walked as the kernel's warps walk them, on the mappings of the LWA-like
layout and of small layouts with complex weights, a ragged grid and many antennas (the mappings
come from the oracle's nearest-cell rule).  The checker is compiled from the kernel's source with
nvcc; see tests/host/gather_tables_check.cu for what it checks."""
import os
import shutil
import subprocess

import numpy as np
import pytest

from oracle import moff
from paper_1510_08318_gb300 import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
NVCC = shutil.which("nvcc") or ("/usr/local/cuda/bin/nvcc" if os.path.exists("/usr/local/cuda/bin/nvcc") else None)


def _layout(n_grid, n_ant, seed, complex_w):
    rng = np.random.default_rng(seed)
    pos = rng.uniform(1.5, n_grid - 2.5, (n_ant, 2))
    kerns = [synth.kernel_square(rng.uniform(0.5, 2.5), 1 / 3) for _ in range(n_ant)]
    ptr, dxdy, w = synth.pack_kernels(kerns)
    if complex_w:
        w = w * np.exp(1j * rng.uniform(0, 2 * np.pi, w.shape))
    return moff.map_antennas(pos, ptr, dxdy, w, 1.0, np.zeros(2), n_grid)


def _write_csr(M, n_grid, path, side=64):
    """The mapping as the library holds it: cell-major over the side x side grid of N_p = 2 side."""
    M = M.tocsr()
    M.sort_indices()
    rows = np.repeat(np.arange(M.shape[0]), np.diff(M.indptr))
    cell = (rows // n_grid) * side + rows % n_grid
    order = np.argsort(cell, kind="stable")
    ptr = np.zeros(side * side + 1, dtype=np.int64)
    np.add.at(ptr, cell + 1, 1)
    ptr = np.cumsum(ptr)
    with open(path, "w") as f:
        f.write("%d %d\n" % (side * side, M.nnz))
        f.write(" ".join(map(str, ptr)) + "\n")
        f.write(" ".join(map(str, M.indices[order])) + "\n")
        f.write(" ".join("%.9g" % v for v in np.float32(M.data.real[order])) + "\n")
        f.write(" ".join("%.9g" % v for v in np.float32(M.data.imag[order])) + "\n")


@pytest.fixture(scope="module")
def checker(tmp_path_factory):
    if NVCC is None:
        pytest.skip("nvcc not available")
    out = str(tmp_path_factory.mktemp("gt") / "gather_tables_check")
    cmd = [NVCC, "-std=c++17", "--expt-relaxed-constexpr", "-gencode", "arch=compute_103a,code=sm_103a",
           "-o", out, os.path.join(ROOT, "tests", "host", "gather_tables_check.cu")]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr[-2000:]
    return out


@pytest.mark.parametrize("case", ["lwa", "complex_weights", "ragged_grid", "many_antennas"])
def test_gather_tables(checker, tmp_path, case):
    if case == "lwa":
        wl = synth.workload_lwa(n_chan=1, n_time=1, chan_index=[0])
        M, n_grid = moff.map_antennas(wl.pos, wl.kern_ptr, wl.kern_dxdy, wl.kern_w, wl.dx, wl.origin,
                                      wl.n_grid), wl.n_grid
    elif case == "complex_weights":
        n_grid = 64
        M = _layout(n_grid, 40, 11, True)
    elif case == "ragged_grid":
        n_grid = 37
        M = _layout(n_grid, 300, 12, False)
    else:
        n_grid = 64
        M = _layout(n_grid, 1500, 13, True)
    path = str(tmp_path / "map.txt")
    _write_csr(M, n_grid, path)
    r = subprocess.run([checker, path], capture_output=True, text=True)
    assert r.returncode == 0, r.stdout + r.stderr


@pytest.mark.parametrize("case", ["hera", "complex_ragged", "calib"])
def test_gather_tables_np256(checker, tmp_path, case):
    """The N_p = 256 form's tables: 128 x 128 grid, 256 slots over its 15 gridding warps."""
    if case == "hera":
        wl = synth.workload_hera(n_chan=1, n_time=1)
        M, n_grid = moff.map_antennas(wl.pos, wl.kern_ptr, wl.kern_dxdy, wl.kern_w, wl.dx, wl.origin,
                                      wl.n_grid), wl.n_grid
    elif case == "complex_ragged":
        n_grid = 101
        M = _layout(n_grid, 200, 14, True)
    else:
        wl = synth.workload_calib(n_chan=1, n_time=1)
        M, n_grid = moff.map_antennas(wl.pos, wl.kern_ptr, wl.kern_dxdy, wl.kern_w, wl.dx, wl.origin,
                                      wl.n_grid), wl.n_grid
    path = str(tmp_path / "map.txt")
    _write_csr(M, n_grid, path, side=128)
    r = subprocess.run([checker, path, "15"], capture_output=True, text=True)
    assert r.returncode == 0, r.stdout + r.stderr
