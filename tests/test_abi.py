"""The C ABI without a GPU: the library builds, loads, exports every symbol declared in
include/epic.h, and rejects bad arguments on the host before touching CUDA."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_1510_08318_gb300 import build, epic

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    build.build()
    return epic.load()


def _declared():
    names = set()
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            src = open(os.path.join(ROOT, "include", f)).read()
            names |= set(re.findall(r"\b(epic_[a-z_0-9]+)\s*\(", src))
    return names


def _enum_values(prefix):
    """Name -> value of the header's enumerators that start with prefix (explicit or implicit)."""
    src = open(os.path.join(ROOT, "include", "epic.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    out = {}
    for body in re.findall(r"typedef\s+enum\s*\{(.*?)\}", src, flags=re.S):
        nxt = 0
        for item in body.split(","):
            m = re.match(r"\s*(\w+)\s*(?:=\s*(-?\d+))?\s*$", item)
            if not m:
                continue
            nxt = int(m.group(2)) if m.group(2) is not None else nxt
            if m.group(1).startswith(prefix):
                out[m.group(1)] = nxt
            nxt += 1
    return out


def test_binding_constants_match_the_header():
    """The binding's transform codes and status codes are the header's enumerators."""
    xf = _enum_values("EPIC_XFORM_")
    assert xf, "no EPIC_XFORM_ enumerators found"
    for name, value in xf.items():
        assert getattr(epic, name[len("EPIC_"):]) == value, name
    assert sorted(epic.XFORMS.values()) == sorted(xf.values())
    st = _enum_values("EPIC_E") | _enum_values("EPIC_OK")
    for name, value in st.items():
        assert getattr(epic, name) == value, name


def test_exports_every_declared_symbol(lib):
    declared = _declared()
    assert {"epic_create", "epic_image", "epic_image_backward", "epic_destroy"} <= declared
    for name in declared:
        assert hasattr(lib, name), name
    assert set(epic.SYMBOLS) <= declared


def _create(**kw):
    args = dict(n_ant=2, pos_xy=np.array([[0.0, 0.0], [3.0, 1.0]]), kern_ptr=np.array([0, 1, 2]),
                kern_dxdy=np.zeros((2, 2)), kern_w=np.ones(2, dtype=np.complex128), dx=1.0,
                origin_xy=np.array([-2.0, -2.0]), n_grid=8, n_pad=16, n_chan=1, n_pol=1, volt_dtype=0, device=0)
    args.update(kw)
    return epic.epic_create(**args)


@pytest.mark.parametrize("kw, status", [
    (dict(n_pad=16), epic.EPIC_EUNSUPPORTED),                       # unsupported padded size
    (dict(n_pad=64, n_grid=33), epic.EPIC_EINVAL),                  # less than 2x padding
    (dict(n_pad=64, n_grid=0), epic.EPIC_EINVAL),
    (dict(n_pad=64, n_ant=0), epic.EPIC_EINVAL),
    (dict(n_pad=64, dx=0.0), epic.EPIC_EINVAL),
    (dict(n_pad=64, dx=float("nan")), epic.EPIC_EINVAL),
    (dict(n_pad=64, volt_dtype=7), epic.EPIC_EINVAL),
    (dict(n_pad=64, n_chan=0), epic.EPIC_EINVAL),
    (dict(n_pad=64, kern_ptr=np.array([1, 1, 2])), epic.EPIC_EINVAL),
    (dict(n_pad=64, kern_ptr=np.array([0, 2, 1])), epic.EPIC_EINVAL),
    (dict(n_pad=64, pos_xy=np.array([[0.0, 0.0], [40.0, 1.0]])), epic.EPIC_EINVAL),   # off the grid
    (dict(n_pad=64, pos_xy=np.array([[0.0, np.inf], [3.0, 1.0]])), epic.EPIC_EINVAL),
    (dict(n_pad=64, n_ant=5000, pos_xy=np.zeros((5000, 2)), kern_ptr=np.zeros(5001, dtype=np.int32)),
     epic.EPIC_EINVAL),
])
def test_create_rejects(lib, kw, status):
    with pytest.raises(epic.EpicError) as e:
        _create(**kw)
    assert e.value.status == status
    assert epic.epic_last_error()


def test_calls_reject_null_plan(lib):
    assert lib.epic_image(None, None, 1, None, None, None, 0, None, None, None) == epic.EPIC_EINVAL
    assert "plan" in epic.epic_last_error()
    assert lib.epic_image_backward(None, None, 1, None, None, None, None) == epic.EPIC_EINVAL
    assert lib.epic_grid(None, None, 1, None, None, None) == epic.EPIC_EINVAL
    assert lib.epic_plan_info(None, None, None, None) == epic.EPIC_EINVAL
    lib.epic_destroy(None)


def test_every_plan_call_rejects_null_plan(lib):
    """Every call that takes a plan or a batch checks it on the host before any CUDA call."""
    plan_calls = {
        "epic_image_xpol": (None, None, 1, None, None, 0, None, None, None),
        "epic_correlate": (None, None, 1, None, None, None),
        "epic_fx_image": (None, None, None, None),
        "epic_weff": (None, None, None),
        "epic_isotropic": (None, None, None, None, 0.05, None, None),
        "epic_set_transform": (None, 0),
    }
    for name, args in plan_calls.items():
        assert getattr(lib, name)(*args) == epic.EPIC_EINVAL, name
        assert "plan" in epic.epic_last_error(), name
    assert lib.epic_batch_image(None, None, None, None, None, None, None) == epic.EPIC_EINVAL
    assert lib.epic_batch_autotune(None, None, None, None, None, None) == epic.EPIC_EINVAL
    assert lib.epic_batch_info(None, None, None, None, 0) == epic.EPIC_EINVAL
    assert "batch" in epic.epic_last_error()
    assert lib.epic_sync(None, None) == epic.EPIC_EINVAL
    assert "plan" in epic.epic_last_error()
    assert lib.epic_set_wait_limit(None, 10) == epic.EPIC_EINVAL
    assert lib.epic_batch_create(None, 1, None) == epic.EPIC_EINVAL
    out = ctypes.c_void_p(1)
    assert lib.epic_batch_create(ctypes.byref(out), 0, None) == epic.EPIC_EINVAL
    assert out.value is None                       # the out-pointer is cleared on failure
    lib.epic_batch_destroy(None)


@pytest.mark.parametrize("args, status", [
    ((0, 2, 128, 4, 2, None, 1, None, 0, None), epic.EPIC_EINVAL),           # no antennas
    ((8, 2, 100, 4, 2, None, 1, None, 0, None), epic.EPIC_EUNSUPPORTED),     # 100 channels
    ((8, 2, 128, 4, 5, None, 1, None, 0, None), epic.EPIC_EINVAL),           # unknown input format
    ((8, 2, 128, 4, 2, None, 2, None, 0, None), epic.EPIC_EINVAL),           # 4+4-bit output
    ((8, 2, 128, 4, 2, None, 1, None, 0, None), epic.EPIC_EINVAL),           # NULL arrays
])
def test_fengine_rejects_on_host(lib, args, status):
    assert lib.epic_fengine(*args) == status
    assert epic.epic_last_error()


def test_fengine_zero_blocks_is_a_no_op(lib):
    assert lib.epic_fengine(8, 2, 128, 0, 2, None, 1, None, 0, None) == epic.EPIC_OK


@pytest.mark.parametrize("in_dtype, raw, out_dtype, volt", [
    (0, 0x1004, 1, 0x2000),       # complex64 samples at a 4-byte offset
    (1, 0x1002, 1, 0x2000),       # FP16 pairs at a 2-byte offset
    (2, 0x1001, 0, 0x2004),       # 4+4-bit samples anywhere, complex64 spectra at a 4-byte offset
])
def test_fengine_rejects_misaligned_arrays_on_host(lib, in_dtype, raw, out_dtype, volt):
    """The alignment of every device array is checked on the host before any CUDA call (the
    addresses here are never dereferenced)."""
    assert lib.epic_fengine(8, 2, 128, 4, in_dtype, raw, out_dtype, volt, 0, None) == epic.EPIC_EINVAL
    assert "aligned" in epic.epic_last_error()
