"""Thin Python binding of the MOFF imaging C ABI (include/epic.h).

The functions named like the C entry points (`epic_create`, `epic_image`,
`epic_image_backward`, `epic_image_xpol`, `epic_correlate`, `epic_weff`, `epic_isotropic`,
`epic_fengine`, `epic_fx_image`, `epic_grid`, `epic_sync`, `epic_set_wait_limit`,
`epic_destroy`, `epic_plan_info`, `epic_last_error`) only marshal arguments; every step of the imaging path runs in the CUDA library.  `Plan` wraps them
for torch tensors, and `MoffImage` is the autograd.Function whose backward is the
library's adjoint kernel.  There is no CPU fallback: if the library has not been built
(paper_1510_08318_gb300.build), loading raises.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libepic.so")

EPIC_OK, EPIC_EINVAL, EPIC_ENOMEM, EPIC_ECUDA, EPIC_EUNSUPPORTED, EPIC_ETIMEOUT = range(6)
VOLT_DTYPES = {"c64": 0, "f16": 1, "ci4": 2}
SYMBOLS = ("epic_create", "epic_destroy", "epic_image", "epic_image_backward", "epic_plan_info",
           "epic_last_error", "epic_set_transform", "epic_batch_create", "epic_batch_image",
           "epic_batch_autotune", "epic_batch_info", "epic_batch_destroy", "epic_grid", "epic_image_xpol", "epic_correlate", "epic_weff", "epic_isotropic", "epic_fengine", "epic_fx_image",
           "epic_sync", "epic_set_wait_limit", "epic_batch_class", "epic_image_noalloc")
XFORM_FFT, XFORM_DFTGEMM, XFORM_DFTGEMM_FP16, XFORM_FFT_TWOPASS, XFORM_DFTGEMM_FP16_GRID = 0, 1, 2, 3, 4
XFORMS = {"fft": XFORM_FFT, "dftgemm": XFORM_DFTGEMM, "dftgemm_fp16": XFORM_DFTGEMM_FP16,
          "fft_twopass": XFORM_FFT_TWOPASS, "dftgemm_fp16grid": XFORM_DFTGEMM_FP16_GRID}

_lib = None


class EpicError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("epic status %d: %s" % (status, msg))
        self.status = status


def load(path=LIB_PATH):
    """Load the shared library (raises if it is missing: there is no fallback)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError("libepic.so not built at %s; run paper_1510_08318_gb300.build.build()" % path)
    lib = ctypes.CDLL(path)
    vp, i32, i64, dbl = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_double
    lib.epic_create.restype = i32
    lib.epic_create.argtypes = [ctypes.POINTER(vp), i32, vp, vp, vp, vp, dbl, vp, i32, i32, i32, i32, i32, i32]
    lib.epic_destroy.restype = None
    lib.epic_destroy.argtypes = [vp]
    lib.epic_image.restype = i32
    lib.epic_image.argtypes = [vp, vp, i32, vp, vp, vp, i64, vp, vp, vp]
    lib.epic_image_noalloc.restype = i32
    lib.epic_image_noalloc.argtypes = [vp, vp, i32, vp, vp, vp, i64, vp, vp, i32, vp]
    lib.epic_image_backward.restype = i32
    lib.epic_image_backward.argtypes = [vp, vp, i32, vp, vp, vp, vp]
    lib.epic_image_xpol.restype = i32
    lib.epic_image_xpol.argtypes = [vp, vp, i32, vp, vp, i64, vp, vp, vp]
    lib.epic_fx_image.restype = i32
    lib.epic_fx_image.argtypes = [vp, vp, vp, vp]
    lib.epic_fengine.restype = i32
    lib.epic_fengine.argtypes = [i32, i32, i32, i32, i32, vp, i32, vp, i32, vp]
    lib.epic_weff.restype = i32
    lib.epic_weff.argtypes = [vp, vp, vp]
    lib.epic_isotropic.restype = i32
    lib.epic_isotropic.argtypes = [vp, vp, vp, vp, ctypes.c_float, vp, vp]
    lib.epic_correlate.restype = i32
    lib.epic_correlate.argtypes = [vp, vp, i32, vp, vp, vp]
    lib.epic_grid.restype = i32
    lib.epic_grid.argtypes = [vp, vp, i32, vp, vp, vp]
    lib.epic_plan_info.restype = i32
    lib.epic_plan_info.argtypes = [vp, ctypes.POINTER(i64), ctypes.POINTER(i64), ctypes.POINTER(i32)]
    lib.epic_set_transform.restype = i32
    lib.epic_set_transform.argtypes = [vp, i32]
    lib.epic_sync.restype = i32
    lib.epic_sync.argtypes = [vp, vp]
    lib.epic_set_wait_limit.restype = i32
    lib.epic_set_wait_limit.argtypes = [vp, i32]
    pp = ctypes.POINTER(vp)
    lib.epic_batch_create.restype = i32
    lib.epic_batch_create.argtypes = [pp, i32, pp]
    lib.epic_batch_image.restype = i32
    lib.epic_batch_image.argtypes = [vp, pp, ctypes.POINTER(i32), pp, pp, pp, vp]
    lib.epic_batch_autotune.restype = i32
    lib.epic_batch_autotune.argtypes = [vp, pp, ctypes.POINTER(i32), pp, pp, vp]
    lib.epic_batch_class.restype = i32
    lib.epic_batch_class.argtypes = [vp, i32, ctypes.POINTER(i32), ctypes.POINTER(i32), ctypes.POINTER(i32)]
    lib.epic_batch_info.restype = i32
    lib.epic_batch_info.argtypes = [vp, ctypes.POINTER(i32), ctypes.POINTER(i32), ctypes.POINTER(i32), i32]
    lib.epic_batch_destroy.restype = None
    lib.epic_batch_destroy.argtypes = [vp]
    lib.epic_last_error.restype = ctypes.c_char_p
    lib.epic_last_error.argtypes = []
    _lib = lib
    return lib


def epic_last_error():
    return load().epic_last_error().decode()


def _check(status):
    if status != EPIC_OK:
        raise EpicError(status, epic_last_error())


def _ptr(x):
    """Device or host address of a torch tensor / numpy array (an int passes through), or None."""
    if x is None or isinstance(x, int):
        return x
    if isinstance(x, np.ndarray):
        return x.ctypes.data
    return x.data_ptr()


# ---- the C entry points, one to one ------------------------------------------------------
def epic_create(n_ant, pos_xy, kern_ptr, kern_dxdy, kern_w, dx, origin_xy, n_grid, n_pad,
                n_chan, n_pol, volt_dtype, device):
    """Host numpy arrays in, opaque plan handle out (see include/epic.h)."""
    lib = load()
    pos = np.ascontiguousarray(pos_xy, dtype=np.float64)
    kp = np.ascontiguousarray(kern_ptr, dtype=np.int32)
    kd = np.ascontiguousarray(kern_dxdy, dtype=np.float64)
    kw = np.ascontiguousarray(kern_w)
    if np.iscomplexobj(kw):
        kw = np.stack([kw.real, kw.imag], axis=-1)
    kw = np.ascontiguousarray(kw, dtype=np.float64)
    org = np.ascontiguousarray(origin_xy, dtype=np.float64)
    h = ctypes.c_void_p()
    _check(lib.epic_create(ctypes.byref(h), int(n_ant), pos.ctypes.data, kp.ctypes.data,
                           kd.ctypes.data if kd.size else None, kw.ctypes.data if kw.size else None,
                           float(dx), org.ctypes.data, int(n_grid), int(n_pad), int(n_chan), int(n_pol),
                           int(volt_dtype), int(device)))
    return h


def epic_destroy(plan):
    load().epic_destroy(plan)


def epic_image(plan, volt, n_time, gains, accum, power, t_prev, image, autocorr, stream):
    _check(load().epic_image(plan, volt, int(n_time), gains, accum, power, int(t_prev), image, autocorr, stream))


def epic_image_noalloc(plan, volt, n_time, gains, accum, power, t_prev, image, autocorr, chunk_items, stream):
    _check(load().epic_image_noalloc(plan, volt, int(n_time), gains, accum, power, int(t_prev), image, autocorr,
                                     int(chunk_items), stream))


def epic_image_backward(plan, volt, n_time, gains, grad_image, grad_gains, stream):
    _check(load().epic_image_backward(plan, volt, int(n_time), gains, grad_image, grad_gains, stream))


def epic_image_xpol(plan, volt, n_time, gains, accum4, t_prev, image, cross, stream):
    _check(load().epic_image_xpol(plan, volt, int(n_time), gains, accum4, int(t_prev), image, cross, stream))


def epic_fengine(n_ant, n_pol, n_chan, n_time, in_dtype, raw, out_dtype, volt, device, stream):
    _check(load().epic_fengine(int(n_ant), int(n_pol), int(n_chan), int(n_time), int(in_dtype), raw,
                               int(out_dtype), volt, int(device), stream))


def fengine(raw, n_chan, in_dtype, out_dtype="f16", stream=None):
    """F-engine on a CUDA tensor of time samples [T C, P, A] (uint8 for "ci4", [.., 2] float16
    for "f16", complex64 for "c64") -> spectra [T, C, P, A] (complex64, or [.., 2] float16)."""
    import torch
    if not raw.is_cuda or not raw.is_contiguous():
        raise ValueError("raw samples must be a contiguous CUDA tensor")
    n_samp, P, A = int(raw.shape[0]), int(raw.shape[1]), int(raw.shape[2])
    if n_samp % n_chan:
        raise ValueError("the number of samples must be a multiple of n_chan")
    T = n_samp // n_chan
    if out_dtype == "f16":
        out = torch.empty((T, n_chan, P, A, 2), dtype=torch.float16, device=raw.device)
    else:
        out = torch.empty((T, n_chan, P, A), dtype=torch.complex64, device=raw.device)
    st = torch.cuda.current_stream(raw.device) if stream is None else stream
    epic_fengine(A, P, n_chan, T, VOLT_DTYPES[in_dtype], raw.data_ptr(), VOLT_DTYPES[out_dtype], out.data_ptr(),
                 raw.device.index or 0, st.cuda_stream)
    return out


def epic_fx_image(plan, vis, image, stream):
    _check(load().epic_fx_image(plan, vis, image, stream))


def epic_weff(plan, weff, stream):
    _check(load().epic_weff(plan, weff, stream))


def epic_isotropic(plan, image, autocorr, weff, rel_floor, iso, stream):
    _check(load().epic_isotropic(plan, image, autocorr, weff, float(rel_floor), iso, stream))


def epic_correlate(plan, volt, n_time, gains, vis, stream):
    _check(load().epic_correlate(plan, volt, int(n_time), gains, vis, stream))


def epic_grid(plan, volt, n_time, gains, grid, stream):
    _check(load().epic_grid(plan, volt, int(n_time), gains, grid, stream))


def epic_set_transform(plan, xform):
    _check(load().epic_set_transform(plan, int(xform)))


def epic_sync(plan, stream):
    _check(load().epic_sync(plan, stream))


def epic_set_wait_limit(plan, tries):
    _check(load().epic_set_wait_limit(plan, int(tries)))


def _ptr_array(xs):
    return (ctypes.c_void_p * len(xs))(*[_ptr(x) for x in xs])


def epic_batch_create(plans):
    h = ctypes.c_void_p()
    arr = (ctypes.c_void_p * len(plans))(*[p.value if isinstance(p, ctypes.c_void_p) else p for p in plans])
    _check(load().epic_batch_create(ctypes.byref(h), len(plans), arr))
    return h


def epic_batch_image(batch, volt, n_time, gains, accum, image, stream):
    n = len(volt)
    nt = (ctypes.c_int * n)(*[int(t) for t in n_time])
    _check(load().epic_batch_image(batch, _ptr_array(volt), nt, None if gains is None else _ptr_array(gains),
                                   _ptr_array(accum), None if image is None else _ptr_array(image), stream))


def epic_batch_autotune(batch, volt, n_time, gains, accum, stream):
    n = len(volt)
    nt = (ctypes.c_int * n)(*[int(t) for t in n_time])
    _check(load().epic_batch_autotune(batch, _ptr_array(volt), nt, None if gains is None else _ptr_array(gains),
                                      _ptr_array(accum), stream))


def epic_batch_class(batch, k):
    npad, w, f = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    _check(load().epic_batch_class(batch, int(k), ctypes.byref(npad), ctypes.byref(w), ctypes.byref(f)))
    return {"n_pad": npad.value, "workers": w.value,
            "form": ("persistent", "two-pass", "persistent, one buffer")[f.value]}


def epic_batch_info(batch, max_classes=16):
    nc, conc = ctypes.c_int(), ctypes.c_int()
    w = (ctypes.c_int * max_classes)()
    _check(load().epic_batch_info(batch, ctypes.byref(nc), ctypes.byref(conc), w, max_classes))
    return {"n_classes": nc.value, "concurrent": bool(conc.value), "workers": list(w)[:nc.value],
            "classes": [epic_batch_class(batch, k) for k in range(nc.value)]}


def epic_batch_destroy(batch):
    load().epic_batch_destroy(batch)


def epic_plan_info(plan):
    nnz, cells, lag = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int()
    _check(load().epic_plan_info(plan, ctypes.byref(nnz), ctypes.byref(cells), ctypes.byref(lag)))
    return {"nnz": nnz.value, "n_cells": cells.value, "lag_side": lag.value}


# ---- torch convenience layer --------------------------------------------------------------
class Plan:
    """An imaging plan on one CUDA device (antenna-to-grid mapping + device tables)."""

    def __init__(self, pos, kern_ptr, kern_dxdy, kern_w, dx, origin, n_grid, n_pad, n_chan, n_pol,
                 vdtype="c64", device=0):
        self.n_ant = int(np.asarray(pos).shape[0])
        self.n_grid, self.n_pad, self.n_chan, self.n_pol = int(n_grid), int(n_pad), int(n_chan), int(n_pol)
        self.vdtype = vdtype
        self.device = int(device)
        self._h = epic_create(self.n_ant, pos, kern_ptr, kern_dxdy, kern_w, dx, origin, n_grid, n_pad,
                              n_chan, n_pol, VOLT_DTYPES[vdtype], device)
        self.info = epic_plan_info(self._h)

    def set_transform(self, xform):
        """'fft' (FP32 shared-memory FFT), 'dftgemm' (tensor-core DFT, FP16 hi+lo, N_p = 128 or
        256), 'dftgemm_fp16' (reduced precision: FP16 gridding operands and one FP16 product
        per real product, N_p = 128), 'dftgemm_fp16grid' (FP16 gridding operands with FP32
        sums, then the hi+lo tensor-core DFT, N_p = 256) or 'fft_twopass' (FP32 FFT in a row and
        a column pass through a scratch buffer, N_p = 512)."""
        epic_set_transform(self._h, XFORMS[xform])
        self.xform = xform
        return self

    def sync(self, stream=None):
        """epic_sync: wait for the stream and raise EpicError (status EPIC_ETIMEOUT) if a bounded
        tensor-core wait of this plan's kernels ran out since the last sync."""
        import torch
        st = torch.cuda.current_stream(torch.device("cuda", self.device)) if stream is None else stream
        epic_sync(self._h, st.cuda_stream)

    def set_wait_limit(self, tries):
        """epic_set_wait_limit: tries (about 1 ms each) of the tensor-core pipelines' waits."""
        epic_set_wait_limit(self._h, tries)
        return self

    @classmethod
    def from_workload(cls, wl, device=0, n_chan=None):
        return cls(wl.pos, wl.kern_ptr, wl.kern_dxdy, wl.kern_w, wl.dx, wl.origin, wl.n_grid, wl.n_pad,
                   wl.n_chan if n_chan is None else n_chan, wl.n_pol, wl.vdtype, device)

    def close(self):
        if getattr(self, "_h", None):
            epic_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # --- argument checks (shape, dtype, device, contiguity) ---
    def _volt_ptr(self, volt):
        import torch
        C, P, A = self.n_chan, self.n_pol, self.n_ant
        if not volt.is_cuda or not volt.is_contiguous():
            raise ValueError("voltages must be a contiguous CUDA tensor")
        if self.vdtype == "ci4":
            ok = volt.dtype == torch.uint8 and volt.dim() == 4 and tuple(volt.shape[1:]) == (C, P, A)
        elif self.vdtype == "f16":
            ok = volt.dtype == torch.float16 and volt.dim() == 5 and tuple(volt.shape[1:]) == (C, P, A, 2)
        else:
            ok = ((volt.dtype == torch.float32 and volt.dim() == 5 and tuple(volt.shape[1:]) == (C, P, A, 2))
                  or (volt.dtype == torch.complex64 and volt.dim() == 4 and tuple(volt.shape[1:]) == (C, P, A)))
        if not ok:
            raise ValueError("voltages %s %s do not match the plan (%s, C=%d, P=%d, A=%d)"
                             % (tuple(volt.shape), volt.dtype, self.vdtype, C, P, A))
        return volt.data_ptr(), int(volt.shape[0])

    def _gains_ptr(self, gains):
        import torch
        if gains is None:
            return None
        if gains.dtype != torch.complex64 or not gains.is_cuda or not gains.is_contiguous() \
                or tuple(gains.shape) != (self.n_chan, self.n_pol, self.n_ant):
            raise ValueError("gains must be a contiguous complex64 CUDA tensor [C, P, A]")
        return gains.data_ptr()

    def image(self, volt, gains=None, accum=None, power=None, t_prev=0, want_image=True,
              want_autocorr=False, stream=None):
        """Run epic_image; returns dict(image, autocorr, accum, power) of CUDA tensors."""
        import torch
        dev = torch.device("cuda", self.device)
        vptr, T = self._volt_ptr(volt)
        C, P, NP, A = self.n_chan, self.n_pol, self.n_pad, self.n_ant
        if accum is None:
            accum = torch.empty((C, P, NP, NP), dtype=torch.float64, device=dev)
        if want_autocorr and power is None:
            power = torch.empty((C, P, A), dtype=torch.float64, device=dev)
        img = torch.empty((C, P, NP, NP), dtype=torch.float32, device=dev) if want_image else None
        ac = torch.empty((C, P, NP, NP), dtype=torch.float32, device=dev) if want_autocorr else None
        st = torch.cuda.current_stream(dev) if stream is None else stream
        epic_image(self._h, vptr, T, self._gains_ptr(gains), accum.data_ptr(), _ptr(power), t_prev,
                   _ptr(img), _ptr(ac), st.cuda_stream)
        return {"image": img, "autocorr": ac, "accum": accum, "power": power}

    def image_backward(self, volt, gains, grad_image, stream=None):
        import torch
        dev = torch.device("cuda", self.device)
        vptr, T = self._volt_ptr(volt)
        g = grad_image.contiguous().to(torch.float32)
        if tuple(g.shape) != (self.n_chan, self.n_pol, self.n_pad, self.n_pad) or not g.is_cuda:
            raise ValueError("grad_image must be a CUDA tensor [C, P, N_p, N_p]")
        out = torch.empty((self.n_chan, self.n_pol, self.n_ant), dtype=torch.complex64, device=dev)
        st = torch.cuda.current_stream(dev) if stream is None else stream
        epic_image_backward(self._h, vptr, T, self._gains_ptr(gains), g.data_ptr(), out.data_ptr(),
                            st.cuda_stream)
        return out

    def image_xpol(self, volt, gains=None, accum4=None, t_prev=0, stream=None):
        """Run epic_image_xpol: dict(image [C, 2, N_p, N_p] float32 (XX, YY), cross [C, N_p, N_p]
        complex64 (XY = <F_X conj F_Y>), accum4 [C, 4, N_p, N_p] float64)."""
        import torch
        dev = torch.device("cuda", self.device)
        vptr, T = self._volt_ptr(volt)
        C, NP = self.n_chan, self.n_pad
        if accum4 is None:
            accum4 = torch.empty((C, 4, NP, NP), dtype=torch.float64, device=dev)
        img = torch.empty((C, 2, NP, NP), dtype=torch.float32, device=dev)
        cross = torch.empty((C, NP, NP), dtype=torch.complex64, device=dev)
        st = torch.cuda.current_stream(dev) if stream is None else stream
        epic_image_xpol(self._h, vptr, T, self._gains_ptr(gains), accum4.data_ptr(), t_prev, img.data_ptr(),
                        cross.data_ptr(), st.cuda_stream)
        return {"image": img, "cross": cross, "accum4": accum4}

    def fx_image(self, vis, stream=None):
        """Run epic_fx_image: the FX-route image [C, P, N_p, N_p] of visibilities [C, P, A, A]."""
        import torch
        dev = torch.device("cuda", self.device)
        if (vis.dtype != torch.complex64 or tuple(vis.shape) != (self.n_chan, self.n_pol, self.n_ant, self.n_ant)
                or not vis.is_cuda or not vis.is_contiguous()):
            raise ValueError("vis must be a contiguous complex64 CUDA tensor [C, P, A, A]")
        out = torch.empty((self.n_chan, self.n_pol, self.n_pad, self.n_pad), dtype=torch.float32, device=dev)
        st = torch.cuda.current_stream(dev) if stream is None else stream
        epic_fx_image(self._h, vis.data_ptr(), out.data_ptr(), st.cuda_stream)
        return out

    def weff(self, stream=None):
        """Run epic_weff: the effective weighting W_eff [N_p, N_p] (float32 CUDA tensor)."""
        import torch
        dev = torch.device("cuda", self.device)
        out = torch.empty((self.n_pad, self.n_pad), dtype=torch.float32, device=dev)
        st = torch.cuda.current_stream(dev) if stream is None else stream
        epic_weff(self._h, out.data_ptr(), st.cuda_stream)
        return out

    def isotropic(self, image, autocorr, weff, rel_floor=1e-3, stream=None):
        """Run epic_isotropic: (image - autocorr) / (A (A - 1) W_eff), NaN where W_eff is below
        rel_floor of its peak."""
        import torch
        dev = torch.device("cuda", self.device)
        shape = (self.n_chan, self.n_pol, self.n_pad, self.n_pad)
        for t in (image, autocorr):
            if t.dtype != torch.float32 or tuple(t.shape) != shape or not t.is_cuda or not t.is_contiguous():
                raise ValueError("image and autocorr must be contiguous float32 CUDA tensors %s" % (shape,))
        if tuple(weff.shape) != (self.n_pad, self.n_pad) or weff.dtype != torch.float32 or not weff.is_contiguous():
            raise ValueError("weff must be a contiguous float32 tensor [N_p, N_p]")
        out = torch.empty(shape, dtype=torch.float32, device=dev)
        st = torch.cuda.current_stream(dev) if stream is None else stream
        epic_isotropic(self._h, image.data_ptr(), autocorr.data_ptr(), weff.data_ptr(), rel_floor, out.data_ptr(),
                       st.cuda_stream)
        return out

    def correlate(self, volt, gains=None, out=None, stream=None):
        """Run epic_correlate: visibilities <g_a V_a conj(g_b V_b)>_t, complex64 [C, P, A, A]."""
        import torch
        dev = torch.device("cuda", self.device)
        vptr, T = self._volt_ptr(volt)
        shape = (self.n_chan, self.n_pol, self.n_ant, self.n_ant)
        if out is None:
            out = torch.empty(shape, dtype=torch.complex64, device=dev)
        elif (out.dtype != torch.complex64 or tuple(out.shape) != shape or not out.is_cuda
              or not out.is_contiguous()):
            raise ValueError("out must be a contiguous complex64 CUDA tensor %s" % (shape,))
        st = torch.cuda.current_stream(dev) if stream is None else stream
        epic_correlate(self._h, vptr, T, self._gains_ptr(gains), out.data_ptr(), st.cuda_stream)
        return out

    def grid(self, volt, gains=None, out=None, stream=None):
        """Run epic_grid: the gridded fields E_t(g), complex64 CUDA tensor [T, C, P, N_g, N_g]."""
        import torch
        dev = torch.device("cuda", self.device)
        vptr, T = self._volt_ptr(volt)
        shape = (T, self.n_chan, self.n_pol, self.n_grid, self.n_grid)
        if out is None:
            out = torch.empty(shape, dtype=torch.complex64, device=dev)
        elif (out.dtype != torch.complex64 or tuple(out.shape) != shape or not out.is_cuda
              or not out.is_contiguous()):
            raise ValueError("out must be a contiguous complex64 CUDA tensor %s" % (shape,))
        st = torch.cuda.current_stream(dev) if stream is None else stream
        epic_grid(self._h, vptr, T, self._gains_ptr(gains), out.data_ptr(), st.cuda_stream)
        return out


class Batch:
    """Many plans imaged by one launch per padded-size class (epic_batch_*)."""

    def __init__(self, plans):
        self.plans = list(plans)
        self._h = epic_batch_create([p._h for p in self.plans])

    def _bufs(self, volts):
        import torch
        ptrs, nts = [], []
        for p, v in zip(self.plans, volts):
            ptr, T = p._volt_ptr(v)
            ptrs.append(ptr)
            nts.append(T)
        return ptrs, nts

    def alloc(self):
        import torch
        acc = [torch.empty((p.n_chan, p.n_pol, p.n_pad, p.n_pad), dtype=torch.float64,
                           device=torch.device("cuda", p.device)) for p in self.plans]
        img = [torch.empty((p.n_chan, p.n_pol, p.n_pad, p.n_pad), dtype=torch.float32,
                           device=torch.device("cuda", p.device)) for p in self.plans]
        return acc, img

    def image(self, volts, accum, image=None, gains=None, stream=None):
        import torch
        ptrs, nts = self._bufs(volts)
        st = torch.cuda.current_stream(torch.device("cuda", self.plans[0].device)) if stream is None else stream
        g = None if gains is None else [None if x is None else self.plans[i]._gains_ptr(x) for i, x in enumerate(gains)]
        epic_batch_image(self._h, ptrs, nts, g, accum, image, st.cuda_stream)

    def autotune(self, volts, accum, gains=None, stream=None):
        import torch
        ptrs, nts = self._bufs(volts)
        st = torch.cuda.current_stream(torch.device("cuda", self.plans[0].device)) if stream is None else stream
        g = None if gains is None else [None if x is None else self.plans[i]._gains_ptr(x) for i, x in enumerate(gains)]
        epic_batch_autotune(self._h, ptrs, nts, g, accum, st.cuda_stream)
        return epic_batch_info(self._h)

    def info(self):
        return epic_batch_info(self._h)

    def close(self):
        if getattr(self, "_h", None):
            epic_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _autograd_function():
    import torch

    class MoffImage(torch.autograd.Function):
        """image = MoffImage.apply(gains, volt, plan): the time-averaged MOFF image as a
        differentiable function of the complex gains [C, P, A] (complex64)."""

        @staticmethod
        def forward(ctx, gains, volt, plan):
            g = gains.detach().contiguous()
            out = plan.image(volt, g)["image"]
            ctx.save_for_backward(g)
            ctx.volt, ctx.plan = volt, plan
            return out

        @staticmethod
        def backward(ctx, grad_image):
            (g,) = ctx.saved_tensors
            return ctx.plan.image_backward(ctx.volt, g, grad_image), None, None

    return MoffImage


_MOFF = None


def moff_image(gains, volt, plan):
    """Differentiable MOFF image (see MoffImage)."""
    global _MOFF
    if _MOFF is None:
        _MOFF = _autograd_function()
    return _MOFF.apply(gains, volt, plan)
