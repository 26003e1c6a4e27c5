"""Python binding of the wiresim C ABI (``include/wiresim.h``).

Argument marshalling only: every step of the path runs in the CUDA library.
The ``ws_*`` functions mirror the C entry points one to one; ``Plane`` wraps
them for torch tensors (PyTorch provides device memory and streams).  If the
library has not been built, loading it raises ``WiresimError``: there is no
fallback.
"""
from __future__ import annotations

import ctypes
import dataclasses
import os
import threading

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libwiresim.so")

WS_OK = 0
STATUS_NAMES = {0: "WS_OK", 1: "WS_ERR_INVALID_ARG", 2: "WS_ERR_UNSUPPORTED_SIZE", 3: "WS_ERR_OOM",
                4: "WS_ERR_CUDA", 5: "WS_ERR_TIMEOUT", 6: "WS_ERR_WORKSPACE", 7: "WS_ERR_BAD_INPUT"}
WS_DEV_BAD_DEPO = 0x1
WS_DEV_PATCH_OVERFLOW = 0x2
WS_DEV_TIMEOUT = 0x4
WS_CONV_LINEAR, WS_CONV_CIRCULAR = 0, 1
WS_PREC_FP32, WS_PREC_FP32_COMP, WS_PREC_FP64 = 0, 1, 2

#: Every symbol include/wiresim.h declares.
EXPORTED = ("ws_plane_workspace_bytes", "ws_plane_create", "ws_plane_destroy", "ws_plane_get_info",
            "ws_patch_capacity", "ws_rasterize", "ws_scatter", "ws_convolve", "ws_simulate",
            "ws_plane_sync", "ws_plane_clear_status", "ws_plane_trace", "ws_plane_trace_read",
            "ws_convolve_noalloc", "ws_plane_set_wire_conv_variant", "ws_plane_set_response", "ws_plane_set_noise",
            "ws_simulate_backward", "ws_batch_workspace_bytes", "ws_simulate_batch", "ws_batch_autotune",
            "ws_selftest_bounded_wait",
            "ws_status_string", "ws_last_error")


class WiresimError(RuntimeError):
    def __init__(self, status: int, where: str, detail: str = ""):
        self.status = status
        msg = f"{where}: {STATUS_NAMES.get(status, status)}"
        if detail:
            msg += f" ({detail})"
        super().__init__(msg)


class WsPlaneDesc(ctypes.Structure):
    _fields_ = [("nwires", ctypes.c_int32), ("nticks", ctypes.c_int32),
                ("pitch_mm", ctypes.c_double), ("tick_us", ctypes.c_double),
                ("resp_nwires", ctypes.c_int32), ("resp_nticks", ctypes.c_int32),
                ("resp_wire_center", ctypes.c_int32), ("conv_mode", ctypes.c_int32),
                ("fft_len_tick", ctypes.c_int32), ("nsigma", ctypes.c_double),
                ("plane_id", ctypes.c_int32), ("fp64", ctypes.c_int32), ("impacts", ctypes.c_int32)]


class WsDepos(ctypes.Structure):
    _fields_ = [("q", ctypes.c_void_p), ("x_mm", ctypes.c_void_p), ("t_us", ctypes.c_void_p),
                ("sigma_t_us", ctypes.c_void_p), ("sigma_x_mm", ctypes.c_void_p),
                ("n", ctypes.c_int64)]


class WsParams(ctypes.Structure):
    _fields_ = [("DL_mm2_us", ctypes.c_double), ("DT_mm2_us", ctypes.c_double),
                ("v_mm_us", ctypes.c_double), ("fluctuate", ctypes.c_int32),
                ("p_survive", ctypes.c_double), ("seed", ctypes.c_uint64),
                ("event_id", ctypes.c_uint32), ("fluct_exact_max", ctypes.c_int32),
                ("precision", ctypes.c_int32), ("depo_offset", ctypes.c_uint32)]


class WsPatches(ctypes.Structure):
    _fields_ = [("val", ctypes.c_void_p), ("w0", ctypes.c_void_p), ("t0", ctypes.c_void_p),
                ("nw", ctypes.c_void_p), ("nt", ctypes.c_void_p), ("off", ctypes.c_void_p),
                ("capacity_bins", ctypes.c_int64), ("n", ctypes.c_int64)]


class WsTraceStat(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char_p), ("launches", ctypes.c_int64), ("total_ms", ctypes.c_double)]


class WsPlaneInfo(ctypes.Structure):
    _fields_ = [("fft_len_tick", ctypes.c_int32), ("nfreq", ctypes.c_int32),
                ("nfreq_stride", ctypes.c_int32), ("npasses", ctypes.c_int32),
                ("radices", ctypes.c_int32 * 16), ("workspace_bytes", ctypes.c_size_t),
                ("wire_conv_variant", ctypes.c_int32), ("row_fft_fixed_shape", ctypes.c_int32),
                ("batch_units_per_wave", ctypes.c_int32), ("batch_wire_conv_variant", ctypes.c_int32)]


_lock = threading.Lock()
_lib = None


def load_library(path: str = LIB_PATH) -> ctypes.CDLL:
    """Load libwiresim.so (built by ``__graft_entry__.build()``); no fallback."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(path):
            raise WiresimError(4, "load_library", f"{path} is missing: build it with "
                               "paper_2203_02479_gb300.build.build()")
        h = ctypes.CDLL(path)
        P = ctypes.c_void_p
        sig = {
            "ws_plane_workspace_bytes": [ctypes.POINTER(WsPlaneDesc), ctypes.POINTER(ctypes.c_size_t)],
            "ws_plane_create": [ctypes.POINTER(WsPlaneDesc), P, P, ctypes.c_size_t, P, ctypes.POINTER(P)],
            "ws_plane_destroy": [P],
            "ws_plane_get_info": [P, ctypes.POINTER(WsPlaneInfo)],
            "ws_patch_capacity": [P, ctypes.POINTER(WsDepos), ctypes.POINTER(WsParams), P,
                                  ctypes.POINTER(ctypes.c_int64)],
            "ws_rasterize": [P, ctypes.POINTER(WsDepos), ctypes.POINTER(WsParams),
                             ctypes.POINTER(WsPatches), P],
            "ws_scatter": [P, ctypes.POINTER(WsPatches), P, P],
            "ws_convolve": [P, P, P, P],
            "ws_simulate": [P, ctypes.POINTER(WsDepos), ctypes.POINTER(WsParams), P, P],
            "ws_plane_sync": [P, P, ctypes.POINTER(ctypes.c_uint32)],
            "ws_selftest_bounded_wait": [P, ctypes.c_int, P, P],
            "ws_plane_clear_status": [P, P],
            "ws_plane_trace": [P, ctypes.c_int],
            "ws_plane_trace_read": [P, ctypes.POINTER(WsTraceStat), ctypes.c_int,
                                    ctypes.POINTER(ctypes.c_int)],
            "ws_convolve_noalloc": [ctypes.POINTER(WsPlaneDesc), P, P, P, P],
            "ws_plane_set_wire_conv_variant": [P, ctypes.c_int],
            "ws_plane_set_response": [P, P, P],
            "ws_plane_set_noise": [P, P, P, ctypes.c_int32, P],
            "ws_batch_workspace_bytes": [ctypes.POINTER(P), ctypes.c_int, ctypes.c_int,
                                         ctypes.POINTER(ctypes.c_size_t)],
            "ws_simulate_batch": [ctypes.POINTER(P), ctypes.c_int, ctypes.POINTER(WsDepos), ctypes.c_int,
                                  ctypes.POINTER(WsParams), ctypes.POINTER(P), P, ctypes.c_size_t, ctypes.c_int, P],
            "ws_simulate_backward": [P, ctypes.POINTER(WsDepos), ctypes.POINTER(WsParams), P, P, P, P, P, P,
                                     P, P],
            "ws_batch_autotune": [ctypes.POINTER(P), ctypes.c_int, ctypes.POINTER(WsDepos), ctypes.c_int,
                                  ctypes.POINTER(WsParams), ctypes.POINTER(P), P, ctypes.c_size_t, P,
                                  ctypes.POINTER(ctypes.c_int)],
        }
        for name, args in sig.items():
            fn = getattr(h, name)
            fn.argtypes = args
            fn.restype = ctypes.c_int
        h.ws_status_string.argtypes = [ctypes.c_int]
        h.ws_status_string.restype = ctypes.c_char_p
        h.ws_last_error.argtypes = []
        h.ws_last_error.restype = ctypes.c_char_p
        _lib = h
        return h


def _check(status: int, where: str):
    if status != WS_OK:
        detail = ""
        if status == 4:
            detail = load_library().ws_last_error().decode(errors="replace")
        raise WiresimError(status, where, detail)


# ------------------------------------------------------------ thin wrappers
def ws_plane_workspace_bytes(desc: WsPlaneDesc) -> int:
    n = ctypes.c_size_t(0)
    _check(load_library().ws_plane_workspace_bytes(ctypes.byref(desc), ctypes.byref(n)),
           "ws_plane_workspace_bytes")
    return int(n.value)


def ws_plane_create(desc: WsPlaneDesc, response_dev: int, workspace_dev: int, workspace_bytes: int,
                    stream: int) -> int:
    h = ctypes.c_void_p(0)
    _check(load_library().ws_plane_create(ctypes.byref(desc), response_dev, workspace_dev,
                                          workspace_bytes, stream, ctypes.byref(h)), "ws_plane_create")
    return int(h.value)


def ws_plane_destroy(plane: int):
    _check(load_library().ws_plane_destroy(plane), "ws_plane_destroy")


def ws_plane_get_info(plane: int) -> WsPlaneInfo:
    info = WsPlaneInfo()
    _check(load_library().ws_plane_get_info(plane, ctypes.byref(info)), "ws_plane_get_info")
    return info


def ws_patch_capacity(plane: int, depos: WsDepos, params: WsParams, stream: int) -> int:
    n = ctypes.c_int64(0)
    _check(load_library().ws_patch_capacity(plane, ctypes.byref(depos), ctypes.byref(params), stream,
                                            ctypes.byref(n)), "ws_patch_capacity")
    return int(n.value)


def ws_rasterize(plane: int, depos: WsDepos, params: WsParams, patches: WsPatches, stream: int):
    _check(load_library().ws_rasterize(plane, ctypes.byref(depos), ctypes.byref(params),
                                       ctypes.byref(patches), stream), "ws_rasterize")


def ws_scatter(plane: int, patches: WsPatches, grid_dev: int, stream: int):
    _check(load_library().ws_scatter(plane, ctypes.byref(patches), grid_dev, stream), "ws_scatter")


def ws_convolve(plane: int, grid_dev: int, out_dev: int, stream: int):
    _check(load_library().ws_convolve(plane, grid_dev, out_dev, stream), "ws_convolve")


def ws_simulate(plane: int, depos: WsDepos, params: WsParams, out_dev: int, stream: int):
    _check(load_library().ws_simulate(plane, ctypes.byref(depos), ctypes.byref(params), out_dev, stream),
           "ws_simulate")


def ws_selftest_bounded_wait(status_dev: int, iters: int, cycles_dev: int, stream: int):
    """Bounded-wait check (see include/wiresim.h): a wait nobody satisfies
    gives up after `iters` attempts and sets WS_DEV_TIMEOUT in *status_dev."""
    _check(load_library().ws_selftest_bounded_wait(status_dev, iters, cycles_dev, stream),
           "ws_selftest_bounded_wait")


def ws_plane_sync(plane: int, stream: int) -> int:
    v = ctypes.c_uint32(0)
    _check(load_library().ws_plane_sync(plane, stream, ctypes.byref(v)), "ws_plane_sync")
    return int(v.value)


def ws_plane_clear_status(plane: int, stream: int):
    _check(load_library().ws_plane_clear_status(plane, stream), "ws_plane_clear_status")


def ws_plane_trace(plane: int, max_records: int):
    _check(load_library().ws_plane_trace(plane, max_records), "ws_plane_trace")


def ws_plane_trace_read(plane: int) -> dict:
    """{kernel name: (launches, total ms)} since tracing began or the last read."""
    stats = (WsTraceStat * 32)()
    n = ctypes.c_int(0)
    _check(load_library().ws_plane_trace_read(plane, stats, 32, ctypes.byref(n)), "ws_plane_trace_read")
    return {stats[i].name.decode(): (int(stats[i].launches), float(stats[i].total_ms))
            for i in range(n.value)}


def ws_convolve_noalloc(desc: WsPlaneDesc, response_dev: int, grid_dev: int, out_dev: int, stream: int):
    """Convolution without any device allocation (scratch is a 16 MiB array
    inside the library, shared by all calls); see include/wiresim.h."""
    _check(load_library().ws_convolve_noalloc(ctypes.byref(desc), response_dev, grid_dev, out_dev, stream),
           "ws_convolve_noalloc")


# ---------------------------------------------------------- torch helpers
def _torch():
    import torch
    return torch


def _stream_handle(stream) -> int:
    torch = _torch()
    if stream is None:
        stream = torch.cuda.current_stream()
    return int(stream.cuda_stream)


def _ptr(t) -> int:
    return 0 if t is None else int(t.data_ptr())


def _require(t, name: str, shape, device, dtype=None):
    """Check a tensor whose raw pointer goes to the library: the kernels
    index it by the plane's sizes, so a tensor of another shape or dtype,
    a strided view or one on another device would be read or written out of
    bounds.  Raises ValueError before any call into the library."""
    torch = _torch()
    dtype = torch.float32 if dtype is None else dtype
    if not hasattr(t, "data_ptr"):
        raise ValueError(f"{name}: expected a torch tensor, got {type(t).__name__}")
    if tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name}: expected shape {tuple(shape)}, got {tuple(t.shape)}")
    if t.dtype != dtype:
        raise ValueError(f"{name}: expected dtype {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name}: expected a contiguous tensor")
    want = torch.device(device)
    if t.device.type != want.type or (want.index is not None and t.device.index != want.index):
        raise ValueError(f"{name}: expected a tensor on {want}, got one on {t.device}")
    return t


@dataclasses.dataclass
class Params:
    """Physics and numerics of a simulation call (mirrors ``ws_params``)."""
    DL_mm2_us: float = 4.0e-4
    DT_mm2_us: float = 8.8e-4
    v_mm_us: float = 1.6
    fluctuate: int = 0        # 0 expected value, 1 (True) binomial per bin, 2 multinomial (charge-conserving)
    p_survive: float = 1.0
    seed: int = 0
    event_id: int = 0
    fluct_exact_max: int = 32
    precision: int = WS_PREC_FP32
    depo_offset: int = 0      # index of the first depo in the event's whole list (random counters)

    def c(self) -> WsParams:
        return WsParams(self.DL_mm2_us, self.DT_mm2_us, self.v_mm_us, int(self.fluctuate),
                        self.p_survive, self.seed & (2 ** 64 - 1), self.event_id, self.fluct_exact_max,
                        self.precision, self.depo_offset)


class DeviceDepos:
    """Depo arrays resident on the device (float32, contiguous)."""

    def __init__(self, q, x_mm, t_us, sigma_t_us=None, sigma_x_mm=None, device="cuda"):
        torch = _torch()

        def dev(a):
            if a is None:
                return None
            if not hasattr(a, "data_ptr"):
                a = torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32))
            return a.to(device=device, dtype=torch.float32).contiguous()

        self.q, self.x_mm, self.t_us = dev(q), dev(x_mm), dev(t_us)
        self.sigma_t_us, self.sigma_x_mm = dev(sigma_t_us), dev(sigma_x_mm)
        if self.q.dim() != 1:
            raise ValueError("depo arrays must be one-dimensional")
        self.n = int(self.q.shape[0])
        # the kernels read n entries of every array given (the widths too)
        for a in (self.x_mm, self.t_us, self.sigma_t_us, self.sigma_x_mm):
            if a is not None and tuple(a.shape) != (self.n,):
                raise ValueError("depo arrays differ in length")

    @classmethod
    def from_plane_depos(cls, d, device="cuda"):
        return cls(d.q, d.x_mm, d.t_us, device=device)

    def c(self) -> WsDepos:
        return WsDepos(_ptr(self.q), _ptr(self.x_mm), _ptr(self.t_us), _ptr(self.sigma_t_us),
                       _ptr(self.sigma_x_mm), self.n)


class Plane:
    """One wire plane with its response spectrum and workspace on the device."""

    def __init__(self, nwires: int, nticks: int, response, *, pitch_mm: float = 5.0,
                 tick_us: float = 0.5, wire_center: int = 10, circular: bool = False,
                 fft_len_tick: int = 0, nsigma: float = 3.0, plane_id: int = 0, fp64: bool = False,
                 device="cuda", stream=None):
        """response: K_w x K_t, or impacts x K_w x K_t for a response that
        depends on the charge's sub-pitch position (impact planes)."""
        torch = _torch()
        resp = response
        if isinstance(resp, np.ndarray):
            resp = torch.from_numpy(np.ascontiguousarray(resp, dtype=np.float32))
        self.response = resp.to(device=device, dtype=torch.float32).contiguous()
        self.impacts = int(self.response.shape[0]) if self.response.dim() == 3 else 1
        kw, kt = int(self.response.shape[-2]), int(self.response.shape[-1])
        self.desc = WsPlaneDesc(nwires, nticks, pitch_mm, tick_us, kw, kt, wire_center,
                                WS_CONV_CIRCULAR if circular else WS_CONV_LINEAR, fft_len_tick,
                                nsigma, plane_id, int(bool(fp64)), self.impacts if self.impacts > 1 else 0)
        self.nwires, self.nticks = nwires, nticks
        nbytes = ws_plane_workspace_bytes(self.desc)
        self.workspace = torch.empty(nbytes + 256, dtype=torch.uint8, device=device)
        base = _ptr(self.workspace)
        aligned = (base + 255) & ~255
        self.handle = ws_plane_create(self.desc, _ptr(self.response), aligned, nbytes,
                                      _stream_handle(stream))
        self.info = ws_plane_get_info(self.handle)
        self.device = device
        self._resp_src = response            # what the plane's spectrum was computed from
        self._resp_held = self._resp_key(response)

    def close(self):
        if getattr(self, "handle", 0):
            ws_plane_destroy(self.handle)
            self.handle = 0

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def new_grid(self):
        """A zeroed grid for scatter / convolve: nwires x nticks, or the fine
        grid nwires*impacts x nticks of an impact plane."""
        torch = _torch()
        return torch.zeros((self.nwires * self.impacts, self.nticks), dtype=torch.float32, device=self.device)

    def simulate(self, depos: DeviceDepos, params: Params, out=None, stream=None):
        if out is None:
            out = _torch().empty((self.nwires, self.nticks), dtype=_torch().float32, device=self.device)
        _require(out, "out", (self.nwires, self.nticks), self.device)
        ws_simulate(self.handle, depos.c(), params.c(), _ptr(out), _stream_handle(stream))
        return out

    def convolve(self, grid, out=None, stream=None):
        if out is None:
            out = _torch().empty((self.nwires, self.nticks), dtype=_torch().float32, device=self.device)
        _require(grid, "grid", (self.nwires * self.impacts, self.nticks), self.device)
        _require(out, "out", (self.nwires, self.nticks), self.device)
        ws_convolve(self.handle, _ptr(grid), _ptr(out), _stream_handle(stream))
        return out

    def patch_capacity(self, depos: DeviceDepos, params: Params, stream=None) -> int:
        return ws_patch_capacity(self.handle, depos.c(), params.c(), _stream_handle(stream))

    def rasterize(self, depos: DeviceDepos, params: Params, capacity: int | None = None, stream=None):
        torch = _torch()
        if capacity is None:
            capacity = self.patch_capacity(depos, params, stream)
        n = depos.n
        p = dict(val=torch.zeros(max(capacity, 1), dtype=torch.float32, device=self.device),
                 w0=torch.zeros(max(n, 1), dtype=torch.int32, device=self.device),
                 t0=torch.zeros(max(n, 1), dtype=torch.int32, device=self.device),
                 nw=torch.zeros(max(n, 1), dtype=torch.int32, device=self.device),
                 nt=torch.zeros(max(n, 1), dtype=torch.int32, device=self.device),
                 off=torch.zeros(n + 1, dtype=torch.int64, device=self.device))
        p["capacity"] = capacity
        p["n"] = n
        ws_rasterize(self.handle, depos.c(), params.c(), self.patches_c(p), _stream_handle(stream))
        return p

    @staticmethod
    def patches_c(p) -> WsPatches:
        return WsPatches(_ptr(p["val"]), _ptr(p["w0"]), _ptr(p["t0"]), _ptr(p["nw"]), _ptr(p["nt"]),
                         _ptr(p["off"]), int(p["capacity"]), int(p["n"]))

    def scatter(self, patches, grid, stream=None):
        _require(grid, "grid", (self.nwires * self.impacts, self.nticks), self.device)
        ws_scatter(self.handle, self.patches_c(patches), _ptr(grid), _stream_handle(stream))
        return grid

    def set_wire_conv_variant(self, variant: int):
        _check(load_library().ws_plane_set_wire_conv_variant(self.handle, variant),
               "ws_plane_set_wire_conv_variant")
        self.info = ws_plane_get_info(self.handle)

    def set_response(self, response, stream=None):
        torch = _torch()
        src = response
        if not hasattr(response, "data_ptr"):
            response = torch.from_numpy(np.ascontiguousarray(response, dtype=np.float32))
        response = response.to(device=self.device, dtype=torch.float32).contiguous()
        # the plane's response shape is fixed at creation (impacts x K_w x K_t or K_w x K_t)
        self.response = _require(response, "response", tuple(self.response.shape), self.device)
        _check(load_library().ws_plane_set_response(self.handle, _ptr(self.response), _stream_handle(stream)),
               "ws_plane_set_response")
        self._resp_src = src
        self._resp_held = self._resp_key(src)

    @staticmethod
    def _resp_key(r):
        """Identity of a response tensor's contents: its storage, offset,
        shape, strides and version counter (None for non-tensors).  The plane
        keeps a reference to the tensor it recorded, so that storage cannot be
        handed to another tensor while the record stands; an in-place change
        bumps the version."""
        if not hasattr(r, "untyped_storage"):
            return None
        return (r.device, r.untyped_storage().data_ptr(), r.storage_offset(), tuple(r.shape), tuple(r.stride()),
                r.dtype, r._version)

    def use_response(self, response, stream=None):
        """Make the plane hold ``response``: recompute the spectrum only if the
        plane holds another response (or this one changed in place since)."""
        key = self._resp_key(response)
        if key is not None and key == self._resp_held:
            return
        self.set_response(response, stream)

    def set_noise(self, amp, coh=None, group: int = 1, stream=None):
        """Noise term of Eq. 1 for later simulate calls: amplitude spectra of
        L/2 + 1 entries (L = info.fft_len_tick), incoherent ``amp`` per wire and
        optional coherent ``coh`` shared by groups of ``group`` wires; both
        None switch it off."""
        torch = _torch()

        def dev(a):
            if a is None:
                return None
            if not hasattr(a, "data_ptr"):
                a = torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32))
            a = a.to(device=self.device, dtype=torch.float32).contiguous()
            if a.numel() != self.info.nfreq:
                raise ValueError(f"noise spectra need {self.info.nfreq} entries (L/2 + 1)")
            return a

        self.noise = (dev(amp), dev(coh))   # kept alive until the copies ran
        _check(load_library().ws_plane_set_noise(self.handle, _ptr(self.noise[0]), _ptr(self.noise[1]),
                                                 int(group), _stream_handle(stream)),
               "ws_plane_set_noise")

    def backward(self, depos: DeviceDepos, params: Params, grad_out, want_response: bool = True, stream=None):
        """(gq, gx, gt, gDL, gDT, gR) as device tensors (gR None if not wanted)."""
        torch = _torch()
        dev = self.device
        n = max(depos.n, 1)
        gq = torch.empty(n, dtype=torch.float32, device=dev)
        gx = torch.empty(n, dtype=torch.float32, device=dev)
        gt = torch.empty(n, dtype=torch.float32, device=dev)
        gD = torch.zeros(2, dtype=torch.float64, device=dev)
        gR = torch.empty(tuple(self.response.shape), dtype=torch.float32, device=dev) if want_response else None
        g = _require(grad_out.contiguous(), "grad_out", (self.nwires, self.nticks), self.device)
        _check(load_library().ws_simulate_backward(
            self.handle, ctypes.byref(depos.c()), ctypes.byref(params.c()), _ptr(g), _ptr(gq), _ptr(gx), _ptr(gt),
            _ptr(gD), _ptr(gD) + 8, _ptr(gR), _stream_handle(stream)), "ws_simulate_backward")
        return gq[:depos.n], gx[:depos.n], gt[:depos.n], gD[0], gD[1], gR

    def trace(self, max_records: int):
        ws_plane_trace(self.handle, max_records)

    def trace_read(self) -> dict:
        return ws_plane_trace_read(self.handle)

    def status(self, stream=None) -> int:
        return ws_plane_sync(self.handle, _stream_handle(stream))

    def clear_status(self, stream=None):
        ws_plane_clear_status(self.handle, _stream_handle(stream))


def batch_workspace_bytes(planes, units_per_wave: int) -> int:
    """Bytes of batch workspace for waves of ``units_per_wave`` units (0: 32)."""
    P = ctypes.c_void_p
    arr = (P * len(planes))(*[pl.handle for pl in planes])
    n = ctypes.c_size_t(0)
    _check(load_library().ws_batch_workspace_bytes(arr, len(planes), int(units_per_wave), ctypes.byref(n)),
           "ws_batch_workspace_bytes")
    return int(n.value)


def batch_workspace(planes, units_per_wave: int, device="cuda"):
    """A device workspace (uint8 tensor, 256 bytes of alignment slack) for
    batches on these planes with waves of up to ``units_per_wave`` units."""
    return _torch().empty(batch_workspace_bytes(planes, units_per_wave) + 256, dtype=_torch().uint8, device=device)


class Batch:
    """Many events x planes through ``ws_simulate_batch``.

    ``events[e][p]`` are DeviceDepos of event e seen by plane p; outputs are
    allocated per unit.  ``run()`` enqueues the batch; ``capture()`` records
    it once into a CUDA graph that ``replay()`` relaunches (the buffers stay
    fixed, so refill the depo tensors in place between replays).

    ``units_per_wave=0`` (the default) leaves the wave size to the library:
    ``autotune()`` times the candidate sizes on these inputs
    (``ws_batch_autotune``) and records the fastest on the planes;
    ``capture()`` runs it first if it has not run.  The workspace is sized
    for the largest wave these units can form (at most 32)."""

    def __init__(self, planes, events, params: Params, units_per_wave: int = 0, device="cuda",
                 workspace=None, outs=None):
        """workspace: a uint8 device tensor from ``batch_workspace`` to share
        between batches that never run at the same time (default: one of
        this batch's own); outs: the units' output tensors (default:
        allocated here)."""
        torch = _torch()
        self.planes = list(planes)
        self.events = events
        self.params = params
        self.units_per_wave = units_per_wave
        self.nplanes = len(self.planes)
        self.nevents = len(events)
        P = ctypes.c_void_p
        self._planes_c = (P * self.nplanes)(*[pl.handle for pl in self.planes])
        units = [events[e][p] for e in range(self.nevents) for p in range(self.nplanes)]
        self._depos_c = (WsDepos * len(units))(*[d.c() for d in units])
        if outs is None:
            outs = [torch.empty((self.planes[u % self.nplanes].nwires, self.planes[u % self.nplanes].nticks),
                                dtype=torch.float32, device=device) for u in range(len(units))]
        if len(outs) != len(units):
            raise ValueError(f"outs: expected {len(units)} tensors, got {len(outs)}")
        self.outs = [_require(o, "outs", (self.planes[u % self.nplanes].nwires, self.planes[u % self.nplanes].nticks),
                              device) for u, o in enumerate(outs)]
        self._outs_c = (P * len(units))(*[o.data_ptr() for o in self.outs])
        ws_upw = units_per_wave if units_per_wave > 0 else max(1, min(32, len(units)))
        need = batch_workspace_bytes(self.planes, ws_upw)
        if workspace is None:
            workspace = batch_workspace(self.planes, ws_upw, device)
        _require(workspace, "workspace", tuple(workspace.shape), device, dtype=torch.uint8)
        self.workspace = workspace
        self._ws_ptr = (self.workspace.data_ptr() + 255) & ~255
        self._ws_bytes = int(self.workspace.numel()) - (self._ws_ptr - self.workspace.data_ptr())
        if self._ws_bytes < need:
            raise ValueError(f"workspace: {need} bytes needed, {self._ws_bytes} given")
        self._params_c = params.c()
        self.graph = None
        self.tuned = units_per_wave > 0

    def autotune(self, stream=None) -> int:
        """Pick the wave size by timing the candidates on these inputs (the
        library's ws_batch_autotune; synchronises); returns it.  Later runs
        with units_per_wave=0 use it."""
        upw = ctypes.c_int(0)
        _check(load_library().ws_batch_autotune(self._planes_c, self.nplanes, self._depos_c, self.nevents,
                                                ctypes.byref(self._params_c), self._outs_c, self._ws_ptr,
                                                self._ws_bytes, _stream_handle(stream), ctypes.byref(upw)),
               "ws_batch_autotune")
        self.chosen_units_per_wave = int(upw.value)
        self.tuned = True
        for pl in self.planes:
            pl.info = ws_plane_get_info(pl.handle)
        return self.chosen_units_per_wave

    def run(self, stream=None):
        _check(load_library().ws_simulate_batch(self._planes_c, self.nplanes, self._depos_c, self.nevents,
                                                ctypes.byref(self._params_c), self._outs_c, self._ws_ptr,
                                                self._ws_bytes, self.units_per_wave, _stream_handle(stream)),
               "ws_simulate_batch")
        return self.outs

    def capture(self):
        torch = _torch()
        if not self.tuned and self.nevents > 0:
            self.autotune()
        s = torch.cuda.Stream()
        s.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(s):
            self.run(s)          # warm-up outside the graph (kernel attributes, lazy loading)
        torch.cuda.current_stream().wait_stream(s)
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            self.run()
        self.graph = g
        return g

    def replay(self):
        self.graph.replay()
        return self.outs
