"""Python binding of libkf.so: the C-ABI entry points under the same names.

Argument marshalling only -- every step of the Kalman path runs in the CUDA
kernels of libkf.so.  Tensors are passed as raw device pointers; PyTorch is
used for device memory and streams.  If the library is not built, or a
tensor is not on a CUDA device, the calls raise: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import dataclasses
import os
import re
from typing import Optional

import numpy as np
import torch

from . import workload as W

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "_build", "libkf.so")
HEADER = os.path.join(os.path.dirname(_PKG), "include", "kf.h")

KF_OK, KF_ERR_ARG, KF_ERR_CUDA, KF_ERR_UNSUPPORTED, KF_ERR_TIMEOUT = 0, 1, 2, 3, 4
NO_INTERSECT, S_NOT_PD, BAD_K, NONFINITE = 1, 2, 4, 8
KF_SOA, KF_AOSOA = 0, 1
KF_FP32, KF_FP64_UPDATE, KF_JOSEPH, KF_FP64, KF_ADAPTIVE, KF_DF_UPDATE = 0, 1, 2, 3, 4, 5


class KfError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"libkf error {code}: {msg}")
        self.code = code


class kf_layout(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("width", ctypes.c_int32), ("n", ctypes.c_int64)]


class kf_params(ctypes.Structure):
    _fields_ = [("bz", ctypes.c_float), ("precision", ctypes.c_int32), ("flags", ctypes.c_uint32)]


class kf_layer(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("pos", ctypes.c_float)]


KF_MAX_LAYERS = 64


class kf_tuning(ctypes.Structure):
    _fields_ = [("step_kernel", ctypes.c_int32), ("threads", ctypes.c_int32),
                ("ctas_per_sm", ctypes.c_int32), ("ms", ctypes.c_float)]


class kf_server_config(ctypes.Structure):
    _fields_ = [("bz", ctypes.c_float), ("precision", ctypes.c_int32), ("L", ctypes.c_int32),
                ("layers", kf_layer * KF_MAX_LAYERS), ("arena", ctypes.c_void_p),
                ("arena_bytes", ctypes.c_int64), ("max_events_in_flight", ctypes.c_int32),
                ("device", ctypes.c_int32)]


class kf_server_stats(ctypes.Structure):
    _fields_ = [("events_done", ctypes.c_int64), ("tracks_done", ctypes.c_int64),
                ("batches", ctypes.c_int64), ("max_batch_events", ctypes.c_int64),
                ("p50_ms", ctypes.c_double), ("p99_ms", ctypes.c_double),
                ("max_ms", ctypes.c_double), ("mean_ms", ctypes.c_double),
                ("queue_p50_ms", ctypes.c_double), ("queue_p99_ms", ctypes.c_double),
                ("ready_p50_ms", ctypes.c_double), ("ready_p99_ms", ctypes.c_double),
                ("compute_p50_ms", ctypes.c_double), ("compute_p99_ms", ctypes.c_double),
                ("out_p50_ms", ctypes.c_double), ("out_p99_ms", ctypes.c_double),
                ("copyin_p50_ms", ctypes.c_double), ("copyin_p99_ms", ctypes.c_double),
                ("gpu_copyin_p50_ms", ctypes.c_double), ("gpu_copyin_p99_ms", ctypes.c_double),
                ("gpu_compute_p50_ms", ctypes.c_double), ("gpu_compute_p99_ms", ctypes.c_double),
                ("gpu_out_p50_ms", ctypes.c_double), ("gpu_out_p99_ms", ctypes.c_double),
                ("copyin_issue_p50_ms", ctypes.c_double), ("copyin_issue_p99_ms", ctypes.c_double),
                ("sched_pass_max_ms", ctypes.c_double), ("sched_gap_max_ms", ctypes.c_double)]


_lib = None
_VP = ctypes.c_void_p


def load():
    """Load libkf.so (built in-tree by ``__graft_entry__.build()``)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is not built; run __graft_entry__.build() first")
    lib = ctypes.CDLL(LIB_PATH)
    step_args = [ctypes.POINTER(kf_params), kf_layout, _VP, _VP, _VP, _VP, _VP, _VP, _VP, _VP,
                 ctypes.c_int32, _VP, _VP]
    for name in ("kf_p2z_propagate_update", "kf_p2r_propagate_update"):
        fn = getattr(lib, name)
        fn.argtypes = step_args
        fn.restype = ctypes.c_int
    host_args = step_args[:-1] + [_VP, ctypes.c_int64, ctypes.c_int64, _VP]
    for name in ("kf_p2z_propagate_update_host", "kf_p2r_propagate_update_host"):
        fn = getattr(lib, name)
        fn.argtypes = host_args
        fn.restype = ctypes.c_int
    lib.kf_propagate_update_host_noalloc.argtypes = [ctypes.c_int32] + step_args[:-1] + [
        ctypes.c_int64, _VP]
    lib.kf_propagate_update_host_noalloc.restype = ctypes.c_int
    lib.kf_host_workspace_bytes.argtypes = [kf_layout, ctypes.c_int64]
    lib.kf_host_workspace_bytes.restype = ctypes.c_int64
    lib.kf_kalman_chain.argtypes = [ctypes.POINTER(kf_params), kf_layout, _VP, _VP, _VP, _VP,
                                    _VP, ctypes.POINTER(kf_layer), ctypes.c_int32, _VP, _VP]
    lib.kf_kalman_chain.restype = ctypes.c_int
    lib.kf_propagate_update_compressed.argtypes = [ctypes.c_int32, ctypes.POINTER(kf_params),
                                                   kf_layout] + [_VP] * 10 + [ctypes.c_int32,
                                                                              _VP, _VP]
    lib.kf_propagate_update_compressed.restype = ctypes.c_int
    srv = ctypes.c_void_p
    lib.kf_server_event_bytes.argtypes = [ctypes.c_int64, ctypes.c_int32]
    lib.kf_server_event_bytes.restype = ctypes.c_int64
    lib.kf_server_create.argtypes = [ctypes.POINTER(kf_server_config), ctypes.POINTER(srv)]
    lib.kf_server_submit.argtypes = [srv, ctypes.c_int64] + [_VP] * 8 + [
        ctypes.POINTER(ctypes.c_uint64)]
    lib.kf_server_poll.argtypes = [srv, ctypes.c_uint64, ctypes.POINTER(ctypes.c_int32)]
    lib.kf_server_wait.argtypes = [srv, ctypes.c_uint64, ctypes.c_double]
    lib.kf_server_pause.argtypes = [srv, ctypes.c_int32]
    lib.kf_server_get_stats.argtypes = [srv, ctypes.POINTER(kf_server_stats)]
    lib.kf_server_reset_stats.argtypes = [srv]
    lib.kf_server_destroy.argtypes = [srv]
    for name in ("kf_server_create", "kf_server_submit", "kf_server_poll", "kf_server_wait",
                 "kf_server_pause", "kf_server_get_stats", "kf_server_reset_stats",
                 "kf_server_destroy"):
        getattr(lib, name).restype = ctypes.c_int
    lib.kf_autotune_step.argtypes = [ctypes.c_int32, ctypes.POINTER(kf_params), kf_layout] + \
        [_VP] * 8 + [ctypes.c_int32, _VP, _VP, ctypes.POINTER(kf_tuning)]
    lib.kf_autotune_chain.argtypes = [ctypes.POINTER(kf_params), kf_layout] + [_VP] * 5 + [
        ctypes.POINTER(kf_layer), ctypes.c_int32, _VP, _VP, _VP, _VP, ctypes.POINTER(kf_tuning)]
    lib.kf_autotune_export.argtypes = [ctypes.c_char_p, ctypes.c_int64,
                                       ctypes.POINTER(ctypes.c_int64)]
    lib.kf_autotune_import.argtypes = [ctypes.c_char_p]
    lib.kf_autotune_clear.argtypes = []
    for name in ("kf_autotune_step", "kf_autotune_chain", "kf_autotune_export",
                 "kf_autotune_import", "kf_autotune_clear"):
        getattr(lib, name).restype = ctypes.c_int
    lib.kf_set_step_kernel.argtypes = [ctypes.c_int32]
    lib.kf_set_step_kernel.restype = ctypes.c_int
    lib.kf_set_staged_ctas_per_sm.argtypes = [ctypes.c_int32]
    lib.kf_set_staged_ctas_per_sm.restype = ctypes.c_int
    lib.kf_set_chain_redo.argtypes = [ctypes.c_int32]
    lib.kf_set_chain_redo.restype = ctypes.c_int
    lib.kf_set_host_path.argtypes = [ctypes.c_int32]
    lib.kf_set_host_path.restype = ctypes.c_int
    lib.kf_set_device_wait_limit.argtypes = [ctypes.c_int64]
    lib.kf_set_device_wait_limit.restype = ctypes.c_int
    lib.kf_take_device_error.argtypes = [ctypes.POINTER(ctypes.c_uint)]
    lib.kf_take_device_error.restype = ctypes.c_int
    lib.kf_version.restype = ctypes.c_int
    lib.kf_last_error_string.restype = ctypes.c_char_p
    _lib = lib
    return lib


def header_functions(path: str = HEADER):
    """Names of the functions declared in include/kf.h."""
    text = open(path).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(kf_[a-z0-9_]+)\s*\(", text)))


def _ptr(t, name: str, dtype: Optional[torch.dtype] = None):
    if t is None:
        return None
    if isinstance(t, int):
        return t
    if not isinstance(t, torch.Tensor):
        raise TypeError(f"{name}: expected a torch.Tensor or an int pointer")
    if not t.is_cuda:
        raise ValueError(f"{name}: tensor must be on a CUDA device")
    if dtype is not None and t.dtype != dtype:
        raise TypeError(f"{name}: expected {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name}: tensor must be contiguous")
    return t.data_ptr()


def _stream(stream):
    if stream is None:
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, torch.cuda.Stream):
        return stream.cuda_stream
    return int(stream)


def _check(rc: int):
    if rc != KF_OK:
        raise KfError(rc, load().kf_last_error_string().decode())


def make_layout(kind: int, width: int, n: int) -> kf_layout:
    return kf_layout(int(kind), int(width), int(n))


def make_params(bz: float, precision: int = KF_FP32, flags: int = 0) -> kf_params:
    return kf_params(float(bz), int(precision), int(flags))


def _step(fn_name, params, layout, state_in, cov_in, state_out, cov_out, charge, hit, hit_cov,
          surf, surf_per_track, status, stream):
    lib = load()
    f32, i8, u8 = torch.float32, torch.int8, torch.uint8
    rc = getattr(lib, fn_name)(
        ctypes.byref(params), layout,
        _ptr(state_in, "state_in", f32), _ptr(cov_in, "cov_in", f32),
        _ptr(state_out, "state_out", f32), _ptr(cov_out, "cov_out", f32),
        _ptr(charge, "charge", i8), _ptr(hit, "hit", f32), _ptr(hit_cov, "hit_cov", f32),
        _ptr(surf, "surf", f32), int(surf_per_track), _ptr(status, "status", u8),
        _stream(stream))
    _check(rc)


def kf_p2z_propagate_update(params, layout, state_in, cov_in, state_out, cov_out, charge, hit,
                            hit_cov, z_surf, surf_per_track=0, status=None, stream=None):
    """C-ABI kf_p2z_propagate_update (include/kf.h); raises KfError on failure."""
    _step("kf_p2z_propagate_update", params, layout, state_in, cov_in, state_out, cov_out,
          charge, hit, hit_cov, z_surf, surf_per_track, status, stream)


def kf_p2r_propagate_update(params, layout, state_in, cov_in, state_out, cov_out, charge, hit,
                            hit_cov, r_surf, surf_per_track=0, status=None, stream=None):
    """C-ABI kf_p2r_propagate_update (include/kf.h); raises KfError on failure."""
    _step("kf_p2r_propagate_update", params, layout, state_in, cov_in, state_out, cov_out,
          charge, hit, hit_cov, r_surf, surf_per_track, status, stream)


def _host_ptr(t, name: str, dtype: torch.dtype):
    if t is None:
        return None
    if isinstance(t, int):
        return t
    if t.is_cuda:
        raise ValueError(f"{name}: the host-array call takes CPU tensors")
    if t.dtype != dtype or not t.is_contiguous():
        raise TypeError(f"{name}: expected a contiguous {dtype} tensor")
    return t.data_ptr()


def _step_host(fn_name, params, layout, state_in, cov_in, state_out, cov_out, charge, hit,
               hit_cov, surf, surf_per_track, status, workspace, chunk_tracks, stream):
    lib = load()
    f32, i8, u8 = torch.float32, torch.int8, torch.uint8
    ws = _ptr(workspace, "workspace")
    if isinstance(workspace, torch.Tensor):
        ws_bytes = workspace.numel() * workspace.element_size()
    else:  # a raw pointer: its extent is checked by the library; None: no workspace
        ws_bytes = int(1 << 62) if isinstance(workspace, int) else 0
    rc = getattr(lib, fn_name)(
        ctypes.byref(params), layout,
        _host_ptr(state_in, "state_in", f32), _host_ptr(cov_in, "cov_in", f32),
        _host_ptr(state_out, "state_out", f32), _host_ptr(cov_out, "cov_out", f32),
        _host_ptr(charge, "charge", i8), _host_ptr(hit, "hit", f32),
        _host_ptr(hit_cov, "hit_cov", f32), _host_ptr(surf, "surf", f32), int(surf_per_track),
        _host_ptr(status, "status", u8), ws, ws_bytes, int(chunk_tracks), _stream(stream))
    _check(rc)


def kf_p2z_propagate_update_host(params, layout, state_in, cov_in, state_out, cov_out, charge,
                                 hit, hit_cov, z_surf, surf_per_track=0, status=None,
                                 workspace=None, chunk_tracks=0, stream=None):
    """C-ABI kf_p2z_propagate_update_host: host arrays in and out."""
    _step_host("kf_p2z_propagate_update_host", params, layout, state_in, cov_in, state_out,
               cov_out, charge, hit, hit_cov, z_surf, surf_per_track, status, workspace,
               chunk_tracks, stream)


def kf_p2r_propagate_update_host(params, layout, state_in, cov_in, state_out, cov_out, charge,
                                 hit, hit_cov, r_surf, surf_per_track=0, status=None,
                                 workspace=None, chunk_tracks=0, stream=None):
    """C-ABI kf_p2r_propagate_update_host: host arrays in and out."""
    _step_host("kf_p2r_propagate_update_host", params, layout, state_in, cov_in, state_out,
               cov_out, charge, hit, hit_cov, r_surf, surf_per_track, status, workspace,
               chunk_tracks, stream)


KF_P2Z, KF_P2R = 0, 1
KF_NOALLOC_MAX_CHUNK = 32768


class PreparedStep:
    """kf_p2z_propagate_update / kf_p2r_propagate_update with the arguments
    checked and marshalled once; each call launches the step again on the
    same arrays, on the given stream or the current one.  The tensors are
    kept referenced for the object's lifetime and must not be resized.  For
    loops over small batches, where the plain wrapper's per-call checks and
    conversions cost several times the C call itself."""

    def __init__(self, kind, params, layout, state_in, cov_in, state_out, cov_out, charge, hit,
                 hit_cov, surf, surf_per_track=0, status=None):
        lib = load()
        self._fn = lib.kf_p2z_propagate_update if kind == KF_P2Z else lib.kf_p2r_propagate_update
        f32, i8, u8 = torch.float32, torch.int8, torch.uint8
        self._params = params
        self._keep = (state_in, cov_in, state_out, cov_out, charge, hit, hit_cov, surf, status)
        self._args = (ctypes.byref(params), layout,
                      _ptr(state_in, "state_in", f32), _ptr(cov_in, "cov_in", f32),
                      _ptr(state_out, "state_out", f32), _ptr(cov_out, "cov_out", f32),
                      _ptr(charge, "charge", i8), _ptr(hit, "hit", f32),
                      _ptr(hit_cov, "hit_cov", f32), _ptr(surf, "surf", f32),
                      int(surf_per_track), _ptr(status, "status", u8))
        self._dev = state_in.device.index if state_in.device.index is not None else 0
        self._raw = getattr(torch._C, "_cuda_getCurrentRawStream", None)

    def __call__(self, stream=None):
        if stream is None:
            s = self._raw(self._dev) if self._raw is not None else _stream(None)
        else:
            s = _stream(stream)
        rc = self._fn(*self._args, s)
        if rc != KF_OK:
            _check(rc)


def kf_propagate_update_host_noalloc(kind, params, layout, state_in, cov_in, state_out, cov_out,
                                     charge, hit, hit_cov, surf, surf_per_track=0, status=None,
                                     chunk_tracks=0, stream=None):
    """C-ABI kf_propagate_update_host_noalloc: host arrays in and out, staged
    through the library's fixed device buffer (no device allocation)."""
    lib = load()
    f32, i8, u8 = torch.float32, torch.int8, torch.uint8
    rc = lib.kf_propagate_update_host_noalloc(
        int(kind), ctypes.byref(params), layout,
        _host_ptr(state_in, "state_in", f32), _host_ptr(cov_in, "cov_in", f32),
        _host_ptr(state_out, "state_out", f32), _host_ptr(cov_out, "cov_out", f32),
        _host_ptr(charge, "charge", i8), _host_ptr(hit, "hit", f32),
        _host_ptr(hit_cov, "hit_cov", f32), _host_ptr(surf, "surf", f32), int(surf_per_track),
        _host_ptr(status, "status", u8), int(chunk_tracks), _stream(stream))
    _check(rc)


def kf_host_workspace_bytes(layout, chunk_tracks: int = 0) -> int:
    return int(load().kf_host_workspace_bytes(layout, int(chunk_tracks)))


def make_layers(kinds, pos):
    arr = (kf_layer * len(kinds))()
    for l, (k, z) in enumerate(zip(kinds, pos)):
        arr[l].kind = int(k)
        arr[l].pos = float(z)
    return arr


def kf_kalman_chain(params, layout, state, cov, charge, hits, hit_covs, layers, status=None,
                    stream=None):
    """C-ABI kf_kalman_chain (in place on state/cov); `layers` from make_layers()."""
    lib = load()
    f32, i8, u8 = torch.float32, torch.int8, torch.uint8
    rc = lib.kf_kalman_chain(ctypes.byref(params), layout, _ptr(state, "state", f32),
                             _ptr(cov, "cov", f32), _ptr(charge, "charge", i8),
                             _ptr(hits, "hits", f32), _ptr(hit_covs, "hit_covs", f32),
                             layers, len(layers), _ptr(status, "status", u8), _stream(stream))
    _check(rc)


def kf_propagate_update_compressed(kind, params, layout, state_in, sigma_in, rho_in, state_out,
                                   sigma_out, rho_out, charge, hit, hit_cov, surf,
                                   surf_per_track=0, status=None, stream=None):
    """C-ABI kf_propagate_update_compressed; rho tensors hold float16 (or int16 bits)."""
    lib = load()
    f32, i8, u8 = torch.float32, torch.int8, torch.uint8
    rc = lib.kf_propagate_update_compressed(
        int(kind), ctypes.byref(params), layout, _ptr(state_in, "state_in", f32),
        _ptr(sigma_in, "sigma_in", f32), _ptr(rho_in, "rho_in", torch.float16),
        _ptr(state_out, "state_out", f32), _ptr(sigma_out, "sigma_out", f32),
        _ptr(rho_out, "rho_out", torch.float16), _ptr(charge, "charge", i8),
        _ptr(hit, "hit", f32), _ptr(hit_cov, "hit_cov", f32), _ptr(surf, "surf", f32),
        int(surf_per_track), _ptr(status, "status", u8), _stream(stream))
    _check(rc)


def to_device_rho(rho: np.ndarray, layout: kf_layout, device) -> torch.Tensor:
    """[15, n] float16 correlations -> the compressed store's rho array in
    `layout` (FP16 pairs, see kf_propagate_update_compressed) on `device`."""
    width = layout.width if layout.kind == KF_AOSOA else None
    return torch.from_numpy(W.rho_to_layout(rho, width).copy()).to(device)


def from_device_rho(t: torch.Tensor, n: int, layout: kf_layout) -> np.ndarray:
    """The compressed store's rho array in `layout` -> [15, n] float16."""
    width = layout.width if layout.kind == KF_AOSOA else None
    return W.rho_from_layout(t.cpu().numpy(), n, width)


KF_STEP_AUTO, KF_STEP_DIRECT, KF_STEP_STAGED = 0, 1, 2
KF_DEVERR_TIMEOUT = 1


def kf_set_step_kernel(mode: int) -> None:
    """C-ABI kf_set_step_kernel: KF_STEP_AUTO / KF_STEP_DIRECT / KF_STEP_STAGED."""
    _check(load().kf_set_step_kernel(int(mode)))


KF_CHAIN_REDO_LIST, KF_CHAIN_REDO_SPAN = 0, 1


def kf_set_chain_redo(mode: int) -> None:
    """C-ABI kf_set_chain_redo: KF_CHAIN_REDO_LIST / KF_CHAIN_REDO_SPAN."""
    _check(load().kf_set_chain_redo(int(mode)))


def kf_set_staged_ctas_per_sm(ctas: int) -> None:
    """C-ABI kf_set_staged_ctas_per_sm: 1..3 CTAs per SM under KF_STEP_STAGED, 0 = default."""
    _check(load().kf_set_staged_ctas_per_sm(int(ctas)))


KF_HOST_AUTO, KF_HOST_COPY, KF_HOST_DIRECT = 0, 1, 2


def kf_set_host_path(mode: int) -> None:
    """C-ABI kf_set_host_path: KF_HOST_AUTO / KF_HOST_COPY / KF_HOST_DIRECT."""
    _check(load().kf_set_host_path(int(mode)))


def kf_set_device_wait_limit(polls: int) -> None:
    """C-ABI kf_set_device_wait_limit: polls before a staged kernel's compute
    warps give up a tile wait (0 .. 2^24; -1 = the default)."""
    _check(load().kf_set_device_wait_limit(int(polls)))


def kf_take_device_error() -> int:
    """C-ABI kf_take_device_error: read and clear the device error word."""
    v = ctypes.c_uint(0)
    _check(load().kf_take_device_error(ctypes.byref(v)))
    return int(v.value)


def kf_version() -> int:
    return int(load().kf_version())


def kf_last_error_string() -> str:
    return load().kf_last_error_string().decode()


# ------------------------------------------------------------ device batches

@dataclasses.dataclass
class DeviceBatch:
    """One workload resident on the GPU in a given layout (plumbing only)."""
    kind: int
    n: int
    layout: kf_layout
    state_in: torch.Tensor
    cov_in: torch.Tensor
    state_out: torch.Tensor
    cov_out: torch.Tensor
    charge: torch.Tensor
    hit: torch.Tensor
    hit_cov: torch.Tensor
    surf: torch.Tensor
    status: torch.Tensor
    bz: float

    def prepare(self, precision: int = KF_FP32) -> PreparedStep:
        """A PreparedStep on this batch's current tensors (out of place)."""
        return PreparedStep(KF_P2Z if self.kind == W.P2Z else KF_P2R,
                            make_params(self.bz, precision), self.layout, self.state_in,
                            self.cov_in, self.state_out, self.cov_out, self.charge, self.hit,
                            self.hit_cov, self.surf, int(self.surf.numel() > 1), self.status)

    def run(self, precision: int = KF_FP32, stream=None, in_place: bool = False):
        fn = kf_p2z_propagate_update if self.kind == W.P2Z else kf_p2r_propagate_update
        so = self.state_in if in_place else self.state_out
        co = self.cov_in if in_place else self.cov_out
        fn(make_params(self.bz, precision), self.layout, self.state_in, self.cov_in, so, co,
           self.charge, self.hit, self.hit_cov, self.surf, int(self.surf.numel() > 1),
           self.status, stream)

    def download(self):
        """Results as SoA numpy arrays: (state [6,n], cov [21,n], status [n])."""
        return (from_device(self.state_out, 6, self.n, self.layout),
                from_device(self.cov_out, 21, self.n, self.layout),
                self.status.cpu().numpy())

    def nbytes(self) -> int:
        return sum(t.numel() * t.element_size() for t in
                   (self.state_in, self.cov_in, self.state_out, self.cov_out, self.charge,
                    self.hit, self.hit_cov, self.surf, self.status))


def to_device(a: np.ndarray, layout: kf_layout, device) -> torch.Tensor:
    """[C, n] float32 SoA -> a flat device tensor in `layout`."""
    a = np.ascontiguousarray(a, dtype=np.float32)
    if layout.kind == KF_AOSOA:
        a = W.to_aosoa(a, layout.width)
    return torch.from_numpy(a.reshape(-1).copy()).to(device)


def from_device(t: torch.Tensor, C: int, n: int, layout: kf_layout) -> np.ndarray:
    a = t.cpu().numpy()
    if layout.kind == KF_AOSOA:
        nb = W.aosoa_blocks(n, layout.width)
        return W.from_aosoa(a.reshape(nb, C, layout.width), n)
    return a.reshape(C, n)


def upload(w: W.Workload, layout_kind: int = KF_SOA, width: int = 32, device="cuda",
           surf_per_track: Optional[np.ndarray] = None) -> DeviceBatch:
    lay = make_layout(layout_kind, width, w.n)
    st_in = to_device(w.state, lay, device)
    cv_in = to_device(w.cov, lay, device)
    if surf_per_track is None and np.ndim(w.surf) > 0:
        surf_per_track = w.surf
    surf = (torch.tensor([w.surf], dtype=torch.float32, device=device) if surf_per_track is None
            else torch.from_numpy(np.ascontiguousarray(surf_per_track, dtype=np.float32)).to(device))
    return DeviceBatch(
        kind=w.kind, n=w.n, layout=lay, state_in=st_in, cov_in=cv_in,
        state_out=torch.empty_like(st_in), cov_out=torch.empty_like(cv_in),
        charge=torch.from_numpy(np.ascontiguousarray(w.charge)).to(device),
        hit=to_device(w.hit, lay, device), hit_cov=to_device(w.hitcov, lay, device),
        surf=surf, status=torch.zeros(w.n, dtype=torch.uint8, device=device), bz=w.bz)


@dataclasses.dataclass
class HostBatch:
    """One workload in pinned host memory for the host-array calls."""
    kind: int
    n: int
    layout: kf_layout
    state_in: torch.Tensor
    cov_in: torch.Tensor
    state_out: torch.Tensor
    cov_out: torch.Tensor
    charge: torch.Tensor
    hit: torch.Tensor
    hit_cov: torch.Tensor
    surf: torch.Tensor
    status: torch.Tensor
    workspace: torch.Tensor
    bz: float
    chunk_tracks: int = 0

    def run(self, precision: int = KF_FP32, stream=None):
        fn = kf_p2z_propagate_update_host if self.kind == W.P2Z else kf_p2r_propagate_update_host
        fn(make_params(self.bz, precision), self.layout, self.state_in, self.cov_in,
           self.state_out, self.cov_out, self.charge, self.hit, self.hit_cov, self.surf,
           int(self.surf.numel() > 1), self.status, self.workspace, self.chunk_tracks, stream)

    def h2d_bytes(self) -> int:
        return sum(t.numel() * t.element_size() for t in
                   (self.state_in, self.cov_in, self.charge, self.hit, self.hit_cov, self.surf))

    def d2h_bytes(self) -> int:
        return sum(t.numel() * t.element_size() for t in (self.state_out, self.cov_out,
                                                          self.status))

    def download(self):
        lay = self.layout

        def conv(t, C):
            a = t.numpy()
            if lay.kind == KF_AOSOA:
                return W.from_aosoa(a.reshape(W.aosoa_blocks(self.n, lay.width), C, lay.width),
                                    self.n)
            return a.reshape(C, self.n)
        return conv(self.state_out, 6), conv(self.cov_out, 21), self.status.numpy().copy()


def host_upload(w: W.Workload, layout_kind: int = KF_SOA, width: int = 32, device="cuda",
                chunk_tracks: int = 0, pinned: bool = True) -> HostBatch:
    lay = make_layout(layout_kind, width, w.n)

    def host(a):
        a = np.ascontiguousarray(a, dtype=np.float32)
        if lay.kind == KF_AOSOA:
            a = W.to_aosoa(a, lay.width)
        t = torch.from_numpy(a.reshape(-1).copy())
        return t.pin_memory() if pinned else t

    st_in, cv_in = host(w.state), host(w.cov)
    st_out = torch.empty_like(st_in, pin_memory=pinned)
    cv_out = torch.empty_like(cv_in, pin_memory=pinned)
    q = torch.from_numpy(np.ascontiguousarray(w.charge))
    status = torch.zeros(w.n, dtype=torch.uint8)
    surf = (torch.tensor([w.surf], dtype=torch.float32) if np.ndim(w.surf) == 0
            else torch.from_numpy(np.ascontiguousarray(w.surf, dtype=np.float32)))
    if pinned:
        surf = surf.pin_memory()
        q, status = q.pin_memory(), status.pin_memory()
    ws_bytes = kf_host_workspace_bytes(lay, chunk_tracks)
    ws = torch.empty(ws_bytes, dtype=torch.uint8, device=device)
    return HostBatch(kind=w.kind, n=w.n, layout=lay, state_in=st_in, cov_in=cv_in,
                     state_out=st_out, cov_out=cv_out, charge=q, hit=host(w.hit),
                     hit_cov=host(w.hitcov), surf=surf, status=status, workspace=ws, bz=w.bz,
                     chunk_tracks=chunk_tracks)


@dataclasses.dataclass
class DeviceChain:
    """A chain workload resident on the GPU (plumbing only)."""
    n: int
    layout: kf_layout
    layers: object
    state0: torch.Tensor    # start state, kept to reset between runs
    cov0: torch.Tensor
    state: torch.Tensor     # worked on in place
    cov: torch.Tensor
    charge: torch.Tensor
    hits: torch.Tensor      # L consecutive hit arrays
    hit_covs: torch.Tensor
    status: torch.Tensor
    bz: float
    f3: int
    f6: int

    def reset(self):
        self.state.copy_(self.state0)
        self.cov.copy_(self.cov0)

    def run(self, precision: int = KF_FP32, stream=None):
        kf_kalman_chain(make_params(self.bz, precision), self.layout, self.state, self.cov,
                        self.charge, self.hits, self.hit_covs, self.layers, self.status, stream)

    def run_plain(self, precision: int = KF_FP32, stream=None):
        """The same chain as L single-step launches, in place."""
        p = make_params(self.bz, precision)
        for l in range(len(self.layers)):
            fn = kf_p2z_propagate_update if self.layers[l].kind == 0 else kf_p2r_propagate_update
            surf = self._surf[l]
            fn(p, self.layout, self.state, self.cov, self.state, self.cov, self.charge,
               self.hits[l * self.f3:(l + 1) * self.f3], self.hit_covs[l * self.f6:(l + 1) * self.f6],
               surf, 0, self.status, stream)

    def download(self):
        return (from_device(self.state, 6, self.n, self.layout),
                from_device(self.cov, 21, self.n, self.layout), self.status.cpu().numpy())


def chain_upload(cw, layout_kind: int = KF_AOSOA, width: int = 32, device="cuda") -> DeviceChain:
    lay = make_layout(layout_kind, width, cw.n)
    st = to_device(cw.state, lay, device)
    cv = to_device(cw.cov, lay, device)
    hits = torch.cat([to_device(cw.hit[l], lay, device) for l in range(cw.L)])
    hcs = torch.cat([to_device(cw.hitcov[l], lay, device) for l in range(cw.L)])
    f3 = hits.numel() // cw.L
    f6 = hcs.numel() // cw.L
    dc = DeviceChain(n=cw.n, layout=lay, layers=make_layers(cw.kinds, cw.pos), state0=st,
                     cov0=cv, state=st.clone(), cov=cv.clone(),
                     charge=torch.from_numpy(np.ascontiguousarray(cw.charge)).to(device),
                     hits=hits, hit_covs=hcs,
                     status=torch.zeros(cw.n, dtype=torch.uint8, device=device), bz=cw.bz,
                     f3=f3, f6=f6)
    dc._surf = [torch.tensor([float(z)], dtype=torch.float32, device=device) for z in cw.pos]
    return dc


# ------------------------------------------------------------ serving loop

class Server:
    """Thin wrapper over kf_server_* (C ABI): one object per server."""

    def __init__(self, bz, kinds, pos, arena: torch.Tensor, max_events_in_flight=64,
                 precision=KF_FP32):
        lib = load()
        if not arena.is_cuda:
            raise ValueError("arena must be a CUDA tensor")
        cfg = kf_server_config()
        cfg.bz = float(bz)
        cfg.precision = int(precision)
        cfg.L = len(kinds)
        for l, (k, z) in enumerate(zip(kinds, pos)):
            cfg.layers[l].kind = int(k)
            cfg.layers[l].pos = float(z)
        cfg.arena = arena.data_ptr()
        cfg.arena_bytes = arena.numel() * arena.element_size()
        cfg.max_events_in_flight = int(max_events_in_flight)
        cfg.device = arena.device.index or 0
        self._arena = arena
        self._h = ctypes.c_void_p()
        _check(lib.kf_server_create(ctypes.byref(cfg), ctypes.byref(self._h)))
        self.L = cfg.L
        self._keep = {}

    def submit(self, state, cov, charge, hits, hit_covs, state_out, cov_out, status_out=None):
        """Host tensors (SoA per event).  Returns a ticket."""
        t = ctypes.c_uint64(0)
        n = state.shape[-1]
        args = [state, cov, charge, hits, hit_covs, state_out, cov_out, status_out]
        ptrs = [None if a is None else _host_ptr(a, "event array", a.dtype) for a in args]
        _check(load().kf_server_submit(self._h, int(n), *ptrs, ctypes.byref(t)))
        self._keep[t.value] = args
        return t.value

    def poll(self, ticket) -> bool:
        d = ctypes.c_int32(0)
        _check(load().kf_server_poll(self._h, ctypes.c_uint64(ticket), ctypes.byref(d)))
        return bool(d.value)

    def wait(self, ticket, timeout_s=60.0):
        _check(load().kf_server_wait(self._h, ctypes.c_uint64(ticket), float(timeout_s)))
        self._keep.pop(ticket, None)

    def pause(self, paused=True):
        _check(load().kf_server_pause(self._h, int(bool(paused))))

    def stats(self) -> dict:
        st = kf_server_stats()
        _check(load().kf_server_get_stats(self._h, ctypes.byref(st)))
        return {f: getattr(st, f) for f, _ in st._fields_}

    def reset_stats(self):
        _check(load().kf_server_reset_stats(self._h))

    def close(self):
        if self._h:
            _check(load().kf_server_destroy(self._h))
            self._h = ctypes.c_void_p()


def kf_server_event_bytes(n: int, L: int) -> int:
    return int(load().kf_server_event_bytes(int(n), int(L)))


# ---------------------------------------------------------------- tuning

def _tuning_dict(t: kf_tuning) -> dict:
    return {"step_kernel": {1: "direct", 2: "staged"}.get(t.step_kernel, t.step_kernel),
            "threads": t.threads, "ctas_per_sm": t.ctas_per_sm, "ms": t.ms}


def autotune_step(batch: "DeviceBatch", precision: int = KF_FP32) -> dict:
    """kf_autotune_step on a resident batch (outputs to its separate arrays)."""
    t = kf_tuning()
    f32, i8, u8 = torch.float32, torch.int8, torch.uint8
    kind = KF_P2Z if batch.kind == W.P2Z else KF_P2R
    _check(load().kf_autotune_step(
        kind, ctypes.byref(make_params(batch.bz, precision)), batch.layout,
        _ptr(batch.state_in, "state_in", f32), _ptr(batch.cov_in, "cov_in", f32),
        _ptr(batch.state_out, "state_out", f32), _ptr(batch.cov_out, "cov_out", f32),
        _ptr(batch.charge, "charge", i8), _ptr(batch.hit, "hit", f32),
        _ptr(batch.hit_cov, "hit_cov", f32), _ptr(batch.surf, "surf", f32),
        int(batch.surf.numel() > 1), _ptr(batch.status, "status", u8), _stream(None),
        ctypes.byref(t)))
    return _tuning_dict(t)


def autotune_chain(chain: "DeviceChain", precision: int = KF_FP32) -> dict:
    """kf_autotune_chain on a resident chain workload (its state is left as it was)."""
    t = kf_tuning()
    f32, i8, u8 = torch.float32, torch.int8, torch.uint8
    st_scr, cv_scr = torch.empty_like(chain.state), torch.empty_like(chain.cov)
    _check(load().kf_autotune_chain(
        ctypes.byref(make_params(chain.bz, precision)), chain.layout,
        _ptr(chain.state, "state", f32), _ptr(chain.cov, "cov", f32),
        _ptr(chain.charge, "charge", i8), _ptr(chain.hits, "hits", f32),
        _ptr(chain.hit_covs, "hit_covs", f32), chain.layers, len(chain.layers),
        _ptr(chain.status, "status", u8), st_scr.data_ptr(), cv_scr.data_ptr(), _stream(None),
        ctypes.byref(t)))
    return _tuning_dict(t)


def autotune_export() -> str:
    lib = load()
    n = ctypes.c_int64(0)
    _check(lib.kf_autotune_export(None, 0, ctypes.byref(n)))
    buf = ctypes.create_string_buffer(n.value + 1)
    _check(lib.kf_autotune_export(buf, n.value + 1, ctypes.byref(n)))
    return buf.value.decode()


def autotune_import(text: str) -> None:
    _check(load().kf_autotune_import(text.encode()))


def autotune_clear() -> None:
    _check(load().kf_autotune_clear())
