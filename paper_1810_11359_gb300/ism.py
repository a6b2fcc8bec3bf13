"""Thin Python binding of libism (include/ism.h).

Argument marshalling only: every step of the simulation runs in the CUDA
kernels of libism.so.  PyTorch provides device memory and the current CUDA
stream.  The functions carry the names of the C entry points.  There is no
CPU fallback: if the library has not been built, or no GPU is present, calls
raise.
"""
from __future__ import annotations

import ctypes
import os
import threading
from typing import Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libism.so")

ISM_OK = 0
STATUS_NAMES = {0: "ISM_OK", 1: "ISM_ERR_INVALID_ARG", 2: "ISM_ERR_INFEASIBLE", 3: "ISM_ERR_WORKSPACE_TOO_SMALL",
                4: "ISM_ERR_OOM", 5: "ISM_ERR_CUDA", 6: "ISM_ERR_TIMEOUT", 7: "ISM_ERR_DEVICE_CHECK",
                8: "ISM_ERR_UNSUPPORTED", 9: "ISM_ERR_CANCELLED"}
PRECISIONS = {"fp32": 0, "fp16x2": 1, "bf16x2": 2, "lut": 3, "fp32_direct": 4, "lut_tex": 5}
# receiver polar patterns (ism_mic_pattern): g = alpha + (1 - alpha) cos(theta)
MIC_PATTERNS = {"omni": 0, "subcardioid": 1, "cardioid": 2, "hypercardioid": 3, "bidirectional": 4}
ENVELOPES = {"sabine": 0, "lj": 1}   # ism_envelope: power envelope of the diffuse tail
ISM_ERR_TIMEOUT_CODE = 6
ISM_DEVICE_FLAG_POSITION = 1   # include/ism.h ISM_DEVICE_FLAG_*
ISM_DEVICE_FLAG_BIN = 2
ISM_DEVICE_FLAG_BETA = 4
STATUS_CODES = {v: k for k, v in STATUS_NAMES.items()}
DEVICE_FLAG_POSITION = 1
DEVICE_FLAG_BIN = 2


class IsmError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


class ism_room(ctypes.Structure):
    _fields_ = [("L", ctypes.c_double * 3), ("beta", ctypes.c_float * 6), ("c", ctypes.c_float)]


class ism_job(ctypes.Structure):
    _fields_ = [("room", ism_room),
                ("pos_src", ctypes.c_void_p), ("n_src", ctypes.c_int),
                ("pos_rcv", ctypes.c_void_p), ("n_rcv", ctypes.c_int),
                ("nb_img", ctypes.c_int * 3),
                ("Tmax", ctypes.c_float), ("fs", ctypes.c_float), ("Tdiff", ctypes.c_float), ("Tw", ctypes.c_float),
                ("seed", ctypes.c_uint64),
                ("out", ctypes.c_void_p), ("env_amp", ctypes.c_void_p),
                ("mic_pattern", ctypes.c_int), ("orient_rcv", ctypes.c_void_p), ("beta_dev", ctypes.c_void_p),
                ("envelope", ctypes.c_int)]


class ism_grad_job(ctypes.Structure):
    _fields_ = [("job", ism_job), ("grad_out", ctypes.c_void_p), ("grad_beta", ctypes.c_void_p),
                ("grad_src", ctypes.c_void_p), ("grad_rcv", ctypes.c_void_p)]


class ism_server_config(ctypes.Structure):
    _fields_ = [("hbm_budget", ctypes.c_size_t), ("host_budget", ctypes.c_size_t), ("max_inflight", ctypes.c_int),
                ("max_batch", ctypes.c_int), ("device", ctypes.c_int), ("prec", ctypes.c_int)]


class ism_server_stats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_longlong), ("completed", ctypes.c_longlong), ("failed", ctypes.c_longlong),
                ("batches", ctypes.c_longlong), ("dev_in_use", ctypes.c_size_t), ("dev_peak", ctypes.c_size_t),
                ("host_in_use", ctypes.c_size_t), ("inflight", ctypes.c_int), ("queued", ctypes.c_int),
                ("inflight_peak", ctypes.c_int)]


# Every symbol include/ism.h declares, with its ctypes signature.
_P = ctypes.POINTER
_SIGS = {
    "ism_status_string": (ctypes.c_char_p, [ctypes.c_int]),
    "ism_last_error_message": (ctypes.c_char_p, []),
    "ism_version": (ctypes.c_int, []),
    "ism_rir_length": (ctypes.c_int, [ctypes.c_float, ctypes.c_float, _P(ctypes.c_int)]),
    "ism_workspace_size": (ctypes.c_int, [_P(ism_room), ctypes.c_int, ctypes.c_int, _P(ctypes.c_int), ctypes.c_float,
                                          ctypes.c_float, ctypes.c_float, ctypes.c_float, ctypes.c_int,
                                          _P(ctypes.c_size_t)]),
    "ism_host_workspace_size": (ctypes.c_int, [_P(ism_room), ctypes.c_int, ctypes.c_int, _P(ctypes.c_int),
                                               ctypes.c_float, ctypes.c_float, ctypes.c_float, ctypes.c_float,
                                               ctypes.c_int, _P(ctypes.c_size_t)]),
    "ism_simulate": (ctypes.c_int, [_P(ism_room), ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_int,
                                    _P(ctypes.c_int), ctypes.c_float, ctypes.c_float, ctypes.c_float, ctypes.c_float,
                                    ctypes.c_int, ctypes.c_uint64, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t,
                                    ctypes.c_void_p]),
    "ism_simulate_host": (ctypes.c_int, [_P(ism_room), ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_int,
                                         _P(ctypes.c_int), ctypes.c_float, ctypes.c_float, ctypes.c_float,
                                         ctypes.c_float, ctypes.c_int, ctypes.c_uint64, ctypes.c_void_p,
                                         ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p]),
    "ism_simulate_noalloc": (ctypes.c_int, [_P(ism_room), ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p,
                                            ctypes.c_int, _P(ctypes.c_int), ctypes.c_float, ctypes.c_float,
                                            ctypes.c_float, ctypes.c_float, ctypes.c_int, ctypes.c_uint64,
                                            ctypes.c_void_p, ctypes.c_void_p]),
    "ism_workspace_status": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, _P(ctypes.c_uint32)]),
    "ism_batch_workspace_size": (ctypes.c_int, [_P(ism_job), ctypes.c_int, ctypes.c_int, _P(ctypes.c_size_t)]),
    "ism_simulate_batch": (ctypes.c_int, [_P(ism_job), ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ctypes.c_size_t,
                                          ctypes.c_void_p]),
    "ism_server_create": (ctypes.c_int, [_P(ism_server_config), _P(ctypes.c_void_p)]),
    "ism_server_submit": (ctypes.c_int, [ctypes.c_void_p, _P(ism_job), _P(ctypes.c_uint64)]),
    "ism_server_submit_batch": (ctypes.c_int, [ctypes.c_void_p, _P(ism_job), ctypes.c_int, _P(ctypes.c_uint64)]),
    "ism_server_poll": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_uint64, _P(ctypes.c_int)]),
    "ism_server_wait": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_uint64, ctypes.c_double, _P(ctypes.c_double)]),
    "ism_server_stats_read": (ctypes.c_int, [ctypes.c_void_p, _P(ism_server_stats)]),
    "ism_server_destroy": (ctypes.c_int, [ctypes.c_void_p]),
    "ism_backward_workspace_size": (ctypes.c_int, [_P(ism_grad_job), ctypes.c_int, _P(ctypes.c_size_t)]),
    "ism_simulate_backward_batch": (ctypes.c_int, [_P(ism_grad_job), ctypes.c_int, ctypes.c_void_p, ctypes.c_size_t,
                                                   ctypes.c_void_p]),
    "ism_simulate_backward": (ctypes.c_int, [_P(ism_room), ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p,
                                             ctypes.c_int, _P(ctypes.c_int), ctypes.c_float, ctypes.c_float,
                                             ctypes.c_float, ctypes.c_float, ctypes.c_void_p, ctypes.c_void_p,
                                             ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t,
                                             ctypes.c_void_p]),
    "ism_diffuse_noise": (ctypes.c_int, [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_int,
                                         ctypes.c_void_p, ctypes.c_void_p]),
    "ism_auralize": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_int, ctypes.c_int,
                                    ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "ism_auralize_workspace_size": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                                   ctypes.c_int, _P(ctypes.c_size_t)]),
    "ism_auralize_ex": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_int, ctypes.c_int,
                                       ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p,
                                       ctypes.c_size_t, ctypes.c_void_p]),
    "ism_t60_sabine": (ctypes.c_int, [_P(ctypes.c_double), _P(ctypes.c_double), _P(ctypes.c_double)]),
    "ism_beta_sabine": (ctypes.c_int, [_P(ctypes.c_double), ctypes.c_double, _P(ctypes.c_double), ctypes.c_int,
                                       _P(ctypes.c_double)]),
    "ism_beta_sabine_device": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int,
                                              ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "ism_nb_img_from_t": (ctypes.c_int, [ctypes.c_double, _P(ctypes.c_double), ctypes.c_double, ctypes.c_double,
                                         _P(ctypes.c_int)]),
    "ism_att2t_sabine": (ctypes.c_int, [ctypes.c_double, ctypes.c_double, _P(ctypes.c_double)]),
    "ism_set_lanes": (ctypes.c_int, [ctypes.c_int]),
    "ism_profile_enable": (ctypes.c_int, [ctypes.c_int]),
    "ism_profile_reset": (ctypes.c_int, []),
    "ism_profile_read": (ctypes.c_int, [ctypes.c_int, _P(ctypes.c_double), _P(ctypes.c_longlong),
                                        _P(ctypes.c_longlong)]),
}

STAGES = ["geometry", "enum_count", "scan", "enum_scatter", "accum", "finalize", "tail", "adjoint"]

_lock = threading.Lock()
_lib = None


def load(path: Optional[str] = None):
    """Load libism.so (raises if it has not been built: there is no fallback)."""
    global _lib
    with _lock:
        if _lib is not None and path is None:
            return _lib
        p = path or LIB_PATH
        if not os.path.exists(p):
            raise RuntimeError(f"libism.so not found at {p}: run __graft_entry__.build() "
                               "(python -c 'import __graft_entry__ as g; g.build()')")
        lib = ctypes.CDLL(p)
        for name, (res, args) in _SIGS.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        if path is None:
            _lib = lib
        return lib


def _check(status: int):
    if status != ISM_OK:
        msg = load().ism_last_error_message().decode(errors="replace")
        raise IsmError(status, msg)


def _room(L, beta, c):
    r = ism_room()
    for a in range(3):
        r.L[a] = float(L[a])
    for w in range(6):
        r.beta[w] = float(beta[w])
    r.c = float(c)
    return r


def _nb(nb_img):
    return (ctypes.c_int * 3)(*[int(v) for v in nb_img])


def _torch():
    import torch
    return torch


def _stream_ptr(stream=None):
    torch = _torch()
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


# --------------------------------------------------------------------------- #
# Helpers of Section 4 (host FP64)
# --------------------------------------------------------------------------- #
def _rir_len(T, fs) -> int:
    key = (float(T), float(fs))
    n = _rir_lens.get(key)
    if n is None:
        if len(_rir_lens) > 256:
            _rir_lens.clear()
        n = _rir_lens[key] = ism_rir_length(T, fs)
    return n


def ism_rir_length(T: float, fs: float) -> int:
    n = ctypes.c_int()
    _check(load().ism_rir_length(float(T), float(fs), ctypes.byref(n)))
    return n.value


def ism_t60_sabine(L, beta) -> float:
    Ld = (ctypes.c_double * 3)(*map(float, L))
    bd = (ctypes.c_double * 6)(*map(float, beta))
    t = ctypes.c_double()
    _check(load().ism_t60_sabine(Ld, bd, ctypes.byref(t)))
    return t.value


def ism_beta_sabine(L, T60: float, abs_weights=None, negative: bool = False) -> np.ndarray:
    Ld = (ctypes.c_double * 3)(*map(float, L))
    w = None if abs_weights is None else (ctypes.c_double * 6)(*map(float, abs_weights))
    out = (ctypes.c_double * 6)()
    _check(load().ism_beta_sabine(Ld, float(T60), w, int(bool(negative)), out))
    return np.array(list(out))


def ism_beta_sabine_device(L, T60, abs_weights=None, negative: bool = False):
    """Batched inverse Sabine in FP64 on the GPU: L [n,3], T60 [n] (CUDA float64
    tensors) -> (beta [n,6] float64, status [n] int32)."""
    torch = _torch()
    L = L.contiguous()
    T60 = T60.contiguous()
    n = T60.shape[0]
    beta = torch.empty((n, 6), dtype=torch.float64, device=L.device)
    st = torch.empty((n,), dtype=torch.int32, device=L.device)
    w = None if abs_weights is None else abs_weights.contiguous()
    _check(load().ism_beta_sabine_device(ctypes.c_void_p(L.data_ptr()), ctypes.c_void_p(T60.data_ptr()),
                                         None if w is None else ctypes.c_void_p(w.data_ptr()), int(bool(negative)),
                                         int(n), ctypes.c_void_p(beta.data_ptr()), ctypes.c_void_p(st.data_ptr()),
                                         _stream_ptr()))
    return beta, st


def ism_nb_img_from_t(T: float, L, c: float = 343.0, Tw: float = 4e-3) -> np.ndarray:
    Ld = (ctypes.c_double * 3)(*map(float, L))
    out = (ctypes.c_int * 3)()
    _check(load().ism_nb_img_from_t(float(T), Ld, float(c), float(Tw), out))
    return np.array(list(out), dtype=np.int32)


def ism_att2t_sabine(att_dB: float, T60: float) -> float:
    t = ctypes.c_double()
    _check(load().ism_att2t_sabine(float(att_dB), float(T60), ctypes.byref(t)))
    return t.value


# --------------------------------------------------------------------------- #
# Simulation
# --------------------------------------------------------------------------- #
def ism_workspace_size(L, beta, n_src, n_rcv, nb_img, Tmax, fs, Tdiff=0.0, Tw=0.0, c=343.0,
                       prec: str = "fp32") -> int:
    b = ctypes.c_size_t()
    r = _room(L, beta, c)
    _check(load().ism_workspace_size(ctypes.byref(r), int(n_src), int(n_rcv), _nb(nb_img), float(Tmax), float(fs),
                                     float(Tdiff or 0.0), float(Tw or 0.0), PRECISIONS[prec], ctypes.byref(b)))
    return b.value


def ism_host_workspace_size(L, beta, n_src, n_rcv, nb_img, Tmax, fs, Tdiff=0.0, Tw=0.0, c=343.0,
                            prec: str = "fp32") -> int:
    b = ctypes.c_size_t()
    r = _room(L, beta, c)
    _check(load().ism_host_workspace_size(ctypes.byref(r), int(n_src), int(n_rcv), _nb(nb_img), float(Tmax),
                                          float(fs), float(Tdiff or 0.0), float(Tw or 0.0), PRECISIONS[prec],
                                          ctypes.byref(b)))
    return b.value


class Workspace:
    """Device scratch memory for the library (a uint8 CUDA tensor), grown on demand."""

    def __init__(self, device=None):
        self.device = device
        self.buf = None

    def get(self, nbytes: int):
        torch = _torch()
        if self.buf is None or self.buf.numel() < nbytes:
            dev = self.device if self.device is not None else torch.device("cuda", torch.cuda.current_device())
            self.buf = torch.empty(max(int(nbytes), 256), dtype=torch.uint8, device=dev)
        return self.buf


_default_ws = {}


def _workspace(ws, nbytes):
    torch = _torch()
    if ws is None:
        dev = torch.cuda.current_device()
        ws = _default_ws.setdefault(dev, Workspace())
    return ws.get(nbytes)


def ism_simulate(L, beta, pos_src, pos_rcv, nb_img, Tmax, fs, Tdiff=0.0, Tw=0.0, c=343.0, prec: str = "fp32",
                 seed: int = 0, out=None, workspace: Optional[Workspace] = None, stream=None,
                 mic_pattern: str = "omni", orient_rcv=None, envelope: str = "sabine"):
    """RIRs [n_src, n_rcv, n_S] (FP32 CUDA tensor) for all source/receiver pairs.

    pos_src/pos_rcv: [n,3] positions (CUDA FP32 tensors, or anything
    convertible; copied to the device if needed).  mic_pattern / orient_rcv:
    receiver polar pattern (a MIC_PATTERNS name) and [n_rcv,3] orientations.
    envelope: power envelope of the diffuse tail (an ENVELOPES name)."""
    torch = _torch()
    dev = torch.device("cuda", torch.cuda.current_device())
    ps = torch.as_tensor(pos_src, dtype=torch.float32).to(dev).reshape(-1, 3).contiguous()
    pr = torch.as_tensor(pos_rcv, dtype=torch.float32).to(dev).reshape(-1, 3).contiguous()
    if out is None:
        out = torch.empty((ps.shape[0], pr.shape[0], _rir_len(Tmax, fs)), dtype=torch.float32, device=dev)
    if mic_pattern != "omni" or envelope != "sabine":   # these travel in the job struct: the batch entry point
        orient = None
        if mic_pattern != "omni":
            orient = torch.as_tensor(orient_rcv, dtype=torch.float32).to(dev).reshape(-1, 3).contiguous()
            if orient.shape[0] != pr.shape[0]:
                raise ValueError("orient_rcv needs one vector per receiver")
        job = make_job(L, beta, ps, pr, nb_img, Tmax, fs, out, Tdiff=Tdiff, Tw=Tw, c=c, seed=seed,
                       mic_pattern=mic_pattern, orient_rcv=orient, envelope=envelope)
        ism_simulate_batch([job], prec=prec, workspace=workspace, stream=stream)
        return out
    # the room struct, images per axis, workspace bytes and RIR length of these arguments
    key = (np.asarray(L, np.float64).tobytes(), np.asarray(beta, np.float64).tobytes(),
           np.asarray(nb_img, np.int64).tobytes(), ps.shape[0], pr.shape[0], float(Tmax), float(fs),
           float(Tdiff or 0.0), float(Tw or 0.0), float(c), prec, _lanes_setting[0])
    hit = _dev_sizes.get(key)
    if hit is None:
        if len(_dev_sizes) > 256:
            _dev_sizes.clear()
        hit = _dev_sizes[key] = (_room(L, beta, c), _nb(nb_img),
                                 ism_workspace_size(L, beta, ps.shape[0], pr.shape[0], nb_img, Tmax, fs, Tdiff, Tw,
                                                    c, prec),
                                 _rir_len(Tmax, fs))
    r, nb, nbytes, n_S = hit
    buf = _workspace(workspace, nbytes)
    _check(load().ism_simulate(ctypes.byref(r), ctypes.c_void_p(ps.data_ptr()), int(ps.shape[0]),
                               ctypes.c_void_p(pr.data_ptr()), int(pr.shape[0]), nb, float(Tmax), float(fs),
                               float(Tdiff or 0.0), float(Tw or 0.0), PRECISIONS[prec], int(seed) & (2 ** 64 - 1),
                               ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(buf.data_ptr()),
                               int(buf.numel()), _stream_ptr(stream)))
    return out


_host_sizes = {}     # (arguments) -> (room struct, nb, host-entry workspace bytes, RIR length)
_rir_lens = {}
_dev_sizes = {}      # the same for the device entry point
_lanes_setting = [2]


def ism_simulate_host(L, beta, pos_src, pos_rcv, nb_img, Tmax, fs, Tdiff=0.0, Tw=0.0, c=343.0, prec: str = "fp32",
                      seed: int = 0, out: Optional[np.ndarray] = None, workspace: Optional[Workspace] = None,
                      stream=None) -> np.ndarray:
    """Same as ism_simulate from host (numpy) positions into a host array;
    the copies happen inside the library call (synchronous)."""
    ps = np.ascontiguousarray(pos_src, dtype=np.float32).reshape(-1, 3)
    pr = np.ascontiguousarray(pos_rcv, dtype=np.float32).reshape(-1, 3)
    # the room struct, images per axis, workspace bytes and RIR length of these arguments
    key = (np.asarray(L, np.float64).tobytes(), np.asarray(beta, np.float64).tobytes(),
           np.asarray(nb_img, np.int64).tobytes(), ps.shape[0], pr.shape[0], float(Tmax), float(fs),
           float(Tdiff or 0.0), float(Tw or 0.0), float(c), prec, _lanes_setting[0])
    hit = _host_sizes.get(key)
    if hit is None:
        r = _room(L, beta, c)
        nb = _nb(nb_img)
        b = ctypes.c_size_t()
        _check(load().ism_host_workspace_size(ctypes.byref(r), int(ps.shape[0]), int(pr.shape[0]), nb, float(Tmax),
                                              float(fs), float(Tdiff or 0.0), float(Tw or 0.0), PRECISIONS[prec],
                                              ctypes.byref(b)))
        if len(_host_sizes) > 256:
            _host_sizes.clear()
        hit = _host_sizes[key] = (r, nb, b.value, ism_rir_length(Tmax, fs))
    r, nb, nbytes, n_S = hit
    if out is None:
        out = np.empty((ps.shape[0], pr.shape[0], n_S), dtype=np.float32)
    buf = _workspace(workspace, nbytes)
    _check(load().ism_simulate_host(ctypes.byref(r), ctypes.c_void_p(ps.ctypes.data), int(ps.shape[0]),
                                    ctypes.c_void_p(pr.ctypes.data), int(pr.shape[0]), nb, float(Tmax),
                                    float(fs), float(Tdiff or 0.0), float(Tw or 0.0), PRECISIONS[prec],
                                    int(seed) & (2 ** 64 - 1), ctypes.c_void_p(out.ctypes.data),
                                    ctypes.c_void_p(buf.data_ptr()), int(buf.numel()), _stream_ptr(stream)))
    return out


def ism_simulate_noalloc(L, beta, pos_src, pos_rcv, nb_img, Tmax, fs, Tdiff=0.0, Tw=0.0, c=343.0,
                         prec: str = "fp32", seed: int = 0, out=None, stream=None):
    """ism_simulate in the library's fixed device scratch area: no workspace,
    no device allocation by the library (the output tensor is the caller's).
    Calls must not overlap on the GPU; see include/ism.h."""
    torch = _torch()
    dev = torch.device("cuda", torch.cuda.current_device())
    ps = torch.as_tensor(pos_src, dtype=torch.float32).to(dev).reshape(-1, 3).contiguous()
    pr = torch.as_tensor(pos_rcv, dtype=torch.float32).to(dev).reshape(-1, 3).contiguous()
    n_S = ism_rir_length(Tmax, fs)
    if out is None:
        out = torch.empty((ps.shape[0], pr.shape[0], n_S), dtype=torch.float32, device=dev)
    r = _room(L, beta, c)
    _check(load().ism_simulate_noalloc(ctypes.byref(r), ctypes.c_void_p(ps.data_ptr()), int(ps.shape[0]),
                                       ctypes.c_void_p(pr.data_ptr()), int(pr.shape[0]), _nb(nb_img), float(Tmax),
                                       float(fs), float(Tdiff or 0.0), float(Tw or 0.0), PRECISIONS[prec],
                                       int(seed) & (2 ** 64 - 1), ctypes.c_void_p(out.data_ptr()),
                                       _stream_ptr(stream)))
    return out


def ism_workspace_status(buf, stream=None) -> int:
    flags = ctypes.c_uint32()
    _check(load().ism_workspace_status(ctypes.c_void_p(buf.data_ptr()), _stream_ptr(stream), ctypes.byref(flags)))
    return flags.value


def make_job(L, beta, pos_src, pos_rcv, nb_img, Tmax, fs, out, Tdiff=0.0, Tw=0.0, c=343.0, seed=0,
             env_amp=None, mic_pattern: str = "omni", orient_rcv=None, envelope: str = "sabine") -> ism_job:
    """An ism_job over CUDA tensors (the tensors must stay alive during the call);
    orient_rcv: [n_rcv, 3] CUDA FP32 tensor for a polar pattern; beta: 6 host
    values, or a contiguous FP32 CUDA tensor of 6 read in place (beta_dev)."""
    j = ism_job()
    on_device = hasattr(beta, "data_ptr")
    j.room = _room(L, [0.0] * 6 if on_device else beta, c)
    j.beta_dev = beta.data_ptr() if on_device else None
    j.pos_src = pos_src.data_ptr()
    j.n_src = int(pos_src.shape[0])
    j.pos_rcv = pos_rcv.data_ptr()
    j.n_rcv = int(pos_rcv.shape[0])
    for a in range(3):
        j.nb_img[a] = int(nb_img[a])
    j.Tmax, j.fs, j.Tdiff, j.Tw = float(Tmax), float(fs), float(Tdiff or 0.0), float(Tw or 0.0)
    j.seed = int(seed) & (2 ** 64 - 1)
    j.out = out.data_ptr()
    j.env_amp = None if env_amp is None else env_amp.data_ptr()
    j.mic_pattern = MIC_PATTERNS[mic_pattern]
    j.orient_rcv = None if orient_rcv is None else orient_rcv.data_ptr()
    j.envelope = ENVELOPES[envelope]
    return j


def make_jobs_strided(L, beta, pos_src, pos_rcv, nb_img, Tmax, fs, out, Tdiff=0.0, Tw=0.0, c=343.0, seed=0):
    """B jobs over batched CUDA tensors pos_src [B, S, 3], pos_rcv [B, M, 3],
    out [B, S, M, n_S] (contiguous FP32; they must stay alive during the call):
    one ctypes array filled through a numpy view, without per-room tensor
    views.  L [B, 3], nb_img [B, 3] are host arrays; beta [B, 6] is a host
    array or a contiguous FP32 CUDA tensor (read by the kernels in place:
    ism_job.beta_dev)."""
    B = int(pos_src.shape[0])
    S, M = int(pos_src.shape[1]), int(pos_rcv.shape[1])
    arr = (ism_job * B)()
    v = np.frombuffer(arr, dtype=np.dtype(ism_job), count=B)
    v["room"]["L"] = np.asarray(L, np.float64).reshape(B, 3)
    if hasattr(beta, "data_ptr"):
        v["beta_dev"] = np.uint64(beta.data_ptr()) + np.arange(B, dtype=np.uint64) * np.uint64(24)
    else:
        v["room"]["beta"] = np.asarray(beta, np.float64).reshape(B, 6).astype(np.float32)
    v["room"]["c"] = np.float32(c)
    idx = np.arange(B, dtype=np.uint64)
    v["pos_src"] = np.uint64(pos_src.data_ptr()) + idx * np.uint64(S * 3 * 4)
    v["n_src"] = S
    v["pos_rcv"] = np.uint64(pos_rcv.data_ptr()) + idx * np.uint64(M * 3 * 4)
    v["n_rcv"] = M
    v["nb_img"] = np.asarray(nb_img, np.int32).reshape(B, 3)
    v["Tmax"], v["fs"], v["Tdiff"], v["Tw"] = float(Tmax), float(fs), float(Tdiff or 0.0), float(Tw or 0.0)
    v["seed"] = int(seed) & (2 ** 64 - 1)
    v["out"] = np.uint64(out.data_ptr()) + idx * np.uint64(out[0].numel() * 4)
    return arr


def make_grad_jobs_strided(jobs, grad_out, grad_beta, grad_src, grad_rcv):
    """ism_grad_job array for the jobs of make_jobs_strided: backward reads
    grad_out [B, S, M, n_S] and writes grad_beta [B, 6], grad_src [B, S, 3],
    grad_rcv [B, M, 3] (the jobs' out is not touched; it is set to grad_out)."""
    B = len(jobs)
    arr = (ism_grad_job * B)()
    v = np.frombuffer(arr, dtype=np.dtype(ism_grad_job), count=B)
    v["job"] = np.frombuffer(jobs, dtype=np.dtype(ism_job), count=B)
    idx = np.arange(B, dtype=np.uint64)
    for name, t in (("grad_out", grad_out), ("grad_beta", grad_beta), ("grad_src", grad_src), ("grad_rcv", grad_rcv)):
        v[name] = np.uint64(t.data_ptr()) + idx * np.uint64(t[0].numel() * 4)
    v["job"]["out"] = v["grad_out"]
    return arr


def ism_batch_workspace_size(jobs: Sequence[ism_job], prec: str = "fp32") -> int:
    arr = jobs if isinstance(jobs, ctypes.Array) else (ism_job * len(jobs))(*jobs)
    b = ctypes.c_size_t()
    _check(load().ism_batch_workspace_size(arr, len(jobs), PRECISIONS[prec], ctypes.byref(b)))
    return b.value


def ism_simulate_batch(jobs: Sequence[ism_job], prec: str = "fp32", workspace: Optional[Workspace] = None,
                       stream=None):
    arr = jobs if isinstance(jobs, ctypes.Array) else (ism_job * len(jobs))(*jobs)
    b = ctypes.c_size_t()
    _check(load().ism_batch_workspace_size(arr, len(jobs), PRECISIONS[prec], ctypes.byref(b)))
    buf = _workspace(workspace, b.value)
    _check(load().ism_simulate_batch(arr, len(jobs), PRECISIONS[prec], ctypes.c_void_p(buf.data_ptr()),
                                     int(buf.numel()), _stream_ptr(stream)))
    return buf


def make_grad_job(job: ism_job, grad_out, grad_beta=None, grad_src=None, grad_rcv=None) -> ism_grad_job:
    """An ism_grad_job: the forward job plus CUDA tensors for dLoss/dh (read)
    and the three gradients (written); the tensors must stay alive."""
    g = ism_grad_job()
    g.job = job
    g.grad_out = grad_out.data_ptr()
    g.grad_beta = None if grad_beta is None else grad_beta.data_ptr()
    g.grad_src = None if grad_src is None else grad_src.data_ptr()
    g.grad_rcv = None if grad_rcv is None else grad_rcv.data_ptr()
    return g


def ism_backward_workspace_size(gjobs: Sequence[ism_grad_job]) -> int:
    arr = gjobs if isinstance(gjobs, ctypes.Array) else (ism_grad_job * len(gjobs))(*gjobs)
    b = ctypes.c_size_t()
    _check(load().ism_backward_workspace_size(arr, len(gjobs), ctypes.byref(b)))
    return b.value


def ism_simulate_backward_batch(gjobs: Sequence[ism_grad_job], workspace: Optional[Workspace] = None, stream=None):
    arr = gjobs if isinstance(gjobs, ctypes.Array) else (ism_grad_job * len(gjobs))(*gjobs)
    b = ctypes.c_size_t()
    _check(load().ism_backward_workspace_size(arr, len(gjobs), ctypes.byref(b)))
    buf = _workspace(workspace, b.value)
    _check(load().ism_simulate_backward_batch(arr, len(gjobs), ctypes.c_void_p(buf.data_ptr()), int(buf.numel()),
                                              _stream_ptr(stream)))
    return buf


def ism_simulate_backward(L, beta, pos_src, pos_rcv, nb_img, Tmax, fs, grad_out, Tdiff=0.0, Tw=0.0, c=343.0,
                          workspace: Optional[Workspace] = None, stream=None):
    """(grad_beta [6], grad_src [n_src, 3], grad_rcv [n_rcv, 3]) CUDA tensors for
    dLoss/dh = grad_out [n_src, n_rcv, n_S] through the image-source samples."""
    torch = _torch()
    dev = torch.device("cuda", torch.cuda.current_device())
    ps = torch.as_tensor(pos_src, dtype=torch.float32).to(dev).reshape(-1, 3).contiguous()
    pr = torch.as_tensor(pos_rcv, dtype=torch.float32).to(dev).reshape(-1, 3).contiguous()
    go = torch.as_tensor(grad_out, dtype=torch.float32).to(dev).contiguous()
    gb = torch.empty(6, dtype=torch.float32, device=dev)
    gs = torch.empty((ps.shape[0], 3), dtype=torch.float32, device=dev)
    gr = torch.empty((pr.shape[0], 3), dtype=torch.float32, device=dev)
    job = make_job(L, beta, ps, pr, nb_img, Tmax, fs, go, Tdiff=Tdiff, Tw=Tw, c=c)
    job.out = None
    gj = make_grad_job(job, go, gb, gs, gr)
    ism_simulate_backward_batch([gj], workspace=workspace, stream=stream)
    return gb, gs, gr


AURALIZE_METHODS = {"auto": 0, "direct": 1, "fft": 2}


def ism_auralize_workspace_size(n_x: int, n_points: int, n_mics: int, n_s: int, method: str = "auto") -> int:
    b = ctypes.c_size_t()
    _check(load().ism_auralize_workspace_size(int(n_x), int(n_points), int(n_mics), int(n_s),
                                              AURALIZE_METHODS[method], ctypes.byref(b)))
    return int(b.value)


def ism_auralize(signal, rirs, starts=None, out=None, stream=None, method: Optional[str] = None,
                 workspace: Optional[Workspace] = None):
    """Moving source (Section 4): signal [n_x] cut into one segment per
    trajectory point, each filtered by its point's RIRs rirs [n_points, n_mics,
    n_S] and overlap-added -> [n_mics, n_x + n_S - 1] (FP32 CUDA tensors).
    starts: optional [n_points] segment starts (default: uniform cut).
    method: None calls ism_auralize (direct form, no workspace); "auto",
    "direct" or "fft" call ism_auralize_ex with a workspace."""
    torch = _torch()
    dev = torch.device("cuda", torch.cuda.current_device())
    x = torch.as_tensor(signal, dtype=torch.float32).to(dev).reshape(-1).contiguous()
    h = torch.as_tensor(rirs, dtype=torch.float32).to(dev).contiguous()
    if h.dim() != 3:
        raise ValueError("rirs must be [n_points, n_mics, n_S]")
    n_points, n_mics, n_s = (int(v) for v in h.shape)
    st = None
    if starts is not None:
        st = torch.as_tensor(starts, dtype=torch.int32).to(dev).reshape(-1).contiguous()
        if st.numel() < n_points:
            raise ValueError("starts needs one entry per trajectory point")
    if out is None:
        out = torch.empty((n_mics, x.numel() + n_s - 1), dtype=torch.float32, device=dev)
    if method is not None:
        nbytes = ism_auralize_workspace_size(x.numel(), n_points, n_mics, n_s, method)
        buf = _workspace(workspace, nbytes) if nbytes else None
        _check(load().ism_auralize_ex(ctypes.c_void_p(x.data_ptr()), int(x.numel()), ctypes.c_void_p(h.data_ptr()),
                                      n_points, n_mics, n_s, None if st is None else ctypes.c_void_p(st.data_ptr()),
                                      ctypes.c_void_p(out.data_ptr()), AURALIZE_METHODS[method],
                                      None if buf is None else ctypes.c_void_p(buf.data_ptr()),
                                      0 if buf is None else int(buf.numel()), _stream_ptr(stream)))
        return out
    _check(load().ism_auralize(ctypes.c_void_p(x.data_ptr()), int(x.numel()), ctypes.c_void_p(h.data_ptr()), n_points,
                               n_mics, n_s, None if st is None else ctypes.c_void_p(st.data_ptr()),
                               ctypes.c_void_p(out.data_ptr()), _stream_ptr(stream)))
    return out


def ism_diffuse_noise(seed: int, rir: int, k0: int, n: int, stream=None):
    torch = _torch()
    z = torch.empty(int(n), dtype=torch.float32, device=torch.device("cuda", torch.cuda.current_device()))
    _check(load().ism_diffuse_noise(int(seed) & (2 ** 64 - 1), int(rir), int(k0), int(n), ctypes.c_void_p(z.data_ptr()),
                                    _stream_ptr(stream)))
    return z


# --------------------------------------------------------------------------- #
# Per-stage timing
# --------------------------------------------------------------------------- #
def ism_set_lanes(n_lanes: int):
    """1: every launch on the caller's stream; 2 (default): large calls run
    as two halves on two internal streams."""
    _check(load().ism_set_lanes(int(n_lanes)))
    _lanes_setting[0] = int(n_lanes)


def ism_profile_enable(enable: bool = True):
    _check(load().ism_profile_enable(int(bool(enable))))


def ism_profile_reset():
    _check(load().ism_profile_reset())


def ism_profile_read():
    """{stage: (total_ms, launches, calls)} accumulated since the last reset."""
    res = {}
    for i, name in enumerate(STAGES):
        ms, ln, cl = ctypes.c_double(), ctypes.c_longlong(), ctypes.c_longlong()
        _check(load().ism_profile_read(i, ctypes.byref(ms), ctypes.byref(ln), ctypes.byref(cl)))
        res[name] = (ms.value, ln.value, cl.value)
    return res


# --------------------------------------------------------------------------- #
# Serving
# --------------------------------------------------------------------------- #
class Server:
    """Continuous-batching RIR server (ism_server_*): submit host-side requests,
    wait for their RIRs.  The ctypes calls release the GIL, so submissions and
    waits from several Python threads run concurrently."""

    def __init__(self, hbm_budget: int = 4 << 30, host_budget: int = 0, max_inflight: int = 3, max_batch: int = 32,
                 device: int = 0, prec: str = "fp32"):
        cfg = ism_server_config(int(hbm_budget), int(host_budget), int(max_inflight), int(max_batch), int(device),
                                PRECISIONS[prec])
        h = ctypes.c_void_p()
        _check(load().ism_server_create(ctypes.byref(cfg), ctypes.byref(h)))
        self._h = h
        self._outs = {}
        self._lock = threading.Lock()

    def submit(self, L, beta, pos_src, pos_rcv, nb_img, Tmax, fs, Tdiff=0.0, Tw=0.0, c=343.0, seed=0,
               out: Optional[np.ndarray] = None, mic_pattern: str = "omni", orient_rcv=None,
               envelope: str = "sabine"):
        """Queues one room; returns (ticket, out) where `out` [n_src, n_rcv, n_S]
        FP32 receives the RIRs once the ticket is done."""
        ps = np.ascontiguousarray(np.asarray(pos_src, dtype=np.float32).reshape(-1, 3))
        pr = np.ascontiguousarray(np.asarray(pos_rcv, dtype=np.float32).reshape(-1, 3))
        n_S = ism_rir_length(Tmax, fs)
        if out is None:
            out = np.empty((ps.shape[0], pr.shape[0], n_S), dtype=np.float32)
        assert out.dtype == np.float32 and out.flags["C_CONTIGUOUS"] and out.size == ps.shape[0] * pr.shape[0] * n_S
        j = ism_job()
        j.room = _room(L, beta, c)
        j.pos_src = ps.ctypes.data
        j.n_src = ps.shape[0]
        j.pos_rcv = pr.ctypes.data
        j.n_rcv = pr.shape[0]
        for a in range(3):
            j.nb_img[a] = int(nb_img[a])
        j.Tmax, j.fs, j.Tdiff, j.Tw = float(Tmax), float(fs), float(Tdiff or 0.0), float(Tw or 0.0)
        j.seed = int(seed) & (2 ** 64 - 1)
        j.out = out.ctypes.data
        j.env_amp = None
        j.mic_pattern = MIC_PATTERNS[mic_pattern]
        j.envelope = ENVELOPES[envelope]
        orient = None
        if mic_pattern != "omni":
            orient = np.ascontiguousarray(np.asarray(orient_rcv, dtype=np.float32).reshape(-1, 3))
            j.orient_rcv = orient.ctypes.data   # copied by the server at submit
        t = ctypes.c_uint64()
        _check(load().ism_server_submit(self._h, ctypes.byref(j), ctypes.byref(t)))
        with self._lock:
            self._outs[t.value] = out
        return t.value, out

    def submit_many(self, reqs, outs=None):
        """Queues omnidirectional requests in one ism_server_submit_batch call.
        reqs: dicts with L, beta, pos_src, pos_rcv, nb_img, Tmax, fs and
        optionally Tdiff, Tw, c, seed.  outs: one FP32 array per request (or
        None: views of one new block).  Returns [(ticket, out)]."""
        n = len(reqs)
        if n == 0:
            return []
        arr = (ism_job * n)()
        v = np.frombuffer(arr, dtype=np.dtype(ism_job), count=n)
        v["room"]["L"] = np.array([r["L"] for r in reqs], np.float64).reshape(n, 3)
        v["room"]["beta"] = np.array([r["beta"] for r in reqs], np.float64).reshape(n, 6).astype(np.float32)
        v["room"]["c"] = [float(r.get("c", 343.0)) for r in reqs]
        ps = [np.asarray(r["pos_src"], np.float32).reshape(-1, 3) for r in reqs]
        pr = [np.asarray(r["pos_rcv"], np.float32).reshape(-1, 3) for r in reqs]
        ns = np.array([a.shape[0] for a in ps], np.int64)
        nr = np.array([a.shape[0] for a in pr], np.int64)
        # every request's positions in one host block (the server copies them in the call)
        pos = np.concatenate([x for a, b in zip(ps, pr) for x in (a.ravel(), b.ravel())])
        off = np.concatenate([[0], np.cumsum(3 * (ns + nr))[:-1]]).astype(np.uint64)
        base = np.uint64(pos.ctypes.data)
        v["pos_src"] = base + off * np.uint64(4)
        v["pos_rcv"] = base + (off + np.uint64(3) * ns.astype(np.uint64)) * np.uint64(4)
        v["n_src"], v["n_rcv"] = ns, nr
        v["nb_img"] = np.array([r["nb_img"] for r in reqs], np.int32).reshape(n, 3)
        for f, d in (("Tmax", None), ("fs", None), ("Tdiff", 0.0), ("Tw", 0.0)):
            v[f] = [float(r[f] if d is None else (r.get(f) or d)) for r in reqs]
        v["seed"] = [int(r.get("seed", 0)) & (2 ** 64 - 1) for r in reqs]
        v["envelope"] = [ENVELOPES[r.get("envelope", "sabine")] for r in reqs]
        lens = {}
        n_S = np.array([lens.setdefault((r["Tmax"], r["fs"]), ism_rir_length(r["Tmax"], r["fs"])) for r in reqs],
                       np.int64)
        sizes = ns * nr * n_S
        if outs is None:
            block = np.empty(int(sizes.sum()), np.float32)
            cuts = np.cumsum(sizes)[:-1]
            outs = [b.reshape(a, c, m) for b, a, c, m in zip(np.split(block, cuts), ns, nr, n_S)]
        for o, sz in zip(outs, sizes):
            assert o.dtype == np.float32 and o.flags["C_CONTIGUOUS"] and o.size == sz
        v["out"] = [o.ctypes.data for o in outs]
        t = (ctypes.c_uint64 * n)()
        _check(load().ism_server_submit_batch(self._h, arr, n, t))
        with self._lock:
            for k in range(n):
                self._outs[t[k]] = outs[k]
        return list(zip(list(t), outs))

    def poll(self, ticket: int) -> bool:
        d = ctypes.c_int()
        _check(load().ism_server_poll(self._h, ctypes.c_uint64(ticket), ctypes.byref(d)))
        return bool(d.value)

    def wait(self, ticket: int, timeout_s: float = -1.0) -> float:
        """Blocks until the request is done; returns its submit-to-ready latency
        in seconds.  Raises IsmError with the request's status if it failed
        (ISM_ERR_TIMEOUT leaves the ticket valid)."""
        lat = ctypes.c_double()
        st = load().ism_server_wait(self._h, ctypes.c_uint64(ticket), float(timeout_s), ctypes.byref(lat))
        if st != ISM_ERR_TIMEOUT_CODE:
            with self._lock:
                self._outs.pop(ticket, None)
        _check(st)
        return lat.value

    def stats(self) -> dict:
        s = ism_server_stats()
        _check(load().ism_server_stats_read(self._h, ctypes.byref(s)))
        return {k: getattr(s, k) for k, _ in ism_server_stats._fields_}

    def close(self):
        if self._h:
            _check(load().ism_server_destroy(self._h))
            self._h = None
            self._outs.clear()

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
