"""Thin Python binding of libbfgc (include/bfgc.h): same names, argument marshalling only.

Every computation happens in the CUDA kernels behind the C ABI.  PyTorch supplies
device memory (tensors) and streams; nothing here falls back to the CPU: if the
library cannot be built or loaded, the first call raises.
"""
import ctypes
import os
import threading

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libbfgc.so")

BF_OK, BF_ERR_INVALID_ARG, BF_ERR_UNSUPPORTED, BF_ERR_NOMEM, BF_ERR_CUDA, BF_ERR_TIMEOUT, \
    BF_ERR_RANGE, BF_ERR_WORKSPACE = range(8)
BF_OPT_FORM, BF_OPT_PRECISION, BF_OPT_RANGE_L, BF_OPT_RANGE_U, BF_OPT_POLY, BF_OPT_SAVE_CHANNELS, \
    BF_OPT_TILE_W, BF_OPT_REFINE, BF_OPT_WAIT_US, BF_OPT_STALL = range(1, 11)
BF_FORM_PLAIN, BF_FORM_FUSED_TC, BF_FORM_RECURSIVE, BF_FORM_AUTO, BF_FORM_FUSED = range(5)
BF_AUTO_FP32_EXACT_MAX_R = 140
BF_PREC_FP32, BF_PREC_BF16, BF_PREC_FP16 = range(3)
BF_POLY_CHEBYSHEV, BF_POLY_TAYLOR = range(2)
BF_MAX_N = 62

FORMS = {"plain": BF_FORM_PLAIN, "fused": BF_FORM_FUSED, "fused_tc": BF_FORM_FUSED_TC, "recursive": BF_FORM_RECURSIVE,
         "auto": BF_FORM_AUTO}
PRECISIONS = {"fp32": BF_PREC_FP32, "bf16": BF_PREC_BF16, "fp16": BF_PREC_FP16}
POLYS = {"chebyshev": BF_POLY_CHEBYSHEV, "taylor": BF_POLY_TAYLOR}


class bf_gc_info(ctypes.Structure):
    _fields_ = [("H", ctypes.c_int), ("W", ctypes.c_int), ("N", ctypes.c_int), ("R", ctypes.c_int),
                ("C", ctypes.c_int), ("form", ctypes.c_int), ("precision", ctypes.c_int),
                ("poly", ctypes.c_int), ("sigma_s", ctypes.c_double), ("sigma_r", ctypes.c_double),
                ("L", ctypes.c_double), ("U", ctypes.c_double), ("t_c", ctypes.c_double),
                ("s_r", ctypes.c_double), ("mu", ctypes.c_double), ("kappa", ctypes.c_double),
                ("fit_err", ctypes.c_double), ("c", ctypes.c_double * (BF_MAX_N + 1)),
                ("c_tilde", ctypes.c_double * (BF_MAX_N + 1))]


class bf_gc_diag(ctypes.Structure):
    _fields_ = [("n_guarded", ctypes.c_ulonglong), ("n_illcond", ctypes.c_ulonglong),
                ("error_flags", ctypes.c_uint), ("n_refined", ctypes.c_ulonglong),
                ("n_refined_fp64", ctypes.c_ulonglong)]


class bf_kernel_time(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 32), ("total_ms", ctypes.c_double), ("launches", ctypes.c_ulonglong)]


# name -> (restype, argtypes) for every entry point of include/bfgc.h
_P, _I, _D, _SZ = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_size_t
SIGNATURES = {
    "bf_gc_plan": (_I, [_I, _I, _D, _D, _I, ctypes.POINTER(_P)]),
    "bf_gc_plan_set": (_I, [_P, _I, _D]),
    "bf_gc_plan_info": (_I, [_P, ctypes.POINTER(bf_gc_info)]),
    "bf_gc_workspace_size": (_I, [_P, ctypes.POINTER(_SZ), ctypes.POINTER(_SZ)]),
    "bf_gc_forward": (_I, [_P, _P, _P, _P, _SZ, _P]),
    "bf_gc_forward_host": (_I, [_P, _P, _P, _P, _P, _P, _SZ, _P]),
    "bf_gc_forward_static": (_I, [_P, _P, _P, _P]),
    "bf_gc_stream_bytes": (_I, [_P, ctypes.POINTER(_SZ)]),
    "bf_gc_forward_host_stream": (_I, [_P, _I, ctypes.POINTER(_P), ctypes.POINTER(_P), _P, _SZ, _P]),
    "bf_gc_backward": (_I, [_P, _P, _P, _P, _P, _P, _SZ, _P]),
    "bf_gc_diagnostics": (_I, [_P, _P, ctypes.POINTER(bf_gc_diag), _P]),
    "bf_gc_plan_destroy": (None, [_P]),
    "bf_gc_profile_enable": (_I, [_P, _I]),
    "bf_gc_profile_read": (_I, [_P, ctypes.POINTER(bf_kernel_time), _I, ctypes.POINTER(_I)]),
    "bf_gc_batch_create": (_I, [_I, ctypes.POINTER(_P), _I, ctypes.POINTER(_P)]),
    "bf_gc_batch_create_persistent": (_I, [_I, ctypes.POINTER(_P), ctypes.POINTER(_P)]),
    "bf_gc_batch_workspace_size": (_I, [_P, ctypes.POINTER(_SZ)]),
    "bf_gc_batch_info": (_I, [_P, ctypes.POINTER(_I), ctypes.POINTER(_I)]),
    "bf_gc_batch_forward": (_I, [_P, ctypes.POINTER(_P), ctypes.POINTER(_P), _P, _SZ, _P]),
    "bf_gc_batch_destroy": (None, [_P]),
    "bf_direct": (_I, [_I, _I, _D, _D, _P, _P, _P]),
    "bf_check_range": (_I, [_I, _I, _D, _D, _P, _P, _P]),
    "bf_status_string": (ctypes.c_char_p, [_I]),
    "bf_version": (ctypes.c_char_p, []),
    "bf_last_cuda_error": (_I, [ctypes.POINTER(ctypes.c_char_p)]),
}

_lib = None
_lock = threading.Lock()


def lib():
    """Load libbfgc.so, building it first if it is missing or older than its sources."""
    global _lib
    if _lib is None:
        with _lock:
            if _lib is None:
                from .csrc import build as _build
                if not _build.up_to_date():
                    _build.build()
                L = ctypes.CDLL(LIB_PATH)
                for name, (res, args) in SIGNATURES.items():
                    fn = getattr(L, name)
                    fn.restype = res
                    fn.argtypes = args
                _lib = L
    return _lib


class BfError(RuntimeError):
    def __init__(self, status, what):
        msg = lib().bf_status_string(status).decode()
        if status == BF_ERR_CUDA:
            code, name = bf_last_cuda_error()
            msg += f" [{name} ({code})]"
        super().__init__(f"{what}: {msg} (status {status})")
        self.status = status


def _check(status, what):
    if status != BF_OK:
        raise BfError(status, what)


def _ptr(t):
    if t is None:
        return None
    if isinstance(t, torch.Tensor):
        return ctypes.c_void_p(t.data_ptr())
    return ctypes.c_void_p(int(t))


def _stream(stream):
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))


def _dev_f32(t, name, numel=None):
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float32 and t.is_contiguous()):
        raise ValueError(f"{name} must be a contiguous float32 CUDA tensor")
    if numel is not None and t.numel() != numel:
        raise ValueError(f"{name} must hold {numel} elements (H x W of the plan), not {t.numel()}")
    return t


def _dev_ws(ws):
    if not (isinstance(ws, torch.Tensor) and ws.is_cuda and ws.is_contiguous()):
        raise ValueError("the workspace must be a contiguous CUDA tensor")
    return ws


def _plan_px(plan):
    i = bf_gc_plan_info(plan)
    return i.H * i.W


# ----------------------------------------------------------------------------- C-ABI mirrors
def bf_gc_plan(H, W, sigma_s, sigma_r, N):
    h = ctypes.c_void_p()
    _check(lib().bf_gc_plan(int(H), int(W), float(sigma_s), float(sigma_r), int(N), ctypes.byref(h)),
           "bf_gc_plan")
    return h


def bf_gc_plan_set(plan, option, value):
    _check(lib().bf_gc_plan_set(plan, int(option), float(value)), "bf_gc_plan_set")


def bf_gc_plan_info(plan):
    info = bf_gc_info()
    _check(lib().bf_gc_plan_info(plan, ctypes.byref(info)), "bf_gc_plan_info")
    return info


def bf_gc_workspace_size(plan):
    fwd, bwd = ctypes.c_size_t(), ctypes.c_size_t()
    _check(lib().bf_gc_workspace_size(plan, ctypes.byref(fwd), ctypes.byref(bwd)), "bf_gc_workspace_size")
    return fwd.value, bwd.value


def bf_gc_forward(plan, f, out, ws, stream=None):
    px = _plan_px(plan)
    _dev_f32(f, "f", px)
    _dev_f32(out, "out", px)
    _dev_ws(ws)
    _check(lib().bf_gc_forward(plan, _ptr(f), _ptr(out), _ptr(ws), ws.numel() * ws.element_size(),
                               _stream(stream)), "bf_gc_forward")
    return out


def bf_gc_forward_host(plan, h_f, h_out, d_f, d_out, ws, stream=None):
    _check(lib().bf_gc_forward_host(plan, _ptr(h_f), _ptr(h_out), _ptr(d_f), _ptr(d_out), _ptr(ws),
                                    ws.numel() * ws.element_size(), _stream(stream)), "bf_gc_forward_host")
    return h_out


def bf_gc_stream_bytes(plan):
    n = ctypes.c_size_t()
    _check(lib().bf_gc_stream_bytes(plan, ctypes.byref(n)), "bf_gc_stream_bytes")
    return n.value


def bf_gc_forward_host_stream(plan, h_fs, h_outs, scratch, stream=None):
    """Streaming forward of host images (float32 CPU tensors, preferably pinned) into h_outs."""
    if len(h_fs) != len(h_outs) or not h_fs:
        raise ValueError("h_fs and h_outs must be non-empty and of equal length")
    pf = (_P * len(h_fs))(*[t.data_ptr() for t in h_fs])
    po = (_P * len(h_outs))(*[t.data_ptr() for t in h_outs])
    _check(lib().bf_gc_forward_host_stream(plan, len(h_fs), pf, po, _ptr(scratch),
                                           scratch.numel() * scratch.element_size(), _stream(stream)),
           "bf_gc_forward_host_stream")
    return h_outs


BF_STATIC_SCRATCH_BYTES = 64 << 20


def bf_gc_forward_static(plan, f, out, stream=None):
    """Forward with the library's fixed device scratch; allocates nothing (see bfgc.h)."""
    px = _plan_px(plan)
    _dev_f32(f, "f", px)
    _dev_f32(out, "out", px)
    _check(lib().bf_gc_forward_static(plan, _ptr(f), _ptr(out), _stream(stream)), "bf_gc_forward_static")
    return out


def bf_gc_backward(plan, f, gout, gf, gsigma_r, ws, stream=None):
    """dL/df into gf (and dL/dsigma_r into gsigma_r, a one-element float64 CUDA tensor, or None)."""
    px = _plan_px(plan)
    _dev_f32(f, "f", px)
    _dev_f32(gout, "gout", px)
    _dev_f32(gf, "gf", px)
    if gsigma_r is not None and not (isinstance(gsigma_r, torch.Tensor) and gsigma_r.is_cuda and
                                     gsigma_r.dtype == torch.float64 and gsigma_r.numel() == 1):
        raise ValueError("gsigma_r must be a one-element float64 CUDA tensor or None")
    _dev_ws(ws)
    _check(lib().bf_gc_backward(plan, _ptr(f), _ptr(gout), _ptr(gf), _ptr(gsigma_r), _ptr(ws),
                                ws.numel() * ws.element_size(), _stream(stream)), "bf_gc_backward")
    return gf


def bf_gc_diagnostics(plan, ws, stream=None):
    d = bf_gc_diag()
    st = lib().bf_gc_diagnostics(plan, _ptr(ws), ctypes.byref(d), _stream(stream))
    if st not in (BF_OK, BF_ERR_TIMEOUT):
        _check(st, "bf_gc_diagnostics")
    return {"n_guarded": d.n_guarded, "n_illcond": d.n_illcond, "error_flags": d.error_flags,
            "n_refined": d.n_refined, "n_refined_fp64": d.n_refined_fp64}


def bf_gc_plan_destroy(plan):
    lib().bf_gc_plan_destroy(plan)


def bf_gc_profile_enable(plan, enable=True):
    _check(lib().bf_gc_profile_enable(plan, 1 if enable else 0), "bf_gc_profile_enable")


def bf_gc_profile_read(plan):
    """{kernel name: (total ms, launches)} since the last enable (waits for the events)."""
    buf = (bf_kernel_time * 32)()
    n = ctypes.c_int(0)
    _check(lib().bf_gc_profile_read(plan, buf, 32, ctypes.byref(n)), "bf_gc_profile_read")
    return {buf[i].name.decode(): (buf[i].total_ms, buf[i].launches) for i in range(min(n.value, 32))}


def bf_gc_batch_create(plans, branches):
    arr = (_P * len(plans))(*[p.value if isinstance(p, ctypes.c_void_p) else p for p in plans])
    h = ctypes.c_void_p()
    _check(lib().bf_gc_batch_create(len(plans), arr, int(branches), ctypes.byref(h)), "bf_gc_batch_create")
    return h


def bf_gc_batch_create_persistent(plans):
    arr = (_P * len(plans))(*[p.value if isinstance(p, ctypes.c_void_p) else p for p in plans])
    h = ctypes.c_void_p()
    _check(lib().bf_gc_batch_create_persistent(len(plans), arr, ctypes.byref(h)), "bf_gc_batch_create_persistent")
    return h


def bf_gc_batch_workspace_size(batch):
    n = ctypes.c_size_t()
    _check(lib().bf_gc_batch_workspace_size(batch, ctypes.byref(n)), "bf_gc_batch_workspace_size")
    return n.value


def bf_gc_batch_info(batch, count):
    """(branch of each image, graphs captured so far)."""
    br = (_I * count)()
    cap = _I(0)
    _check(lib().bf_gc_batch_info(batch, br, ctypes.byref(cap)), "bf_gc_batch_info")
    return list(br), cap.value


def bf_gc_batch_forward(batch, fs, outs, ws, stream=None):
    if len(fs) != len(outs):
        raise ValueError("fs and outs differ in length")
    for f, o in zip(fs, outs):
        _dev_f32(f, "f")
        _dev_f32(o, "out", f.numel())
    _dev_ws(ws)
    pf = (_P * len(fs))(*[t.data_ptr() for t in fs])
    po = (_P * len(outs))(*[t.data_ptr() for t in outs])
    _check(lib().bf_gc_batch_forward(batch, pf, po, _ptr(ws), ws.numel() * ws.element_size(), _stream(stream)),
           "bf_gc_batch_forward")
    return outs


def bf_gc_batch_destroy(batch):
    lib().bf_gc_batch_destroy(batch)


def bf_direct(f, sigma_s, sigma_r, out=None, stream=None):
    _dev_f32(f, "f")
    out = torch.empty_like(f) if out is None else _dev_f32(out, "out", f.numel())
    H, W = f.shape[-2], f.shape[-1]
    _check(lib().bf_direct(H, W, float(sigma_s), float(sigma_r), _ptr(f), _ptr(out), _stream(stream)),
           "bf_direct")
    return out


def bf_check_range(f, L=0.0, U=255.0, stream=None):
    """(pixels outside [L, U], non-finite pixels) of the device image f, after a stream sync."""
    _dev_f32(f, "f")
    H, W = f.shape[-2], f.shape[-1]
    counts = torch.empty(2, dtype=torch.int64, device=f.device)
    _check(lib().bf_check_range(H, W, float(L), float(U), _ptr(f), _ptr(counts), _stream(stream)),
           "bf_check_range")
    c = counts.cpu()
    return int(c[0]), int(c[1])


def bf_status_string(status):
    return lib().bf_status_string(int(status)).decode()


def bf_version():
    return lib().bf_version().decode()


def bf_last_cuda_error():
    """(code, name) of the CUDA error behind the last BF_ERR_CUDA of this thread."""
    name = ctypes.c_char_p()
    code = lib().bf_last_cuda_error(ctypes.byref(name))
    return code, (name.value or b"").decode()
