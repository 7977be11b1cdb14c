"""ctypes binding of libtnrd.so (include/tnrd.h) -- argument marshalling only.

Every step of the stage runs in the library's CUDA kernels; this module turns
torch CUDA tensors into the pointers, sizes and stream handle of the C calls
and raises on a non-OK status.  It never computes anything itself and has no
CPU fallback: if the shared library is missing it raises.
"""
from __future__ import annotations

import ctypes
import os
import threading

PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(PKG, "_build", "libtnrd.so")

TNRD_OK = 0
STATUS_NAMES = {0: "TNRD_OK", 1: "TNRD_ERR_INVALID_ARG", 2: "TNRD_ERR_UNSUPPORTED",
                3: "TNRD_ERR_CUDA", 4: "TNRD_ERR_TIMEOUT", 5: "TNRD_ERR_WORKSPACE"}

ALGO = {"fused": 0, "unfused": 1, "tf32": 2, "bf16": 3, "tf32x3": 4}
OP_FORWARD, OP_BACKWARD = 0, 1

# Every symbol include/tnrd.h declares (checked by the tests).
EXPORTS = ["tnrd_workspace_size", "tnrd_forward", "tnrd_backward", "tnrd_plan_create",
           "tnrd_batch_forward", "tnrd_plan_status", "tnrd_plan_set_wait_limit",
           "tnrd_plan_tile_height", "tnrd_plan_tile_width", "tnrd_plan_launches",
           "tnrd_plan_destroy",
           "tnrd_forward_noalloc", "tnrd_forward_kernel", "tnrd_quality_workspace_size",
           "tnrd_quality", "tnrd_device_status", "tnrd_stage_wait_test", "tnrd_last_error",
           "tnrd_version"]

# Largest N * H * pitch (floats) tnrd_forward_noalloc accepts (TNRD_NOALLOC_MAX_FLOATS).
NOALLOC_MAX_FLOATS = 1 << 22


class TnrdError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class tnrd_params(ctypes.Structure):
    _fields_ = [("T", ctypes.c_int), ("ksize", ctypes.c_int), ("nfilt", ctypes.c_int),
                ("nrbf", ctypes.c_int), ("rbf_mu0", ctypes.c_float),
                ("rbf_delta", ctypes.c_float), ("rbf_gamma", ctypes.c_float),
                ("filters", ctypes.c_void_p), ("rbf_w", ctypes.c_void_p),
                ("lambda_", ctypes.c_void_p), ("data_term", ctypes.c_int),
                ("proj_c", ctypes.c_float)]


# tnrd_data_term
DATA_TERM = {"idiv": 0, "gauss": 1, "proj": 2}


class tnrd_image(ctypes.Structure):
    _fields_ = [("f", ctypes.c_void_p), ("u", ctypes.c_void_p), ("H", ctypes.c_int),
                ("W", ctypes.c_int), ("pitch", ctypes.c_int), ("param_set", ctypes.c_int)]


_lock = threading.Lock()
_lib = None


def load(path: str = LIB_PATH):
    """Load libtnrd.so and declare the C signatures."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(path):
            raise RuntimeError(f"libtnrd.so not found at {path}: the CUDA library must be "
                               "built first (paper_1702_07482_gb300.build.build())")
        L = ctypes.CDLL(path)
        P, i, sz = ctypes.c_void_p, ctypes.c_int, ctypes.c_size_t
        pp = ctypes.POINTER(tnrd_params)
        L.tnrd_workspace_size.restype = sz
        L.tnrd_workspace_size.argtypes = [i, pp, i, i, i, i, i, i]
        L.tnrd_forward.restype = i
        L.tnrd_forward.argtypes = [pp, i, i, i, i, P, P, i, i, P, sz, P]
        L.tnrd_backward.restype = i
        L.tnrd_backward.argtypes = [pp, i, i, i, i, P, P, P, P, P, P, P, i, P, sz, P]
        L.tnrd_plan_create.restype = i
        L.tnrd_plan_create.argtypes = [ctypes.POINTER(ctypes.c_void_p), ctypes.POINTER(tnrd_image),
                                       i, pp, i, i, i, P]
        L.tnrd_batch_forward.restype = i
        L.tnrd_batch_forward.argtypes = [P, P]
        L.tnrd_plan_status.restype = i
        L.tnrd_plan_status.argtypes = [P]
        L.tnrd_plan_set_wait_limit.restype = i
        L.tnrd_plan_set_wait_limit.argtypes = [P, ctypes.c_longlong]
        L.tnrd_plan_tile_height.restype = i
        L.tnrd_plan_tile_height.argtypes = [P]
        L.tnrd_plan_tile_width.restype = i
        L.tnrd_plan_tile_width.argtypes = [P]
        L.tnrd_plan_launches.restype = i
        L.tnrd_plan_launches.argtypes = [P]
        L.tnrd_plan_destroy.restype = None
        L.tnrd_plan_destroy.argtypes = [P]
        L.tnrd_forward_noalloc.restype = i
        L.tnrd_forward_noalloc.argtypes = [pp, i, i, i, i, P, P, P]
        L.tnrd_forward_kernel.restype = i
        L.tnrd_forward_kernel.argtypes = [pp, i, i, i, i, ctypes.c_char_p, sz]
        L.tnrd_quality_workspace_size.restype = sz
        L.tnrd_quality_workspace_size.argtypes = [i, i, i]
        L.tnrd_quality.restype = i
        L.tnrd_quality.argtypes = [P, P, P, i, i, i, i, ctypes.c_float, P, P, sz, P]
        L.tnrd_device_status.restype = i
        L.tnrd_device_status.argtypes = []
        L.tnrd_stage_wait_test.restype = i
        L.tnrd_stage_wait_test.argtypes = [ctypes.c_longlong, i]
        L.tnrd_last_error.restype = ctypes.c_char_p
        L.tnrd_last_error.argtypes = []
        L.tnrd_version.restype = i
        L.tnrd_version.argtypes = []
        _lib = L
        return _lib


def last_error() -> str:
    return load().tnrd_last_error().decode()


def check(status: int) -> None:
    if status != TNRD_OK:
        raise TnrdError(status, last_error())


def version() -> int:
    return load().tnrd_version()


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def make_params(model) -> tnrd_params:
    """tnrd_params from a model holding device float32 tensors (see ops.Model)."""
    p = tnrd_params()
    p.T, p.ksize, p.nfilt, p.nrbf = model.T, model.ksize, model.nfilt, model.nrbf
    p.rbf_mu0, p.rbf_delta, p.rbf_gamma = model.mu0, model.delta, model.gamma
    p.filters = model.filters.data_ptr()
    p.rbf_w = model.rbf_w.data_ptr()
    p.lambda_ = model.lam.data_ptr()
    p.data_term = int(getattr(model, "data_term", 0))
    p.proj_c = float(getattr(model, "proj_c", 1.0))
    return p


def tnrd_workspace_size(op: int, params: tnrd_params, N: int, H: int, W: int, pitch: int,
                        keep_stages: int, algo: int) -> int:
    return load().tnrd_workspace_size(op, ctypes.byref(params), N, H, W, pitch,
                                      keep_stages, algo)


def tnrd_forward(params: tnrd_params, N, H, W, pitch, f, u, keep_stages, algo,
                 workspace, workspace_bytes, stream) -> None:
    check(load().tnrd_forward(ctypes.byref(params), N, H, W, pitch, _ptr(f), _ptr(u),
                              int(keep_stages), int(algo), _ptr(workspace),
                              int(workspace_bytes), ctypes.c_void_p(stream)))


def tnrd_backward(params: tnrd_params, N, H, W, pitch, f, u_stages, grad_uT, grad_u0,
                  grad_filters, grad_rbf_w, grad_lambda, algo, workspace,
                  workspace_bytes, stream) -> None:
    check(load().tnrd_backward(ctypes.byref(params), N, H, W, pitch, _ptr(f), _ptr(u_stages),
                               _ptr(grad_uT), _ptr(grad_u0), _ptr(grad_filters),
                               _ptr(grad_rbf_w), _ptr(grad_lambda), int(algo),
                               _ptr(workspace), int(workspace_bytes), ctypes.c_void_p(stream)))


def tnrd_forward_noalloc(params: tnrd_params, N, H, W, pitch, f, u, stream) -> None:
    """Forward cascade (keep_stages 0, fused) with the library's built-in
    scratch instead of a workspace; for callers that cannot allocate."""
    check(load().tnrd_forward_noalloc(ctypes.byref(params), N, H, W, pitch, _ptr(f), _ptr(u),
                                      ctypes.c_void_p(stream)))


class Plan:
    """Owns a tnrd_plan (tnrd_plan_create ... tnrd_plan_destroy)."""

    def __init__(self, images, sets, algo=0, autotune=False, stream=0):
        arr = (tnrd_image * len(images))(*images)
        parr = (tnrd_params * len(sets))(*sets)
        self._keep = (arr, parr)
        self.handle = ctypes.c_void_p()
        check(load().tnrd_plan_create(ctypes.byref(self.handle), arr, len(images), parr,
                                      len(sets), int(algo), int(bool(autotune)),
                                      ctypes.c_void_p(stream)))

    def forward(self, stream) -> None:
        check(load().tnrd_batch_forward(self.handle, ctypes.c_void_p(stream)))

    def status(self) -> int:
        return load().tnrd_plan_status(self.handle)

    def set_wait_limit(self, cycles: int) -> None:
        check(load().tnrd_plan_set_wait_limit(self.handle, int(cycles)))

    @property
    def tile_height(self) -> int:
        return load().tnrd_plan_tile_height(self.handle)

    @property
    def tile_width(self) -> int:
        """Tile width: 32 - 2R, or 64 - 2R for the column-pair schedule."""
        return load().tnrd_plan_tile_width(self.handle)

    @property
    def launches(self) -> int:
        """Kernel launches per forward: 1 (persistent) or T (one per stage)."""
        return load().tnrd_plan_launches(self.handle)

    def close(self) -> None:
        if self.handle:
            load().tnrd_plan_destroy(self.handle)
            self.handle = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def tnrd_forward_kernel(params, N: int, H: int, W: int, algo: int) -> str:
    """Name and tile geometry of the stage kernel tnrd_forward would launch."""
    buf = ctypes.create_string_buffer(160)
    check(load().tnrd_forward_kernel(ctypes.byref(params), N, H, W, algo, buf, len(buf)))
    return buf.value.decode()


QUALITY_NAMES = ("psnr", "mssim", "ec", "ri_mean", "ri_var", "cv")
QUALITY_COUNT = len(QUALITY_NAMES)   # TNRD_QUALITY_COUNT


def tnrd_quality_workspace_size(N: int, H: int, W: int) -> int:
    return int(load().tnrd_quality_workspace_size(N, H, W))


def tnrd_quality(ref, img, noisy, N, H, W, pitch, peak, out, workspace, workspace_bytes,
                 stream) -> None:
    """Quality indexes into out (device [N][6] float64); ref / noisy may be None."""
    check(load().tnrd_quality(_ptr(ref), _ptr(img), _ptr(noisy), N, H, W, pitch, float(peak),
                              _ptr(out), _ptr(workspace), int(workspace_bytes),
                              ctypes.c_void_p(stream)))


def tnrd_device_status() -> int:
    """Synchronous: 0, or TNRD_ERR_TIMEOUT if a tensor-core stage gave up waiting."""
    return load().tnrd_device_status()


def tnrd_stage_wait_test(cycles: int, never_complete: bool) -> None:
    """Test hook: wait limit of the fused stages' tile copies, and whether every
    copy's wait is made to run out (see include/tnrd.h)."""
    check(load().tnrd_stage_wait_test(int(cycles), int(bool(never_complete))))
